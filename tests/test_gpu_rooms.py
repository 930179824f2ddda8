"""RIRs generated where they are consumed (Eq. 1 into Eq. 7-9 and Eq. 2):
rsim_filter_mix_rooms against the FP64 oracle and against the two-call path.

The fused path lands every image of an RIR in shared memory, cuts it there and
keeps only the taps [0, L).  Checks:
* the generated taps (asked for through rir_out) are the oracle's image-method
  RIRs, near-integer images settled (image_checks);
* the cut-off lengths are exact wherever no tap sits within 1e-5 of the Eq. 7
  threshold, and a valid Eq. 8 cut otherwise;
* the two-call path (the same taps through rsim_filter_mix) gives bitwise the
  same lengths and mix (one cut-off decision, the same kept taps, the same
  spectra) and the kept-energy fractions within 1e-6 (their sums are rounded
  in another order);
* the mix and the gradients are the oracle's at the kernel's lengths, per
  channel, source and RIR within a relative L2 of 1e-5 and a max-abs of
  1e-5 x peak.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from image_checks import _near_threshold, _valid_cut, check_rir, settle
from paper_1712_03439_gb300 import synth
from parity_checks import close_vec, grads_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_03439_gb300 import build
    build.build()


def dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def rooms_batch(seed=50, n_utts=6, rt60=(0.1, 0.7)):
    b = synth.config_home(seed=synth.SEED_BASE + seed, n_utts=n_utts)
    geom, rir_len, _ = synth.room_geometry(synth.SEED_BASE + seed + 1, b.num_sources, synth.linear_pair_array(),
                                           rt60_range=rt60)
    b = dataclasses.replace(b, rir_len=rir_len, rir=np.zeros(int(rir_len.sum()), np.float32))
    return b, np.ascontiguousarray(geom, np.float32)


def run_rooms(b, geom, eta, gain_mode=1, gains=None, graphs=True, order=8):
    from paper_1712_03439_gb300 import Plan
    plan = Plan.for_batch(b, eta_db=eta, gain_mode=gain_mode, rooms=True, graphs=graphs)
    out = dict(x=dev(b.x), geom=dev(geom), y=torch.full((plan.y_size,), float("nan"), device="cuda"),
               tl=torch.empty(plan.R, dtype=torch.int32, device="cuda"),
               ekf=torch.empty(plan.R, device="cuda"), rir=torch.full((plan.rir_size,), float("nan"), device="cuda"))
    out["gains"] = dev(gains) if gains is not None else torch.empty(plan.G, device="cuda")
    plan.filter_mix_rooms(out["x"], out["geom"], out["gains"], out["y"], snr_db=dev(b.snr_db) if gain_mode == 0 else None,
                          trunc_len=out["tl"], energy_kept_frac=out["ekf"], rir_out=out["rir"], order=order)
    plan.sync_status()
    return plan, out


def settled(b, geom, h_gpu, order=8):
    off = b.rir_offsets()
    return np.concatenate([settle(h_gpu[off[r]:off[r + 1]], geom[r], int(b.rir_len[r]), order, 16000.0, 343.0)[0]
                           for r in range(b.num_rirs)])


def check_lengths(b, h_or, L, eta):
    off = b.rir_offsets()
    bo = dataclasses.replace(b, rir=h_or.astype(np.float32))
    L_or = oracle.truncate_batch(bo, eta)["L"]
    for r in range(b.num_rirs):
        h = h_or[off[r]:off[r + 1]]
        if _near_threshold(h, eta):
            assert _valid_cut(h, int(L[r]), eta), f"RIR {r}: cut {L[r]} is no reading of Eq. 8"
        else:
            assert L[r] == L_or[r], f"RIR {r}: cut {L[r]} vs {L_or[r]}"
    return bo


@pytest.mark.parametrize("eta", [20.0, 10.0, math.inf])
def test_fused_rooms_forward_matches_oracle_and_the_two_call_path(eta):
    from paper_1712_03439_gb300 import Plan
    b, geom = rooms_batch()
    S = int(b.num_sources.sum())
    alpha = np.linspace(0.4, 1.2, S).astype(np.float32)
    plan, out = run_rooms(b, geom, eta, gains=alpha)
    h_gpu = out["rir"].cpu().numpy()
    h_or = settled(b, geom, h_gpu)
    off = b.rir_offsets()
    for r in range(b.num_rirs):
        check_rir(h_gpu[off[r]:off[r + 1]], h_or[off[r]:off[r + 1]], f"RIR {r}")
    L = out["tl"].cpu().numpy()
    bo = check_lengths(b, h_or, L, eta)
    # the two-call path on the same taps: bitwise the same
    p2 = Plan.for_batch(b, eta_db=eta, gain_mode=1)
    y2 = torch.empty(p2.y_size, device="cuda")
    tl2 = torch.empty(p2.R, dtype=torch.int32, device="cuda")
    ekf2 = torch.empty(p2.R, device="cuda")
    p2.filter_mix(out["x"], out["rir"], out["gains"], y2, trunc_len=tl2, energy_kept_frac=ekf2)
    p2.sync_status()
    np.testing.assert_array_equal(tl2.cpu().numpy(), L)
    np.testing.assert_array_equal(y2.cpu().numpy(), out["y"].cpu().numpy())
    # the energy sums run over different thread counts (another rounding order)
    np.testing.assert_allclose(ekf2.cpu().numpy(), out["ekf"].cpu().numpy(), rtol=1e-6)
    # the mix against the oracle at the kernel's lengths
    want = oracle.forward_with_lengths(bo, L.astype(np.int64), alpha.astype(np.float64))
    yo = b.y_offsets()
    y = out["y"].cpu().numpy()
    for u in range(b.num_utts):
        n = int(b.num_samples[u])
        for j in range(b.num_mics):
            s = slice(int(yo[u]) + j * n, int(yo[u]) + (j + 1) * n)
            close_vec(y[s], want[s], f"y u={u} j={j}")
    # kept energy against the oracle's bookkeeping on the settled RIRs
    tr = oracle.truncate_batch(bo, eta)
    sure = np.array([not _near_threshold(h_or[off[r]:off[r + 1]], eta) for r in range(b.num_rirs)])
    np.testing.assert_allclose(out["ekf"].cpu().numpy()[sure], (tr["e_kept"] / tr["e_tot"])[sure], rtol=1e-5)


def test_fused_rooms_backward_matches_oracle():
    b, geom = rooms_batch(seed=60, n_utts=4)
    S = int(b.num_sources.sum())
    alpha = np.linspace(0.6, 1.3, S).astype(np.float32)
    plan, out = run_rooms(b, geom, 20.0, gains=alpha)
    h_or = settled(b, geom, out["rir"].cpu().numpy())
    L = out["tl"].cpu().numpy()
    bo = check_lengths(b, h_or, L, 20.0)
    gy = synth.grad_like(61, b.y_size)
    gx, gr, gg = torch.empty_like(out["x"]), torch.full((plan.rir_size,), float("nan"), device="cuda"), \
        torch.empty(S, device="cuda")
    plan.filter_mix_backward(dev(gy), out["x"], out["gains"], gx, gr, gg)
    plan.sync_status()
    ref = oracle.backward(bo, L.astype(np.int64), alpha.astype(np.float64), gy)
    grads_close(b, ref, L, dx=gx.cpu().numpy(), dh=gr.cpu().numpy(), dalpha=gg.cpu().numpy())


@pytest.mark.parametrize("gain_mode", [0, 2])
def test_fused_rooms_gain_modes(gain_mode):
    b, geom = rooms_batch(seed=70, n_utts=4)
    if gain_mode == 2:
        alpha = np.linspace(-0.8, 1.1, b.num_rirs).astype(np.float32)
        plan, out = run_rooms(b, geom, 20.0, gain_mode=2, gains=alpha)
    else:
        plan, out = run_rooms(b, geom, 20.0, gain_mode=0)
    h_or = settled(b, geom, out["rir"].cpu().numpy())
    L = out["tl"].cpu().numpy()
    bo = check_lengths(b, h_or, L, 20.0)
    if gain_mode == 2:
        # alpha_ij scales each cut RIR (Eq. 2's general form): the per-source mix of the
        # scaled RIRs with unit gains, at the kernel's lengths
        scaled = dataclasses.replace(bo, rir=oracle._scaled_rirs(bo, alpha.astype(np.float64)))
        want = oracle.forward_with_lengths(scaled, L.astype(np.int64), np.ones(int(b.num_sources.sum())))
    else:
        ref = oracle.forward(bo, 20.0)
        np.testing.assert_allclose(out["gains"].cpu().numpy(), ref["alpha"], rtol=2e-6)
        want = oracle.forward_with_lengths(bo, L.astype(np.int64), ref["alpha"])
    yo = b.y_offsets()
    y = out["y"].cpu().numpy()
    for u in range(b.num_utts):
        n = int(b.num_samples[u])
        for j in range(b.num_mics):
            s = slice(int(yo[u]) + j * n, int(yo[u]) + (j + 1) * n)
            close_vec(y[s], want[s], f"y u={u} j={j}")


def test_fused_rooms_order_change_and_replay():
    # the graph holds order, fs and c0: a call with another order re-captures, and
    # replays of each give the eager result
    b, geom = rooms_batch(seed=80, n_utts=3)
    S = int(b.num_sources.sum())
    alpha = np.linspace(0.5, 1.0, S).astype(np.float32)
    _, eager8 = run_rooms(b, geom, 20.0, gains=alpha, graphs=False, order=8)
    _, eager3 = run_rooms(b, geom, 20.0, gains=alpha, graphs=False, order=3)
    from paper_1712_03439_gb300 import Plan
    plan = Plan.for_batch(b, eta_db=20.0, gain_mode=1, rooms=True)
    x, g, gm = eager8["x"], eager8["gains"], eager8["geom"]
    y = torch.empty(plan.y_size, device="cuda")
    tl = torch.empty(plan.R, dtype=torch.int32, device="cuda")
    for order, ref in ((8, eager8), (3, eager3), (8, eager8), (3, eager3)):
        plan.filter_mix_rooms(x, gm, g, y, trunc_len=tl, order=order)
        plan.sync_status()
        np.testing.assert_array_equal(tl.cpu().numpy(), ref["tl"].cpu().numpy())
        close_vec(y.cpu().numpy(), ref["y"].cpu().numpy().astype(np.float64), f"order {order}", rel=1e-6, mabs=1e-6)


def test_bad_geometry_is_reported_and_zeroes_its_rir():
    from paper_1712_03439_gb300 import Plan
    from paper_1712_03439_gb300._lib import RsimError
    b, geom = rooms_batch(seed=90, n_utts=2)
    geom = geom.copy()
    geom[1, 6:9] = geom[1, 3:6]                  # microphone at the source: an image at distance 0
    plan = Plan.for_batch(b, eta_db=20.0, gain_mode=1, rooms=True)
    rir = torch.full((plan.rir_size,), float("nan"), device="cuda")
    tl = torch.empty(plan.R, dtype=torch.int32, device="cuda")
    plan.filter_mix_rooms(dev(b.x), dev(geom), torch.ones(plan.G, device="cuda"),
                          torch.empty(plan.y_size, device="cuda"), trunc_len=tl, rir_out=rir)
    torch.cuda.synchronize()
    off = b.rir_offsets()
    assert not np.any(rir.cpu().numpy()[off[1]:off[2]])
    assert tl.cpu().numpy()[1] == 1
    assert np.any(rir.cpu().numpy()[off[0]:off[1]])   # the valid RIRs are made as usual
    with pytest.raises(RsimError) as e:
        plan.sync_status()
    assert e.value.status == 1


def test_rooms_call_needs_a_rooms_plan():
    from paper_1712_03439_gb300 import Plan
    from paper_1712_03439_gb300._lib import RsimError
    b, geom = rooms_batch(seed=95, n_utts=1)
    plan = Plan.for_batch(b, eta_db=20.0, gain_mode=1)
    with pytest.raises(RsimError) as e:
        plan.filter_mix_rooms(dev(b.x), dev(geom), torch.ones(plan.G, device="cuda"),
                              torch.empty(plan.y_size, device="cuda"))
    assert e.value.status == 6
