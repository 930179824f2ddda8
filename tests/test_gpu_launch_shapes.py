"""Launch shapes and allocation failure (GPU).

* A plan made with RSIM_TEST_ONE_CTA=1 in the environment runs every
  persistent kernel with a single CTA: the forward's work lists and the
  backward's partition then go to one CTA.  The forward output and the source
  gradient are bitwise those of the full grid (every block is computed the same
  way); the RIR and gain gradients are summed over other pieces, so they are
  compared within the parity tolerance, and all of them with the oracle.
* A batch whose plan needs more device memory than the GPU has (a 2^36-sample
  utterance: about 0.5 TB of segment carries) is refused with RSIM_E_NOMEM,
  and the context stays usable.
"""
import numpy as np
import pytest

import oracle
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def run(b, gains, gy, one_cta, monkeypatch):
    from paper_1712_03439_gb300 import Plan
    if one_cta:
        monkeypatch.setenv("RSIM_TEST_ONE_CTA", "1")
    else:
        monkeypatch.delenv("RSIM_TEST_ONE_CTA", raising=False)
    plan = Plan.for_batch(b, eta_db=20.0, gain_mode=1)
    monkeypatch.delenv("RSIM_TEST_ONE_CTA", raising=False)
    x, rir, g = dev(b.x), dev(b.rir), dev(gains)
    y = torch.empty(plan.y_size, device="cuda")
    plan.filter_mix(x, rir, g, y)
    gx, gr, gg = torch.empty_like(x), torch.empty_like(rir), torch.empty_like(g)
    plan.filter_mix_backward(dev(gy), x, g, gx, gr, gg)
    plan.sync_status()
    return {k: v.cpu().numpy() for k, v in dict(y=y, dx=gx, dh=gr, da=gg).items()}


@pytest.mark.parametrize("sizes", [None, [4096]])
def test_one_cta_equals_the_full_grid(monkeypatch, sizes):
    b = synth.make_batch(301, [900, 20011, 50000, 33333, 7000], [2, 3, 1, 4, 6], synth.linear_pair_array(),
                         (0.1, 0.3))
    S = int(b.num_sources.sum())
    gains = np.linspace(0.5, 1.4, S).astype(np.float32)
    gy = synth.grad_like(302, b.y_size)
    full = run(b, gains, gy, False, monkeypatch)
    one = run(b, gains, gy, True, monkeypatch)
    np.testing.assert_array_equal(one["y"], full["y"])
    np.testing.assert_array_equal(one["dx"], full["dx"])
    L = oracle.truncate_batch(b, 20.0)["L"]
    ref = oracle.backward(b, L, gains.astype(np.float64), gy)
    for got in (one, full):
        grads_close(b, ref, L, dx=got["dx"], dh=got["dh"], dalpha=got["da"])
    yref = oracle.forward(b, 20.0, alpha=gains.astype(np.float64))["y"]
    yo = b.y_offsets()
    for u in range(b.num_utts):
        n = int(b.num_samples[u])
        for j in range(b.num_mics):
            s = slice(int(yo[u]) + j * n, int(yo[u]) + (j + 1) * n)
            close_vec(one["y"][s], yref[s], f"y u={u} j={j}")


def test_plan_beyond_device_memory_is_nomem_and_the_context_survives():
    from paper_1712_03439_gb300 import Plan
    from paper_1712_03439_gb300._lib import RsimError
    with pytest.raises(RsimError) as e:
        Plan([1], [1 << 36], [100, 100], 2, eta_db=20.0, gain_mode=1)
    assert e.value.status == 3
    assert "cudaMalloc" in str(e.value)
    b = synth.make_batch(303, [5000], [2], synth.linear_pair_array(), (0.1, 0.2))
    out = run(b, np.ones(2, np.float32), synth.grad_like(304, b.y_size), False, pytest.MonkeyPatch())
    assert np.all(np.isfinite(out["y"]))
