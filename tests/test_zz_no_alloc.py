"""The allocation-free gains entry point against the plan path (GPU).

rsim_source_gains_noalloc serves callers that cannot allocate device memory
when they need the gains (a memory manager owns every device allocation, or
an allocation would stall the device at the wrong moment), so they cannot
make a plan.  Its scratch is a fixed array inside the library that every
call reuses; these tests call it through the C-ABI twice in a row, on two
different batches, and check each result against the gains rsim_filter_mix
computes with gain_mode = 0 and against the FP64 oracle's gains.  This file
is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1712_03439_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 2e-6   # the gains tolerance of the parity tests


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_03439_gb300 import _lib, build
    build.build()
    return _lib.load()


def _plan_gains(b):
    from paper_1712_03439_gb300 import Plan, filter_mix
    plan = Plan.for_batch(b, eta_db=20.0, gain_mode=0)
    out = filter_mix(plan, torch.from_numpy(b.x).cuda(), torch.from_numpy(b.rir).cuda(),
                     snr_db=torch.from_numpy(b.snr_db).cuda())
    plan.sync_status()
    return out["gains"].cpu().numpy()


def _noalloc_gains(lib, b):
    ns = np.ascontiguousarray(b.num_sources, np.int32)
    nx = np.ascontiguousarray(b.num_samples, np.int64)
    x = torch.from_numpy(b.x).cuda()
    snr = torch.from_numpy(b.snr_db).cuda()
    gains = torch.full((int(ns.sum()),), -1.0, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.rsim_source_gains_noalloc(stream, ns.shape[0], ctypes.c_void_p(ns.ctypes.data),
                                       ctypes.c_void_p(nx.ctypes.data), ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(snr.data_ptr()), ctypes.c_void_p(gains.data_ptr()))
    assert st == 0, lib.rsim_last_error().decode()
    torch.cuda.synchronize()
    return gains.cpu().numpy()


def test_noalloc_gains_match_the_plan_path_on_two_calls_in_a_row(lib):
    big = synth.config_home(n_utts=40)
    small = synth.make_batch(77, [5000, 33000, 70001], [3, 1, 4], synth.linear_pair_array(), (0.1, 0.3))
    ref_big, ref_small = _plan_gains(big), _plan_gains(small)
    # the second call reuses the scratch the first one left behind
    got_big = _noalloc_gains(lib, big)
    got_small = _noalloc_gains(lib, small)
    np.testing.assert_allclose(got_big, ref_big, rtol=RTOL, atol=0)
    np.testing.assert_allclose(got_small, ref_small, rtol=RTOL, atol=0)
    # and the same batch twice in a row
    np.testing.assert_allclose(_noalloc_gains(lib, small), ref_small, rtol=RTOL, atol=0)


def _oracle_gains(b):
    si, xo = b.src_index(), b.x_offsets()
    out = []
    for u in range(b.num_utts):
        nx = int(b.num_samples[u])
        xs = b.x[xo[si[u]]:xo[si[u + 1]]].reshape(-1, nx)
        out.append(oracle.gains(xs, b.snr_db[si[u]:si[u + 1]]))
    return np.concatenate(out)


def test_noalloc_gains_match_the_oracle(lib):
    b = synth.make_batch(78, [900, 40000, 70001, 12345], [2, 4, 1, 3], synth.linear_pair_array(), (0.1, 0.3))
    np.testing.assert_allclose(_noalloc_gains(lib, b), _oracle_gains(b), rtol=RTOL, atol=0)


def test_noalloc_silent_noise_source_gets_nan_and_the_others_stay_finite(lib):
    # the plan path reports a silent noise source as an error; this entry point has
    # no plan to latch it in and writes NaN for that source only
    b = synth.make_batch(79, [3000, 5000], [3, 2], synth.linear_pair_array(), (0.1, 0.3))
    xo = b.x_offsets()
    b.x[xo[1]:xo[2]] = 0                   # utterance 0, noise source 1
    got = _noalloc_gains(lib, b)
    assert np.isnan(got[1])
    assert np.all(np.isfinite(got[[0, 2, 3, 4]]))
    # source 2 of utterance 0: the oracle on that utterance without the silent source
    nx = int(b.num_samples[0])
    xs = np.stack([b.x[xo[0]:xo[1]], b.x[xo[2]:xo[3]]]).reshape(2, nx)
    a02 = oracle.gains(xs, np.array([0.0, b.snr_db[2]], np.float32))[1]
    np.testing.assert_allclose(got[2], a02, rtol=RTOL)
    assert got[0] == 1.0
    np.testing.assert_allclose(got[3:], _oracle_gains(b.subset([1])), rtol=RTOL)


def test_noalloc_python_wrapper_on_a_side_stream(lib):
    from paper_1712_03439_gb300 import api
    b = synth.make_batch(80, [20000, 7000], [2, 3], synth.linear_pair_array(), (0.1, 0.3))
    side = torch.cuda.Stream()
    x = torch.from_numpy(b.x).cuda()
    snr = torch.from_numpy(b.snr_db).cuda()
    gains = torch.full((int(b.num_sources.sum()),), -1.0, device="cuda")
    side.wait_stream(torch.cuda.current_stream())   # the inputs' copies are done
    with torch.cuda.stream(side):
        api.source_gains_noalloc(b.num_sources, b.num_samples, x, snr, gains, stream=side)
    side.synchronize()
    np.testing.assert_allclose(gains.cpu().numpy(), _oracle_gains(b), rtol=RTOL, atol=0)


def test_noalloc_rejects_a_batch_beyond_its_fixed_scratch(lib):
    # 2048 utterances of 4 sources and 82 s need about 2.7 MB of partial sums,
    # more than the 2 MiB of scratch
    U = 2048
    ns = np.full(U, 4, np.int32)
    nx = np.full(U, 40 * 32768, np.int64)
    dummy = torch.zeros(1, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    st = lib.rsim_source_gains_noalloc(None, U, ctypes.c_void_p(ns.ctypes.data),
                                       ctypes.c_void_p(nx.ctypes.data), p, p, p)
    assert st == 2
    assert "fixed maximum" in lib.rsim_last_error().decode()
