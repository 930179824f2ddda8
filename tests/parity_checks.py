"""Comparisons shared by the GPU parity tests.

The tolerances are those of the filter-and-mix path: every compared vector
(an output channel, one source's gradient, one RIR's gradient) within a
relative L2 error of 1e-5 and a max-abs error of 1e-5 x its own peak,
against the FP64 oracle; gain gradients elementwise within 1e-5 relative
(absolute floor 1e-5 x the largest); RIR gradients exactly zero beyond each
kept length.
"""
import numpy as np

REL_L2 = 1e-5
MAX_ABS = 1e-5


def close_vec(got, ref, what, rel=REL_L2, mabs=MAX_ABS):
    g = np.asarray(got, np.float64)
    r = np.asarray(ref, np.float64)
    assert g.shape == r.shape, f"{what}: shape {g.shape} vs {r.shape}"
    assert np.all(np.isfinite(g)), f"{what}: non-finite values"
    if r.size == 0:
        return
    peak = np.abs(r).max()
    if peak == 0:
        assert np.abs(g).max() == 0, f"{what}: nonzero values against a zero reference"
        return
    rl2 = np.linalg.norm(g - r) / np.linalg.norm(r)
    assert rl2 <= rel, f"{what}: rel L2 {rl2:.3e}"
    ma = np.abs(g - r).max() / peak
    assert ma <= mabs, f"{what}: max abs {ma:.3e} x peak"


def gains_close(got, ref, what="dalpha", rel=REL_L2):
    ref = np.asarray(ref, np.float64)
    np.testing.assert_allclose(np.asarray(got, np.float64), ref, rtol=rel,
                               atol=rel * max(np.abs(ref).max(), 1e-30), err_msg=what)


def grads_close(batch, ref, L, dx=None, dh=None, dalpha=None, what=""):
    """dx per source, dh per RIR (zero beyond L), dalpha elementwise, each
    against the oracle's ref dict (keys dx, dh, dalpha); None skips a part."""
    if dx is not None:
        xo = batch.x_offsets()
        for s in range(int(np.sum(batch.num_sources))):
            close_vec(dx[xo[s]:xo[s + 1]], ref["dx"][xo[s]:xo[s + 1]], f"{what}dx[{s}]")
    if dh is not None:
        ro = batch.rir_offsets()
        for r in range(batch.num_rirs):
            seg = dh[ro[r]:ro[r + 1]]
            close_vec(seg, ref["dh"][ro[r]:ro[r + 1]], f"{what}dh[{r}]")
            assert np.all(seg[int(L[r]):] == 0), f"{what}dh[{r}] nonzero beyond L = {L[r]}"
    if dalpha is not None:
        gains_close(dalpha, ref["dalpha"], f"{what}dalpha")
