"""The allocation-free residual entry point (mag_residual_noalloc).

Some callers cannot let a library call cudaMalloc: code running under a
framework's own memory manager or a fixed memory budget, and latency-bound
loops where an allocation would synchronize the device.  For them the library
offers the FP64 residual r = b - Z w with its scratch in a static device
array instead of a context workspace.  This test calls it through the C ABI
twice in a row and checks both results against the allocating entry point
mag_residual, within the tolerance the other residual tests use.  It lives in
its own file, collected last, and needs no state from other tests.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_2607_23354_gb300")


def _setup(n, m, seed):
    rng = np.random.default_rng(seed)
    X = torch.from_numpy(rng.random((n, m))).cuda()
    w = torch.from_numpy(rng.standard_normal(n) * 0.1 + 0.5).cuda()
    return X, w


@pytest.mark.parametrize("n,m,t,use_b", [(1500, 8, 1.0, False), (4099, 3, 5.0, True)])
def test_noalloc_matches_allocating_residual_twice(n, m, t, use_b):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X, w = _setup(n, m, seed=n)
    b = torch.from_numpy(np.random.default_rng(n + 1).standard_normal(n)).cuda() if use_b else None
    ctx = M.Context()
    r_ref, nr_ref = ctx.residual(X, t, w, b=b)
    scale = nr_ref["z_norm_inf"] * nr_ref["w_norm_inf"]
    bmax = 0.0 if b is None else float(b.abs().max())
    for _ in range(2):
        r, nr = M.residual_noalloc(X, t, w, b=b)
        torch.cuda.synchronize()
        # different column splits of the compensated row sums: a few ulps of the row scale
        assert float((r - r_ref).abs().max()) <= 2e-15 * scale + 4e-16 * bmax
        assert nr["z_norm_inf"] == pytest.approx(nr_ref["z_norm_inf"], rel=1e-14)
        assert nr["w_norm_inf"] == nr_ref["w_norm_inf"]
        assert nr["r_norm_inf"] == pytest.approx(nr_ref["r_norm_inf"], rel=1e-12, abs=4e-15 * scale)
        assert nr["rel_residual"] == pytest.approx(nr_ref["rel_residual"], rel=1e-12, abs=4e-15)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = M.NOALLOC_MAX_N + 1
    X = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MagnitudeError) as e:
        M.residual_noalloc(X, 1.0, w)
    assert e.value.status == M.MAG_ENOMEM
