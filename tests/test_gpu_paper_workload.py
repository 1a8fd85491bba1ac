"""Parity on the paper's runtime workload (Sec. 4, experimental results):
points from N(0, I_m) and N(0, diag 2^-(j-1)) for n in {1000, 3000} and
m in {3, 10, 30, 100} (run 0 of each), the task being the cutoff t_+ on
[1e-3, log(n-1)/min d] to a relative width of 1e-6 and the weighting there.
Both root-finders of the library (bisection and Ridders' method) run through
the C ABI and are checked against the oracle:

  * the oracle's own sweep (orc_tplus, bisection) on every n = 1000 cloud and
    on the n = 3000 clouds with m in {3, 100}: t_+ and the bracket ends within
    1e-6 relative and the same "below the bracket" flag;
  * every GPU bracket [lo, hi] by the oracle's weighting at its two ends:
    min w >= 0 at hi and < 0 at lo (up to the forward error, 1e-10 max|w|),
    width <= 1e-6 hi, and the sign pattern of w(t_+) equal to the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

M = pytest.importorskip("paper_2607_23354_gb300")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return M.Context()


def _signs(w):
    keep = np.abs(w) >= 1e-12 * np.abs(w).max()
    return np.sign(w) * keep


@pytest.mark.parametrize("cov", workloads.PAPER_RUNTIME_COVS)
@pytest.mark.parametrize("m", workloads.PAPER_RUNTIME_MS)
@pytest.mark.parametrize("n", [1000, 3000])
def test_paper_runtime_cloud_cutoff(ctx, n, m, cov):
    X = workloads.paper_runtime_cloud(n, m, cov, 0)
    Xd = torch.from_numpy(X).cuda()
    res = {meth: ctx.sweep_tplus(Xd, 1e-3, 0.0, 1e-6, method=meth) for meth in ("bisection", "ridders")}
    full = n == 1000 or m in (3, 100)
    if full:
        for meth in ("bisection", "ridders") if n == 1000 else ("bisection",):
            ro = oracle.tplus(X, 1e-3, 0.0, 1e-6, method=meth)
            r = res[meth]
            assert r["below"] == ro["below"]
            assert r["t_plus"] == pytest.approx(ro["t_plus"], rel=1.01e-6)
            assert r["bracket"][0] == pytest.approx(ro["bracket"][0], rel=1.01e-6)
            assert r["bracket"][1] == pytest.approx(ro["bracket"][1], rel=1.01e-6)
    for meth, r in res.items():
        lo, hi = r["bracket"]
        w_hi, _, _ = oracle.weighting(X, hi)
        scale = np.abs(w_hi).max()
        assert w_hi.min() >= -1e-10 * scale, (meth, hi, w_hi.min())
        assert np.array_equal(_signs(r["w"].cpu().numpy()), _signs(w_hi)), meth
        if r["below"]:
            assert hi == 1e-3
            continue
        assert hi - lo <= 1e-6 * hi
        w_lo, _, _ = oracle.weighting(X, lo)
        assert w_lo.min() < 1e-10 * np.abs(w_lo).max(), (meth, lo, w_lo.min())
    assert res["bisection"]["t_plus"] == pytest.approx(res["ridders"]["t_plus"], rel=1.01e-6)
