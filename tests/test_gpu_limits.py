"""Limits and failure paths of the CUDA path, through the C ABI: arguments at
the edge of the FP64 exponential's range, the Sec. 1 bound requested inside a
multi-t call, a bounded device wait that runs out, a workspace limit, and the
loss gradient for a constant dL/dw.  Every failure here is made on the host
(an option or a size limit); nothing faults the GPU, and each test checks that
the same context solves correctly afterwards.
"""
import math

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_2607_23354_gb300")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return M.Context()


def _dev(X):
    return torch.from_numpy(np.ascontiguousarray(X)).cuda()


def _cube(n, m, seed):
    return np.random.default_rng(seed).random((n, m))


# ------------------------------------------- exponential far below its range

@pytest.mark.parametrize("t", [1e3, 6e6, 1e7, 1e8, 1e13])
def test_exponential_of_huge_arguments_is_zero(ctx, t):
    # points 1, 2, ... apart on a line: t d runs from t to 299 t, far beyond
    # the point (about 5.8e6) where round(256 x / ln 2) leaves int32; Z must
    # be the identity and the residual of w = 1 exactly zero
    n = 300
    X = np.zeros((n, 2))
    X[:, 0] = np.arange(n, dtype=float)
    Xd = _dev(X)
    Zg = ctx.similarity_matrix(Xd, t, "fp64").cpu().numpy()
    assert np.array_equal(Zg, np.eye(n))
    ones = torch.ones(n, dtype=torch.float64, device="cuda")
    r, nr = ctx.residual(Xd, t, ones)
    assert float(r.abs().max()) == 0.0
    assert nr["z_norm_inf"] == 1.0 and nr["rel_residual"] == 0.0
    ro, rso = oracle.residual_rows(X, t, np.ones(n))
    assert np.all(ro == 0.0) and np.all(rso == 1.0)
    w, mag, info = ctx.solve(Xd, t)
    assert np.array_equal(w.cpu().numpy(), np.ones(n)) and mag == n
    dt, dx = ctx.grad(Xd, t, w=w)
    assert dt == 0.0 and float(dx.abs().max()) == 0.0


def test_exponential_near_its_underflow(ctx):
    # t d across the FP64 underflow (x from -700 to -760 in steps of 0.5): the
    # device exponential against the host libm (0 below 2^-1021 is allowed)
    n = 121
    X = np.zeros((n, 1))
    X[:, 0] = np.arange(n) * 0.5
    t = 1.0
    base = 700.0
    X[1:, 0] += base
    Zg = ctx.similarity_matrix(_dev(X), t, "fp64").cpu().numpy()
    ref = np.exp(-t * np.abs(X[:, 0][:, None] - X[:, 0][None, :]))
    small = ref < 2.0 ** -1021
    assert np.all(np.abs(Zg - ref)[~small] <= 2 * np.spacing(ref[~small]))
    assert np.all((Zg[small] == 0.0) | (np.abs(Zg[small] - ref[small]) <= 2 ** -1021))


# ------------------------------------------ Sec. 1 bound inside a multi-t call

def test_solve_multi_bound_sentinel(ctx):
    X = _cube(1500, 8, 801)
    Xd = _dev(X)
    bound = oracle.tplus_bound(X)
    W, mags, infos = ctx.solve_multi(Xd, [1.0, "bound", 10.0])
    assert infos[1]["t"] == pytest.approx(bound, rel=1e-15)
    assert infos[0]["t"] == 1.0 and infos[2]["t"] == 10.0
    assert infos[1]["min_distance"] == pytest.approx(oracle.min_distance(X), rel=1e-15)
    for i, t in enumerate([1.0, bound, 10.0]):
        w_ref, mag_ref, _ = oracle.weighting(X, t)
        wg = W[i].cpu().numpy()
        assert oracle.relative_residual(X, t, wg) <= 1e-14
        assert np.abs(wg - w_ref).max() <= 1e-9 * np.abs(w_ref).max()
        assert abs(mags[i] - mag_ref) <= 1e-10 * abs(mag_ref)
    # the bound alone: one min-distance pass, then the solve
    W1, mags1, infos1 = ctx.solve_multi(Xd, [0.0])
    assert infos1[0]["t"] == infos[1]["t"]
    assert abs(mags1[0] - mags[1]) <= 1e-12 * abs(mags[1])


def test_solve_multi_bound_with_duplicates_reports_each_entry(ctx):
    X = _cube(300, 3, 802)
    X[7] = X[100]
    with pytest.raises(M.MagnitudeError) as e:
        ctx.solve_multi(_dev(X), [0.0, 1.0])
    assert e.value.status == M.MAG_EDUPLICATE
    w, mag, _ = ctx.solve(_dev(_cube(300, 3, 803)), 1.0)  # the context still works
    assert np.isfinite(mag)


# ------------------------------------------------------- bounded device waits

def test_sweep_wait_timeout_then_recovery(ctx):
    # a 1 us bound on the triangular sweeps' waits for other CTAs' tiles:
    # with 128 row tiles a sweep takes far longer, so a wait gives up, the
    # kernel raises its timeout flag and the solve returns MAG_ETIMEOUT; the
    # context then solves the same problem with the default bound
    X = _cube(16384, 8, 804)
    Xd = _dev(X)
    c = M.Context(M.Options(precision="fp16x3", wait_timeout_ns=1000))
    with pytest.raises(M.MagnitudeError) as e:
        c.solve(Xd, 5.0)
    assert e.value.status == M.MAG_ETIMEOUT
    c.set_options(M.Options(precision="fp16x3"))
    w, mag, info = c.solve(Xd, 5.0)
    assert info["rel_residual"] <= 1e-14
    wg = w.cpu().numpy()
    rows = np.random.default_rng(5).choice(len(X), 256, replace=False)
    r, rs = oracle.residual_rows(X, 5.0, wg, rows=rows)
    assert np.abs(r).max() <= 1e-14 * info["z_norm_inf"] * np.abs(wg).max()
    c.close()


def test_wait_timeout_must_be_positive(ctx):
    with pytest.raises(M.MagnitudeError) as e:
        ctx.set_options(M.Options(wait_timeout_ns=0))
    assert e.value.status == M.MAG_EINVAL
    ctx.set_options(M.Options())


# ---------------------------------------------------------- workspace limit

def test_workspace_limit_gives_enomem_then_recovers():
    X = _cube(4096, 8, 805)
    Xd = _dev(X)
    c = M.Context(M.Options(workspace_limit_bytes=1e6))
    need = c.workspace_bytes(4096, 8)
    assert need > 1e6
    with pytest.raises(M.MagnitudeError) as e:
        c.solve(Xd, 2.0)
    assert e.value.status == M.MAG_ENOMEM
    c.set_options(M.Options(workspace_limit_bytes=2 * need))
    w, mag, info = c.solve(Xd, 2.0)
    w_ref, mag_ref, _ = oracle.weighting(X, 2.0)
    assert np.abs(w.cpu().numpy() - w_ref).max() <= 1e-9 * np.abs(w_ref).max()
    assert abs(mag - mag_ref) <= 1e-10 * abs(mag_ref)
    c.close()


def test_dimension_limit(ctx):
    X = torch.zeros(10, M.MAX_DIM + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MagnitudeError) as e:
        ctx.solve(X, 1.0)
    assert e.value.status == M.MAG_EINVAL


def test_residual_at_large_dimension(ctx):
    # m = 1000 > 703: eight staged points need more than the default 48 KB of
    # shared memory; the residual kernel opts in and matches the oracle
    X = np.random.default_rng(806).standard_normal((700, 1000)) / math.sqrt(1000)
    w = np.random.default_rng(807).standard_normal(700)
    r, nr = ctx.residual(_dev(X), 0.8, torch.from_numpy(w).cuda())
    ro, rso = oracle.residual_rows(X, 0.8, w)
    # d^2 sums 1000 squares (FMA on the device, none on the host): a few
    # dozen ulps of Z per entry
    scale = rso.max() * np.abs(w).max()
    assert np.abs(r.cpu().numpy() - ro).max() <= 1e-13 * scale
    assert nr["z_norm_inf"] == pytest.approx(rso.max(), rel=1e-14)


# --------------------------------------------- gradient of c Mag without a solve

def test_constant_loss_gradient_is_scaled_magnitude_gradient(ctx):
    X = np.random.default_rng(808).standard_normal((2000, 5)) / math.sqrt(5)
    Xd = _dev(X)
    t = 1.5
    w, _, _ = ctx.solve(Xd, t)
    dt1, dx1 = ctx.grad(Xd, t, w=w)
    c = -2.75
    dt2, dx2 = ctx.grad(Xd, t, w=w, dL_dw=torch.full_like(w, c))
    assert dt2 == pytest.approx(c * dt1, rel=1e-14)
    assert float((dx2 - c * dx1).abs().max()) <= 1e-14 * float(dx1.abs().max()) * abs(c)
    dto, dxo = oracle.grad(X, t, oracle.weighting(X, t)[0])
    assert dt1 == pytest.approx(dto, rel=1e-9)


# ------------------------------------------- the adjoint solve reuses the factor

def test_adjoint_solve_reuses_the_forward_factor(ctx):
    # after a solve, a solve with another right-hand side for the same points
    # and t refines with the factor still in the context (no new factor); a
    # change of the points in place (same pointer) is seen by the checksum
    X = np.random.default_rng(809).random((3000, 6))
    Xd = _dev(X)
    t = 1.5
    w, mag, info = ctx.solve(Xd, t)
    g = np.random.default_rng(810).standard_normal(3000)
    lam, ai = ctx.solve_rhs(Xd, t, torch.from_numpy(g).cuda())
    assert ai["factor_reused"] == 1 and ai["ms_factor"] == 0.0
    lam_ref, oi = oracle.solve(X, t, b=g)
    assert oracle.relative_residual(X, t, lam.cpu().numpy(), b=g) <= 1e-14
    assert np.abs(lam.cpu().numpy() - lam_ref).max() <= 1e-9 * np.abs(lam_ref).max()
    # another t: no reuse
    _, ai2 = ctx.solve_rhs(Xd, 1.6, torch.from_numpy(g).cuda())
    assert ai2["factor_reused"] == 0
    # the same t again after the points changed in place: no reuse, and the
    # result is the new points' solution
    ctx.solve(Xd, t)
    Xd[17, 3] += 1e-3
    X2 = Xd.cpu().numpy()
    lam3, ai3 = ctx.solve_rhs(Xd, t, torch.from_numpy(g).cuda())
    assert ai3["factor_reused"] == 0
    assert oracle.relative_residual(X2, t, lam3.cpu().numpy(), b=g) <= 1e-14
    # mag_grad with a general loss right after the forward solve
    w, _, _ = ctx.solve(Xd, t)
    dt, dx = ctx.grad(Xd, t, w=w, dL_dw=2 * w)
    dto, dxo = oracle.grad_loss(X2, t, 2 * w.cpu().numpy(), w=w.cpu().numpy())
    assert dt == pytest.approx(dto, rel=1e-8)
    assert np.abs(dx.cpu().numpy() - dxo).max() <= 1e-7 * np.abs(dxo).max()
