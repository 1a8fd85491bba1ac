"""GMRES-IR with the one-product FP16 factor: the inner products Z v in
float-float from the stored FP64 tiles (options.gmres_matvec) against the
FP64 products, the float-float residuals of the early refinement steps,
and the AUTO branch that takes the FP16 factor with GMRES-IR
straight after the first solve (options.fp16_gmres, mag_info.fallback = 4).
The weighting is compared with the oracle's (LAPACK factor step, FP64
refinement), elementwise.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_2607_23354_gb300")

N_CUBE = 9600  # 75 tiles: the precision probe needs three panels of 24 tiles


def _dev(X):
    return torch.from_numpy(np.ascontiguousarray(X)).cuda()


def _signs(w):
    keep = np.abs(w) >= 1e-12 * np.abs(w).max()
    return np.sign(w) * keep


@pytest.fixture(scope="module")
def cube():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X = workloads.unit_cube_cloud(n=N_CUBE)
    return X, oracle.weighting_lapack(X, 1.0)


def _check(X, t, w, mag, ref):
    w_ref, mag_ref, _ = ref
    wg = w.cpu().numpy()
    assert oracle.relative_residual(X, t, wg) <= 1e-14
    assert np.abs(wg - w_ref).max() <= 1e-9 * np.abs(w_ref).max()
    assert abs(mag - mag_ref) <= 1e-10 * abs(mag_ref)
    assert np.array_equal(_signs(wg), _signs(w_ref))


@pytest.mark.parametrize("matvec", ["float_float", "fp64"])
def test_gmres_fallback_with_either_product(cube, matvec):
    # FP16 factor forced, plain refinement cut after two steps: GMRES-IR
    # finishes with the float-float or the FP64 inner products
    X, ref = cube
    c = M.Context(M.Options(precision="fp16", residual_mode="stored", ir_max_iters=2, gmres_matvec=matvec))
    w, mag, info = c.solve(_dev(X), 1.0)
    c.close()
    assert info["fallback"] == 1 and info["gmres_iters"] > 0
    _check(X, 1.0, w, mag, ref)


def test_float_float_products_take_as_many_iterations(cube):
    # the inner solves see the same operator to ~2^-46: the iteration counts
    # of the two products stay within a couple of iterations
    X, _ = cube
    its = {}
    for matvec in ("float_float", "fp64"):
        c = M.Context(M.Options(precision="fp16", residual_mode="stored", ir_max_iters=2, gmres_matvec=matvec))
        _, _, info = c.solve(_dev(X), 1.0)
        c.close()
        its[matvec] = info["gmres_iters"]
    assert abs(its["float_float"] - its["fp64"]) <= 2, its


def test_auto_takes_fp16_with_gmres(cube):
    # fp16_gmres = 1: the probe's contraction (<= 16) sends AUTO to the FP16
    # factor with GMRES-IR from the first solve on
    X, ref = cube
    Xd = _dev(X)
    c = M.Context(M.Options(fp16_gmres=1, residual_mode="stored"))
    w, mag, info = c.solve(Xd, 1.0)
    assert info["precision_used"] == M.PREC_FP16, info
    assert info["fallback"] == 4 and info["gmres_iters"] > 0, info
    assert 0.0 < info["probe_rho"] <= 16.0, info
    # the first outer residual (far above the tolerance) in float-float
    assert info["residual_evals_ff"] >= 1 and info["residual_evals"] >= 1, info
    _check(X, 1.0, w, mag, ref)
    # the adjoint solve reuses that factor and goes to GMRES-IR at once
    b = torch.linspace(0.5, 1.5, X.shape[0], dtype=torch.float64, device="cuda")
    x, ai = c.solve_rhs(Xd, 1.0, b)
    c.close()
    assert ai["factor_reused"] == 1 and ai["fallback"] == 4
    xo = np.linalg.solve(oracle.similarity_matrix(X, 1.0), b.cpu().numpy())
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-9 * np.abs(xo).max()


def test_auto_default_keeps_the_split_factor_below_the_size_rule(cube):
    # fp16_gmres = 0 (default) at n = 9600 < 72,000: the split factor
    X, ref = cube
    c = M.Context(M.Options(residual_mode="stored"))
    w, mag, info = c.solve(_dev(X), 1.0)
    c.close()
    assert info["precision_used"] == M.PREC_FP16X3 and info["fallback"] == 0
    _check(X, 1.0, w, mag, ref)


def test_short_gmres_outer_steps(cube):
    # two inner iterations per outer step: an outer step that gains less
    # than two digits hands the solve to the split factor (fallback = 3);
    # either way the weighting is the oracle's
    X, ref = cube
    c = M.Context(M.Options(fp16_gmres=1, residual_mode="stored", gmres_max_iters=2))
    w, mag, info = c.solve(_dev(X), 1.0)
    c.close()
    assert info["gmres_iters"] >= 1
    if info["fallback"] == 3:
        assert info["precision_used"] == M.PREC_FP16X3
    else:
        assert info["fallback"] == 4 and info["precision_used"] == M.PREC_FP16
    _check(X, 1.0, w, mag, ref)


def test_early_refinement_residuals_in_float_float(cube):
    # the split factor at t = 1 refines in three steps: the first residuals
    # (far above the tolerance) come from the float-float product, the last
    # ones from FP64; with the float-float products switched off the
    # weighting matches the oracle as well
    X, ref = cube
    Xd = _dev(X)
    c = M.Context(M.Options(precision="fp16x3", residual_mode="stored"))
    w, mag, info = c.solve(Xd, 1.0)
    c.close()
    assert info["residual_evals_ff"] >= 1 and info["residual_evals"] >= 1, info
    _check(X, 1.0, w, mag, ref)
    c = M.Context(M.Options(precision="fp16x3", residual_mode="stored", gmres_matvec="fp64"))
    w2, mag2, info2 = c.solve(Xd, 1.0)
    c.close()
    assert info2["residual_evals_ff"] == 0
    # the residuals differ in their last bits: a step more or less at the
    # stopping test
    assert abs(info2["ir_iters"] - info["ir_iters"]) <= 1
    # both meet the tolerance, so both match the oracle to kappa(Z) times it
    _check(X, 1.0, w2, mag2, ref)
