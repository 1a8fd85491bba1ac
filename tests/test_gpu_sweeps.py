"""Triangular sweeps of the refinement corrections (options.sweeps): the
chain sweeps (one 128 x 128 product with B_I = inv(L_II) L_{I,I-1} per tile
on the critical path; off-diagonal tiles read as FP16 with the one-product
factor), the same with FP32 tiles, and the progress-counter sweeps.  The
weighting each gives is compared with the oracle's (LAPACK factor step,
FP64 refinement) elementwise at n = 9600 (75 row tiles: one per block),
and by the oracle's residual rows at n = 39,963 (313 row tiles, several per
block, a ragged last tile).  With the same factor the three sweeps give the
same corrections to FP32 rounding, so refinement takes the same number of
steps (within one).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_2607_23354_gb300")

KINDS = {"chain": None, "chain_fp32": 1, "progress": 2}


def _dev(X):
    return torch.from_numpy(np.ascontiguousarray(X)).cuda()


@pytest.fixture(scope="module")
def small():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X = workloads.unit_cube_cloud(n=9600)
    return X, {t: oracle.weighting_lapack(X, t) for t in (1.0, 10.0)}


def _solve(X, t, precision, sweeps, **kw):
    c = M.Context(M.Options(precision=precision, residual_mode="stored", sweeps=sweeps, **kw))
    w, mag, info = c.solve(_dev(X), t)
    c.close()
    return w.cpu().numpy(), mag, info


@pytest.mark.parametrize("precision,t", [("fp16x3", 1.0), ("fp16", 10.0)])
def test_sweep_kinds_match_oracle(small, precision, t):
    X, refs = small
    w_ref, mag_ref, _ = refs[t]
    iters = {}
    for kind, used in KINDS.items():
        w, mag, info = _solve(X, t, precision, kind)
        expect = used if used is not None else (0 if precision == "fp16" else 1)
        assert info["sweeps_used"] == expect, (kind, info["sweeps_used"])
        assert oracle.relative_residual(X, t, w) <= 1e-14
        assert np.abs(w - w_ref).max() <= 1e-9 * np.abs(w_ref).max()
        assert abs(mag - mag_ref) <= 1e-10 * abs(mag_ref)
        iters[kind] = info["ir_iters"]
    assert max(iters.values()) - min(iters.values()) <= 1, iters


@pytest.mark.parametrize("precision,t", [("fp16x3", 1.0), ("fp16", 10.0)])
def test_sweep_kinds_several_tiles_per_block(precision, t):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X = workloads.unit_cube_cloud(n=39_963, seed=2102)
    rows = np.random.default_rng(7).choice(len(X), 384, replace=False)
    rows = np.unique(np.concatenate([rows, np.arange(len(X) - 37, len(X))]))  # the ragged last tile
    sol = {}
    for kind in KINDS:
        w, mag, info = _solve(X, t, precision, kind)
        assert info["rel_residual"] <= 1e-14, (kind, info)
        r, _ = oracle.residual_rows(X, t, w, rows=rows)
        assert np.abs(r).max() <= 1e-14 * info["z_norm_inf"] * np.abs(w).max(), kind
        sol[kind] = (w, info["ir_iters"])
    w0 = sol["progress"][0]
    for kind in ("chain", "chain_fp32"):
        # both solutions meet the tolerance: they agree to kappa(Z) times it
        assert np.abs(sol[kind][0] - w0).max() <= 1e-9 * np.abs(w0).max(), kind
        assert abs(sol[kind][1] - sol["progress"][1]) <= 1, (kind, sol[kind][1], sol["progress"][1])


def test_gmres_with_fp16_chain_sweeps(small):
    # the FP16 factor with GMRES-IR (t = 1: plain refinement with it would
    # crawl): every inner correction through the FP16-tile chain sweeps
    X, refs = small
    w_ref, mag_ref, _ = refs[1.0]
    w, mag, info = _solve(X, 1.0, "auto", "chain", fp16_gmres=1)
    assert info["precision_used"] == M.PREC_FP16 and info["fallback"] == 4, info
    assert info["sweeps_used"] == 0 and info["gmres_iters"] > 0, info
    assert np.abs(w - w_ref).max() <= 1e-9 * np.abs(w_ref).max()
    w2, _, info2 = _solve(X, 1.0, "auto", "progress", fp16_gmres=1)
    assert info2["sweeps_used"] == 2
    # the FP16 tiles are the operands the factor's updates used: GMRES needs
    # about as many inner iterations as with the FP32 tiles
    assert abs(info["gmres_iters"] - info2["gmres_iters"]) <= 3, (info["gmres_iters"], info2["gmres_iters"])
    assert np.abs(w2 - w_ref).max() <= 1e-9 * np.abs(w_ref).max()
