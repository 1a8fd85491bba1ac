"""The out-of-core factor (the factor of a matrix whose packed tiles do not fit
in device memory): forced at small n by a workspace limit that leaves room
for only a few hundred tiles, so that the factor runs in many slabs, most of
them moved to host memory; the weighting against the oracle's, elementwise,
and against the in-core solve.  The last test runs past one GB300's memory:
n = 380,000 points in [0,1]^8 (2.9e11 bytes of FP32 tiles), checked by the
oracle's FP64 residual on sampled rows.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_2607_23354_gb300")

TILE_BYTES = 128 * 128 * 4


def _dev(X):
    return torch.from_numpy(np.ascontiguousarray(X)).cuda()


def _signs(w):
    keep = np.abs(w) >= 1e-12 * np.abs(w).max()
    return np.sign(w) * keep


def _limit_for_pool(n, pool_tiles, panel_tiles=0):
    """A workspace limit that leaves `pool_tiles` FP32 tiles for the slabs
    next to the rest of the workspace (vectors, panel buffers, inverses)."""
    c = M.Context(M.Options(residual_mode="matrix_free", panel_tiles=panel_tiles))
    total = c.workspace_bytes(n, 8)
    c.close()
    N = (n + 127) // 128
    base = total - N * (N + 1) // 2 * TILE_BYTES
    return base + pool_tiles * TILE_BYTES + 4096 + 256 * 16


@pytest.fixture(scope="module")
def ref_cube():
    X = workloads.unit_cube_cloud(n=8192)
    return X, {t: oracle.weighting_lapack(X, t) for t in (2.0, 10.0)}


@pytest.mark.parametrize("prec", ["fp16x3", "fp16", "auto"])
@pytest.mark.parametrize("t", [2.0, 10.0])
def test_slabs_on_host_match_oracle(ref_cube, prec, t):
    X, refs = ref_cube
    n = X.shape[0]
    opts = M.Options(precision=prec, out_of_core=1, workspace_limit_bytes=_limit_for_pool(n, 700))
    c = M.Context(opts)
    w, mag, info = c.solve(_dev(X), t)
    c.close()
    assert info["slabs"] >= 5 and info["host_slabs"] >= 3, info
    assert info["host_bytes"] > 0 and math.isnan(info["gershgorin_lmin"])
    w_ref, mag_ref, _ = refs[t]
    wg = w.cpu().numpy()
    assert oracle.relative_residual(X, t, wg) <= 1e-14
    assert np.abs(wg - w_ref).max() <= 1e-9 * np.abs(w_ref).max()
    assert abs(mag - mag_ref) <= 1e-10 * abs(mag_ref)
    assert np.array_equal(_signs(wg), _signs(w_ref))
    # the same weighting in core
    w2, mag2, info2 = M.Context(M.Options(precision=prec)).solve(_dev(X), t)
    assert info2["slabs"] == 0
    assert abs(mag2 - mag) <= 1e-12 * abs(mag)


@pytest.mark.parametrize("n,pool,panel", [(5000, 300, 0), (5000, 400, 3), (3000, 10 ** 6, 0)])
def test_ragged_sizes_and_a_single_slab(n, pool, panel):
    # n = 5000: a ragged last tile row inside host slabs, and slab widths that
    # are no multiple of a 3-tile panel; n = 3000 with room for everything:
    # the forced out-of-core path as one device slab
    X = np.random.default_rng(n).random((n, 5))
    t = 3.0
    c = M.Context(M.Options(precision="fp16x3", out_of_core=1, panel_tiles=panel,
                            workspace_limit_bytes=_limit_for_pool(n, pool, panel)))
    w, mag, info = c.solve(_dev(X), t)
    c.close()
    if pool < 10 ** 6:
        assert info["host_slabs"] >= 1
    else:
        assert info["slabs"] == 1 and info["host_slabs"] == 0
    w_ref, mag_ref, _ = oracle.weighting(X, t)
    wg = w.cpu().numpy()
    assert oracle.relative_residual(X, t, wg) <= 1e-14
    assert np.abs(wg - w_ref).max() <= 1e-9 * np.abs(w_ref).max()
    assert abs(mag - mag_ref) <= 1e-10 * abs(mag_ref)


def test_out_of_core_rejects_other_precisions():
    X = np.random.default_rng(3).random((600, 3))
    c = M.Context(M.Options(precision="tf32x3", out_of_core=1))
    with pytest.raises(M.MagnitudeError) as e:
        c.solve(_dev(X), 1.0)
    assert e.value.status == M.MAG_EINVAL
    c.close()


def test_host_limit_gives_enomem():
    X = workloads.unit_cube_cloud(n=8192)
    c = M.Context(M.Options(out_of_core=1, workspace_limit_bytes=_limit_for_pool(8192, 700),
                            host_limit_bytes=1e6))
    with pytest.raises(M.MagnitudeError) as e:
        c.solve(_dev(X), 2.0)
    assert e.value.status == M.MAG_ENOMEM
    c.close()


@pytest.mark.slow
def test_beyond_device_memory_n380000():
    # 380,000 points in [0,1]^8: the packed FP32 tiles alone (2.9e11 bytes)
    # exceed the GPU's memory; the default options factor out of core
    n = 380_000
    X = workloads.unit_cube_cloud(n=n)
    t = 10.0
    c = M.Context(M.Options())
    w, mag, info = c.solve(_dev(X), t)
    assert info["slabs"] >= 2 and info["host_slabs"] >= 1, info
    assert info["rel_residual"] <= 1e-14
    wg = w.cpu().numpy()
    rows = np.random.default_rng(380).choice(n, 192, replace=False)
    r, rs = oracle.residual_rows(X, t, wg, rows=rows)
    # the sampled rows' residual against the norm ||Z||inf ||w||inf (the
    # oracle's row sums bound ||Z||inf from below)
    assert np.abs(r).max() <= 1e-14 * info["z_norm_inf"] * np.abs(wg).max()
    assert rs.max() <= info["z_norm_inf"] * (1 + 1e-12)
    assert mag == pytest.approx(oracle.kahan_sum(wg), rel=1e-13)
    c.close()
