"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle on the
same seeded inputs.

Tolerances (stated per quantity, from the arithmetic):
  * FP64 Z entries: both sides take d^2 in FP64 (GPU with FMA, CPU without),
    sqrt correctly rounded, exp within 1 ulp on each side, so
    |dZ| <= 4u (1 + t d) Z  with u = 2^-53  -> rtol 1e-15 (1 + t d) used as 2e-15 (1 + t d).
  * FP32 Z entries (factor input): FP32 sqrt/exp from the FP64 d^2:
    |dZ| <= (4 + 4 t d) 2^-24 Z.
  * w and Mag: the refined solution meets ||1-Zw||/(||Z|| ||w||) <= 1e-14 (checked by the
    oracle's own residual), max|w - w_ref| / max|w_ref| <= 1e-9, |dMag|/Mag <= 1e-10, the
    same sign pattern ignoring |w_i| < 1e-12 max|w| (the target accuracy of the method).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_2607_23354_gb300")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return M.Context()


def _cloud(n, m, seed, kind="cube"):
    rng = np.random.default_rng(seed)
    if kind == "cube":
        return rng.random((n, m))
    if kind == "normal":
        return rng.standard_normal((n, m)) / math.sqrt(m)
    raise ValueError(kind)


def _dev(X):
    return torch.from_numpy(np.ascontiguousarray(X)).cuda()


def _sign_pattern(w):
    w = np.asarray(w)
    keep = np.abs(w) >= 1e-12 * np.abs(w).max()
    return np.sign(w) * keep


def check_solution(X, t, w_gpu, mag_gpu, w_ref=None, mag_ref=None, rel_tol=1e-14):
    w_gpu = np.asarray(w_gpu)
    rel = oracle.relative_residual(X, t, w_gpu)
    assert rel <= rel_tol, f"relative residual {rel:.3e}"
    if w_ref is not None:
        err = np.abs(w_gpu - w_ref).max() / np.abs(w_ref).max()
        assert err <= 1e-9, f"max|dw|/max|w| = {err:.3e}"
        assert np.array_equal(_sign_pattern(w_gpu), _sign_pattern(w_ref))
    if mag_ref is not None:
        assert abs(mag_gpu - mag_ref) <= 1e-10 * abs(mag_ref), (mag_gpu, mag_ref)
    return rel


# ------------------------------------------------------------ generator K1
@pytest.mark.parametrize("n,m,t", [(2, 1, 1.0), (3, 2, 0.5), (17, 3, 2.0), (129, 8, 1.0), (257, 33, 0.3),
                                   (300, 5, 10.0)])
def test_similarity_fp64_elementwise(ctx, n, m, t):
    X = _cloud(n, m, seed=n * 7 + m)
    Zg = ctx.similarity_matrix(_dev(X), t, "fp64").cpu().numpy()
    Zo = oracle.similarity_matrix(X, t)
    td = t * oracle.distance_matrix(X)
    assert np.all(np.abs(Zg - Zo) <= 2e-15 * (1 + td) * Zo + 1e-300)
    assert np.all(np.diag(Zg) == 1.0)


@pytest.mark.parametrize("n,m,t", [(5, 2, 1.0), (200, 8, 1.0), (260, 16, 0.2)])
def test_similarity_fp32_elementwise(ctx, n, m, t):
    X = _cloud(n, m, seed=n + m)
    Zg = ctx.similarity_matrix(_dev(X), t, "fp32").cpu().numpy().astype(np.float64)
    Zo = oracle.similarity_matrix(X, t)
    td = t * oracle.distance_matrix(X)
    assert np.all(np.abs(Zg - Zo) <= (4 + 4 * td) * 2.0 ** -24 * Zo + 1e-38)


def test_min_distance(ctx):
    X = _cloud(700, 4, seed=3)
    dmin, tb = ctx.min_distance(_dev(X))
    assert dmin == pytest.approx(oracle.min_distance(X), rel=1e-15)
    assert tb == pytest.approx(oracle.tplus_bound(X), rel=1e-15)
    G = workloads.grid_support_cloud()
    dmin, tb = ctx.min_distance(_dev(G))
    assert dmin == 1.0 and tb == pytest.approx(math.log(len(G) - 1), rel=1e-15)


# --------------------------------------------------------------- factor K2
@pytest.mark.parametrize("n", [3, 128, 129, 300])
def test_cholesky_fp64_elementwise(ctx, n):
    X = _cloud(n, 3, seed=n)
    t = 2.0
    Lg = ctx.cholesky_factor(_dev(X), t, "fp64").cpu().numpy()
    Lo = oracle.cholesky(oracle.similarity_matrix(X, t))
    assert np.abs(Lg - Lo).max() <= 1e-12 * np.abs(Lo).max()


@pytest.mark.parametrize("prec,tol", [("tf32x3", 2e-4), ("tf32", 5e-3), ("fp16x3", 2e-4), ("fp16", 5e-3)])
@pytest.mark.parametrize("n", [130, 300, 1100, 2100, 3300])
def test_cholesky_tensor_core_normwise(ctx, prec, tol, n):
    # one panel (n <= 1024), a trapezoid (1100), several panels (2100, 3300:
    # the look-ahead schedule with a ragged last panel)
    X = _cloud(n, 3, seed=n)
    t = 2.0
    Lg = ctx.cholesky_factor(_dev(X), t, prec).cpu().numpy().astype(np.float64)
    Z = oracle.similarity_matrix(X, t)
    Lo = oracle.cholesky(Z)
    assert np.abs(Lg - Lo).max() <= tol * np.abs(Lo).max()
    assert np.all(np.triu(Lg, 1) == 0)


@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3", "fp16"])
@pytest.mark.parametrize("n,panel,sms", [(3300, 8, 16), (3300, 2, 1), (5000, 4, 40), (2500, 3, 150),
                                         (5000, 4, 0), (3300, 8, -1), (6000, 16, -3)])
def test_lookahead_and_cta_pairs_give_bitwise_the_serial_factor(prec, n, panel, sms):
    # the look-ahead schedule applies the same products to every tile in the
    # same order as the one-stream schedule, so the factors agree exactly;
    # sms > 0 reserves SMs for the panel stream, sms <= 0 shares them through
    # stream priority with trailing CTAs that leave after -sms (default) tasks
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X = _dev(_cloud(n, 4, seed=n + panel))
    base = dict(panel_tiles=panel, lookahead_sms=sms)
    La = M.Context(M.Options(lookahead=True, **base)).cholesky_factor(X, 1.5, prec)
    Ls = M.Context(M.Options(lookahead=False, **base)).cholesky_factor(X, 1.5, prec)
    assert torch.equal(La, Ls)
    assert torch.isfinite(La).all()
    # the CTA-pair kernel (one M=256 MMA per K step over two SMs) forms the
    # same products per output tile in the same order
    for la in (True, False):
        Lp = M.Context(M.Options(lookahead=la, cta_pairs=True, **base)).cholesky_factor(X, 1.5, prec)
        Lq = M.Context(M.Options(lookahead=la, cta_pairs=False, **base)).cholesky_factor(X, 1.5, prec)
        assert torch.equal(Lp, Lq)


def test_cholesky_bf16_well_conditioned(ctx):
    X = _cloud(700, 8, seed=5)
    t = 20.0  # Z close to the identity
    Lg = ctx.cholesky_factor(_dev(X), t, "bf16").cpu().numpy().astype(np.float64)
    Lo = oracle.cholesky(oracle.similarity_matrix(X, t))
    assert np.abs(Lg - Lo).max() <= 2e-2 * np.abs(Lo).max()


def test_bf16_ill_conditioned_reports_not_pd_then_falls_back(ctx):
    X = _cloud(1500, 3, seed=6)
    with pytest.raises(M.MagnitudeError) as e:
        ctx.cholesky_factor(_dev(X), 2.0, "bf16")
    assert e.value.status == M.MAG_ENOTPD
    ctx.set_options(M.Options(precision="bf16"))
    w, mag, info = ctx.solve(_dev(X), 2.0)
    ctx.set_options(M.Options())
    assert info["fallback"] == 2 and info["precision_used"] == M.PREC_FP64
    check_solution(X, 2.0, w.cpu().numpy(), mag, *oracle.weighting(X, 2.0)[:2])


@pytest.mark.parametrize("n", [130, 400])
def test_cholesky_fp32_normwise(ctx, n):
    X = _cloud(n, 8, seed=n)
    t = 3.0
    Lg = ctx.cholesky_factor(_dev(X), t, "fp32").cpu().numpy().astype(np.float64)
    Lo = oracle.cholesky(oracle.similarity_matrix(X, t))
    assert np.abs(Lg - Lo).max() <= 1e-4 * np.abs(Lo).max()
    Z = oracle.similarity_matrix(X, t)
    assert np.abs(Lg @ Lg.T - Z).max() <= 1e-5


# ------------------------------------------------------------ full solve
@pytest.mark.parametrize("prec", ["fp32", "fp64", "tf32x3", "fp16x3", "auto"])
@pytest.mark.parametrize("n,m,t", [(2, 1, 0.7), (3, 2, 1.0), (5, 3, 0.4), (17, 8, 1.0), (129, 8, 1.0),
                                   (257, 16, 0.5), (1000, 8, 1.0), (1031, 3, 10.0), (600, 40, 0.8),
                                   (2500, 8, 1.0), (2049, 3, 30.0)])
def test_solve_matches_oracle(ctx, prec, n, m, t):
    X = _cloud(n, m, seed=1000 + n + m)
    ctx.set_options(M.Options(precision=prec))
    w, mag, info = ctx.solve(_dev(X), t)
    w_ref, mag_ref, _ = oracle.weighting(X, t)
    check_solution(X, t, w.cpu().numpy(), mag, w_ref, mag_ref)
    assert info["rel_residual"] <= 1e-14
    ctx.set_options(M.Options())


@pytest.mark.parametrize("t", [0.01, 0.5, 3.0])
def test_two_point_closed_form_gpu(ctx, t):
    X = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 2.0]])
    w, mag, _ = ctx.solve(_dev(X), t)
    # refinement stops at relative residual 1e-14, so the forward error is
    # bounded by kappa(Z) * 1e-14 with kappa = (1 + z) / (1 - z), z = exp(-3t)
    z = math.exp(-3 * t)
    tol = 2e-14 * (1 + z) / (1 - z)
    np.testing.assert_allclose(w.cpu().numpy(), 1 / (1 + z), rtol=tol)
    assert mag == pytest.approx(2 / (1 + z), rel=tol)


def test_collinear_closed_form_gpu(ctx):
    rng = np.random.default_rng(5)
    gaps = rng.uniform(0.05, 2.0, size=299)
    s = np.concatenate([[0.0], np.cumsum(gaps)])
    u = rng.standard_normal(4)
    u /= np.linalg.norm(u)
    X = s[:, None] * u[None, :]
    t = 1.3
    w, mag, _ = ctx.solve(_dev(X), t)
    assert mag == pytest.approx(1 + np.sum(np.tanh(t * gaps / 2)), rel=1e-12)


def test_rejects_bad_inputs(ctx):
    X = _cloud(50, 3, seed=1)
    Xd = X.copy()
    Xd[7] = Xd[3]
    with pytest.raises(M.MagnitudeError) as e:
        ctx.solve(_dev(Xd), 1.0)
    assert e.value.status == M.MAG_EDUPLICATE
    Xn = X.copy()
    Xn[10, 1] = np.nan
    with pytest.raises(M.MagnitudeError) as e:
        ctx.solve(_dev(Xn), 1.0)
    assert e.value.status == M.MAG_EINVAL
    for t in [0.0, -1.0, float("inf"), float("nan")]:
        with pytest.raises(M.MagnitudeError) as e:
            ctx.solve(_dev(X), t)
        assert e.value.status == M.MAG_EINVAL
    with pytest.raises(M.MagnitudeError) as e:
        ctx.solve(_dev(X[:1]), 1.0)
    assert e.value.status == M.MAG_EINVAL
    # the context stays usable after errors
    w, mag, _ = ctx.solve(_dev(X), 1.0)
    assert mag == pytest.approx(oracle.magnitude(X, 1.0), rel=1e-10)


def test_general_rhs(ctx):
    X = _cloud(300, 4, seed=9)
    b = np.random.default_rng(10).standard_normal(300)
    x, info = ctx.solve_rhs(_dev(X), 0.9, torch.from_numpy(b).cuda())
    xr, _ = oracle.solve(X, 0.9, b=b)
    assert np.abs(x.cpu().numpy() - xr).max() <= 1e-9 * np.abs(xr).max()
    assert oracle.relative_residual(X, 0.9, x.cpu().numpy(), b=b) <= 1e-14


# ------------------------------------------------------------- sweep a8
def test_sweep_grid_support_matches_oracle(ctx):
    G = workloads.grid_support_cloud()
    r = ctx.sweep_tplus(_dev(G), 1e-3, 0.0, 1e-6)
    ro = oracle.tplus(G, 1e-3, 0.0, 1e-6)
    assert r["t_plus"] == pytest.approx(ro["t_plus"], rel=1e-6)
    lo, hi = r["bracket"]
    assert hi - lo <= 1e-6 * hi
    assert r["w"].min().item() >= 0
    assert r["mag"] == pytest.approx(ro["mag"], rel=1e-6)


@pytest.mark.parametrize("cloud", ["grid", "normal120", "kgon12"])
def test_sweep_ridders_matches_oracle(ctx, cloud):
    # Ridders' method on min_j w_j(t), the same bracketed protocol on both sides
    if cloud == "grid":
        X = workloads.grid_support_cloud()
    elif cloud == "normal120":
        X = np.random.default_rng(32).standard_normal((120, 4))
    else:
        k = 12
        X = np.array([[0.0, 0.0]] + [[math.cos(2 * math.pi * j / k), math.sin(2 * math.pi * j / k)]
                                     for j in range(k)])
    r = ctx.sweep_tplus(_dev(X), 1e-3, 0.0, 1e-6, method="ridders")
    ro = oracle.tplus(X, 1e-3, 0.0, 1e-6, method="ridders")
    rb = oracle.tplus(X, 1e-3, 0.0, 1e-6)
    lo, hi = r["bracket"]
    assert hi - lo <= 1e-6 * hi
    assert r["t_plus"] == pytest.approx(ro["t_plus"], rel=1e-6)
    assert r["t_plus"] == pytest.approx(rb["t_plus"], rel=1e-6)
    assert r["w"].min().item() >= 0
    assert r["probes"] < rb["probes"]
    assert ctx.options.tplus_method == "bisection"  # the per-call method did not stick


def test_sweep_below_bracket_collinear(ctx):
    X = np.stack([np.linspace(0, 5, 40), np.zeros(40)], axis=1)
    r = ctx.sweep_tplus(_dev(X), 1e-3, 0.0, 1e-6)
    assert r["below"] and r["t_plus"] == 1e-3 and r["probes"] == 2


def test_sweep_no_bracket(ctx):
    ang = 2 * np.pi * np.arange(12) / 12
    X = np.vstack([[0.0, 0.0], np.stack([np.cos(ang), np.sin(ang)], 1)])
    with pytest.raises(M.MagnitudeError) as e:
        ctx.sweep_tplus(_dev(X), 1e-3, 1.0, 1e-6)
    assert e.value.status == M.MAG_ENOBRACKET


# ------------------------------------------------------------ gradients a9
def test_grad_matches_oracle(ctx):
    X = workloads.normal_cloud(n=512, m=16, seed=4)
    t = 2.0
    dt, dx = ctx.grad(_dev(X), t)
    dto, dxo = oracle.grad(X, t)
    assert dt == pytest.approx(dto, rel=1e-9)
    assert np.abs(dx.cpu().numpy() - dxo).max() <= 1e-9 * np.abs(dxo).max()


def test_grad_general_loss_matches_oracle(ctx):
    X = workloads.normal_cloud(n=300, m=8, seed=6)
    t = 2.0
    w, _, _ = ctx.solve(_dev(X), t)
    g = 2 * w
    dt, dx = ctx.grad(_dev(X), t, w=w, dL_dw=g)
    wo = oracle.weighting(X, t)[0]
    dto, dxo = oracle.grad_loss(X, t, 2 * wo, w=wo)
    assert dt == pytest.approx(dto, rel=1e-8)
    assert np.abs(dx.cpu().numpy() - dxo).max() <= 1e-8 * np.abs(dxo).max()


def test_autograd_function(ctx):
    X = workloads.normal_cloud(n=200, m=4, seed=8)
    Xt = _dev(X).requires_grad_(True)
    tt = torch.tensor(1.5, dtype=torch.float64, requires_grad=True)
    w, mag = M.magnitude(Xt, tt)
    mag.backward()
    dto, dxo = oracle.grad(X, 1.5)
    assert tt.grad.item() == pytest.approx(dto, rel=1e-9)
    assert np.abs(Xt.grad.cpu().numpy() - dxo).max() <= 1e-9 * np.abs(dxo).max()


# --------------------------------------------------------------- batch a10
def test_batch_matches_oracle(ctx):
    clouds, ts = workloads.batch_clouds(count=6, m=8, n_min=20, n_max=300, n_t=3, seed=2)
    ws, mags, sts = ctx.solve_batch([_dev(c) for c in clouds], list(ts))
    assert int(sts.abs().sum()) == 0
    k = 0
    for i, c in enumerate(clouds):
        for j, t in enumerate(ts):
            w_ref, mag_ref, _ = oracle.weighting(c, t)
            check_solution(c, t, ws[k].cpu().numpy(), mags[i, j].item(), w_ref, mag_ref)
            k += 1


# ----------------------------------------------------- residual modes a5
@pytest.mark.parametrize("resid", ["matrix_free", "stored", "auto"])
@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3", "bf16", "fp16", "fp64"])
@pytest.mark.parametrize("n,m,t", [(300, 8, 1.0), (1500, 3, 5.0), (2100, 8, 20.0)])
def test_residual_modes_match_oracle(ctx, resid, prec, n, m, t):
    X = _cloud(n, m, seed=77 + n)
    ctx.set_options(M.Options(precision=prec, residual_mode=resid))
    try:
        w, mag, info = ctx.solve(_dev(X), t)
    finally:
        ctx.set_options(M.Options())
    w_ref, mag_ref, _ = oracle.weighting(X, t)
    check_solution(X, t, w.cpu().numpy(), mag, w_ref, mag_ref)
    if resid == "stored" and prec != "fp64" and info["fallback"] == 0:
        assert info["residual_mode"] == M.RESID_STORED


def test_residual_entry_point_matches_oracle(ctx):
    X = _cloud(700, 5, seed=31)
    t = 0.8
    w_ref = oracle.weighting(X, t)[0]
    w = w_ref + 1e-9 * np.random.default_rng(32).standard_normal(700)  # a perturbed weighting
    r, nr = ctx.residual(_dev(X), t, torch.from_numpy(w).cuda())
    ro, rs = oracle.residual_rows(X, t, w)
    scale = np.abs(rs).max() * np.abs(w).max()
    # exp within 1 ulp each side, d^2 with and without FMA: |dr_j| <= (2 + t d) u sum_k Z_jk |w_k|
    assert np.abs(r.cpu().numpy() - ro).max() <= 2e-15 * scale
    assert nr["rel_residual"] == pytest.approx(np.abs(ro).max() / scale, rel=1e-6)
    assert nr["z_norm_inf"] == pytest.approx(np.abs(rs).max(), rel=1e-14)
    b = np.random.default_rng(33).standard_normal(700)
    r2, _ = ctx.residual(_dev(X), t, torch.from_numpy(w).cuda(), b=torch.from_numpy(b).cuda())
    ro2, _ = oracle.residual_rows(X, t, w, b=b)
    assert np.abs(r2.cpu().numpy() - ro2).max() <= 2e-15 * scale + 4e-16 * np.abs(b).max()


def test_batch_mixed_sizes_and_fallbacks(ctx):
    rng = np.random.default_rng(41)
    clouds = [rng.standard_normal((n, 6)) for n in (2, 5, 64, 129, 700, 2100)]
    bad = rng.standard_normal((40, 3))
    bad[17] = bad[3]  # coincident points: Z singular
    clouds.append(bad)
    ts = [0.3, 3.0]
    ws, mags, sts = ctx.solve_batch([_dev(c) for c in clouds], ts)
    sts = sts.cpu().numpy()
    k = 0
    for i, c in enumerate(clouds):
        for j, t in enumerate(ts):
            if i == len(clouds) - 1:
                assert sts[i, j] == M.MAG_EDUPLICATE
            else:
                assert sts[i, j] == M.MAG_OK
                w_ref, mag_ref, _ = oracle.weighting(c, t)
                check_solution(c, t, ws[k].cpu().numpy(), mags[i, j].item(), w_ref, mag_ref)
            k += 1


def test_batch_config_shape_sample(ctx):
    clouds, ts = workloads.batch_clouds(count=12, seed=5)
    ws, mags, sts = ctx.solve_batch([_dev(c) for c in clouds], list(ts))
    assert int(sts.abs().sum()) == 0
    k = 0
    for i, c in enumerate(clouds):
        for j, t in enumerate(ts):
            if j in (0, 7):  # smallest and largest t against the oracle
                w_ref, mag_ref, _ = oracle.weighting(c, t)
                check_solution(c, t, ws[k].cpu().numpy(), mags[i, j].item(), w_ref, mag_ref)
            else:
                assert oracle.relative_residual(c, t, ws[k].cpu().numpy()) <= 1e-14
            k += 1


@pytest.mark.parametrize("shape,threads,per_sm,tc,left", [(1, 512, 1, 0, 0), (2, 256, 2, 0, 0), (3, 256, 3, 0, 0),
                                                          (4, 256, 2, 1, 0), (5, 256, 3, 1, 0), (6, 256, 2, 0, 1),
                                                          (7, 256, 3, 0, 1)])
def test_batch_every_launch_shape_matches_oracle(shape, threads, per_sm, tc, left):
    # ragged sizes (not multiples of the 64-point factor block, one of 2048)
    # through each launch shape of the batch kernel
    rng = np.random.default_rng(400 + shape)
    clouds = [rng.standard_normal((n, 7)) / 2 for n in (3, 63, 65, 130, 511, 777, 2048)]
    ts = [0.7, 4.0]
    c = M.Context(M.Options(batch_shape=shape))
    ws, mags, sts = c.solve_batch([_dev(x) for x in clouds], ts)
    info = c.last_batch_info
    c.close()
    assert info["batch_threads"] == threads and info["batch_ctas_per_sm"] == per_sm
    assert info["batch_tensor_cores"] == tc and info["batch_left_looking"] == left
    assert int(sts.abs().sum()) == 0
    k = 0
    for i, x in enumerate(clouds):
        for j, t in enumerate(ts):
            if x.shape[0] <= 777:
                w_ref, mag_ref, _ = oracle.weighting(x, t)
                check_solution(x, t, ws[k].cpu().numpy(), mags[i, j].item(), w_ref, mag_ref)
            else:
                assert oracle.relative_residual(x, t, ws[k].cpu().numpy()) <= 1e-14
            k += 1


def test_batch_tuner_picks_a_shape():
    # 130 clouds x 8 t = 1040 problems: at least twice the largest grid
    # (3 CTAs per SM), so the first call tunes the launch shape on a sample
    clouds, ts = workloads.batch_clouds(count=130, m=8, n_min=20, n_max=160, n_t=8, seed=9)
    c = M.Context()
    ws, mags, sts = c.solve_batch([_dev(x) for x in clouds], list(ts))
    info = c.last_batch_info
    ws2, mags2, sts2 = c.solve_batch([_dev(x) for x in clouds], list(ts))
    info2 = c.last_batch_info
    c.close()
    keys = ("batch_threads", "batch_ctas_per_sm", "batch_tensor_cores", "batch_left_looking")
    shape = tuple(info[k] for k in keys)
    assert shape in {(512, 1, 0, 0), (256, 2, 0, 0), (256, 3, 0, 0), (256, 2, 1, 0), (256, 3, 1, 0), (256, 2, 0, 1),
                     (256, 3, 0, 1)}
    assert tuple(info2[k] for k in keys) == shape
    assert int(sts.abs().sum()) == 0 and int(sts2.abs().sum()) == 0
    assert torch.equal(mags, mags2)
    for i in range(0, 130, 26):
        for j in (0, 7):
            x, t = clouds[i], ts[j]
            w_ref, mag_ref, _ = oracle.weighting(x, t)
            check_solution(x, t, ws[i * 8 + j].cpu().numpy(), mags[i, j].item(), w_ref, mag_ref)


@pytest.mark.parametrize("prec,resid", [("fp16x3", "stored"), ("fp16x3", "matrix_free"), ("tf32x3", "stored")])
def test_gmres_ir_finishes_after_refinement_is_cut_short(ctx, prec, resid):
    X = _cloud(1500, 8, seed=61)
    t = 1.0
    ctx.set_options(M.Options(precision=prec, residual_mode=resid, ir_max_iters=1))
    try:
        w, mag, info = ctx.solve(_dev(X), t)
    finally:
        ctx.set_options(M.Options())
    assert info["fallback"] == 1 and info["gmres_iters"] > 0
    assert info["precision_used"] == M.PRECISIONS[prec]
    w_ref, mag_ref, _ = oracle.weighting(X, t)
    check_solution(X, t, w.cpu().numpy(), mag, w_ref, mag_ref)


def test_fp64_exponential_over_its_range(ctx):
    # points i * 2^-4 on a line and t = 32: every t * d_ij = 2 |i - j| is exact,
    # so the FP64 tiles must equal exp(-2 |i - j|) to within two ulps (the
    # device uses its own table-driven exp, the reference is the host libm).
    n = 300
    X = np.zeros((n, 2))
    X[:, 0] = np.arange(n) * 0.0625
    Zg = ctx.similarity_matrix(_dev(X), 32.0, "fp64").cpu().numpy()
    k = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :])
    ref = np.exp(-2.0 * k)
    assert np.all(np.abs(Zg - ref) <= 2 * np.spacing(ref))


@pytest.mark.parametrize("m,offset,kind", [(8, 0.0, "cube"), (20, 0.0, "normal"), (3, 1e6, "cube")])
def test_exact_distances_match_the_oracle(ctx, m, offset, kind):
    # a multi-t call's distances from the quantized coordinates (exact
    # integer sums; m <= 8 with the column coordinates in registers, m = 20
    # the general loop; a cloud far from the origin exercises the exact
    # offset) against FP64 differences and the oracle; ragged n
    X = _cloud(1500 - 37, m, seed=91 + m, kind=kind) + offset
    Xd = _dev(X)
    ts = [1.0, 10.0]
    out = {}
    for exact in (True, False):
        ctx.set_options(M.Options(exact_distances=exact))
        try:
            W, mags, infos = ctx.solve_multi(Xd, ts)
        finally:
            ctx.set_options(M.Options())
        assert all(i["exact_distances"] == int(exact) for i in infos), infos
        out[exact] = (W.cpu().numpy(), mags, infos)
    for k, t in enumerate(ts):
        w_ref, mag_ref, _ = oracle.weighting(X, t)
        for exact in (True, False):
            check_solution(X, t, out[exact][0][k], out[exact][1][k], w_ref, mag_ref)
        # both distance passes agree to the FP64 differences' rounding: the
        # weightings to kappa(Z) times it
        w1, w0 = out[True][0][k], out[False][0][k]
        assert np.abs(w1 - w0).max() <= 1e-10 * np.abs(w0).max()
    d1, d0 = out[True][2][0]["min_distance"], out[False][2][0]["min_distance"]
    assert abs(d1 - d0) <= 4e-16 * d0
    # a single-t solve: distances and Z in one pass from the quantized points
    w_ref, mag_ref, _ = oracle.weighting(X, ts[0])
    for exact in (True, False):
        ctx.set_options(M.Options(exact_distances=exact))
        try:
            w, mag, info = ctx.solve(Xd, ts[0])
        finally:
            ctx.set_options(M.Options())
        assert info["exact_distances"] == int(exact)
        check_solution(X, ts[0], w.cpu().numpy(), mag, w_ref, mag_ref)


def test_fp64_exponential_random_arguments(ctx):
    # points at random multiples of 2^-30 in [0, 1) on a line and t = 64:
    # every t d_ij is an exact FP64 value in [0, 64), the range of the
    # four-FP64-operation exponential (float-float polynomial).  Against an
    # extended-precision reference it is within about half a unit in the
    # last place (the final rounding); a plain-double reference adds its
    # own half unit.
    n = 1500
    rng = np.random.default_rng(61)
    X = np.zeros((n, 1))
    X[:, 0] = rng.integers(0, 2 ** 30, n) * 2.0 ** -30
    Zg = ctx.similarity_matrix(_dev(X), 64.0, "fp64").cpu().numpy()
    a = 64.0 * np.abs(X[:, 0][:, None] - X[:, 0][None, :])
    ext = np.finfo(np.longdouble).nmant >= 63
    ref = np.exp(-a.astype(np.longdouble)) if ext else np.exp(-a)
    ulp = np.spacing(np.exp(-a))
    err = np.abs(Zg.astype(np.longdouble) - ref) / ulp
    assert float(err.max()) <= (0.6 if ext else 1.1), float(err.max())


@pytest.mark.parametrize("resid", ["stored", "matrix_free"])
def test_solve_multi_reuses_distances_and_matches(ctx, resid):
    X = _cloud(1500, 8, seed=71)
    ts = [0.5, 2.0, 30.0]
    ctx.set_options(M.Options(residual_mode=resid))
    try:
        W, mags, infos = ctx.solve_multi(_dev(X), ts)
        for i, t in enumerate(ts):
            w_ref, mag_ref, _ = oracle.weighting(X, t)
            check_solution(X, t, W[i].cpu().numpy(), mags[i], w_ref, mag_ref)
            w1, m1, _ = ctx.solve(_dev(X), t)
            assert abs(m1 - mags[i]) <= 1e-12 * abs(mags[i])
    finally:
        ctx.set_options(M.Options())


# ------------------------------------------------- scale zero (App. C, Eq. scaleZero)

SCALE_ZERO_CASES = ["two", "three", "normal300x5", "ragged129x10", "cube1000x8", "normal2500x3", "grid",
                    "normal700x100"]


@pytest.mark.parametrize("case", SCALE_ZERO_CASES)
def test_scale_zero_matches_oracle(ctx, case):
    rng = np.random.default_rng(1000 + SCALE_ZERO_CASES.index(case))
    if case == "two":
        X = np.array([[0.0, 0.0], [1.5, 0.5]])
    elif case == "three":
        X = np.array([[0.0, 0.0], [3.0, 0.0], [3.0, 0.1]])
    elif case == "grid":
        X = workloads.grid_support_cloud()
    else:
        kind, dims = case[:-len(case.lstrip("abcdefghijklmnopqrstuvwxyz"))], case.lstrip("abcdefghijklmnopqrstuvwxyz")
        n, m = (int(v) for v in dims.split("x"))
        X = rng.random((n, m)) if kind == "cube" else rng.standard_normal((n, m))
    w0, s, info = ctx.scale_zero(_dev(X))
    w0r, sr, ir = oracle.scale_zero(X)
    w0 = w0.cpu().numpy()
    assert info["rel_residual"] <= 1e-14  # of M z = 1, refined in FP64
    assert abs(w0.sum() - 1.0) <= 1e-12
    # backward stability on the paper's system d v = 1 with v = s w0 (FP64 check)
    D = np.sqrt(np.maximum(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1), 0.0))
    v = s * w0
    rel_d = np.abs(1.0 - D @ v).max() / (np.abs(D).sum(1).max() * np.abs(v).max())
    assert rel_d <= 1e-13, rel_d
    # forward error: the refinement leaves ||1 - M z|| <= 1e-14 ||M|| ||z||, so w0
    # agrees with the oracle to kappa(M) 1e-14 (1e-9 when that is smaller), M
    # = 1 1^T - d / c with the library's first c = 4 max_j ||x_j - x_0||
    c = 4.0 * np.sqrt(((X - X[0]) ** 2).sum(1)).max()
    kappa = np.linalg.cond(1.0 - D / c)
    tol = max(1e-9, 2e-14 * kappa)
    assert np.abs(w0 - w0r).max() <= tol * np.abs(w0r).max()
    assert s == pytest.approx(sr, rel=tol)


def test_scale_zero_closed_forms(ctx):
    # points on a line: w0 = 1/2 at the ends, 0 inside, 1^T d^{-1} 1 = 2 / L
    rng = np.random.default_rng(44)
    gaps = rng.uniform(0.05, 2.0, size=299)
    pos = np.concatenate([[0.0], np.cumsum(gaps)])
    u = rng.standard_normal(4)
    u /= np.linalg.norm(u)
    X = pos[:, None] * u[None, :]
    w0, s, _ = ctx.scale_zero(_dev(X))
    expect = np.zeros(300)
    expect[0] = expect[-1] = 0.5
    # d on a line is ill-conditioned (kappa(M) ~ 1e6 here): the forward error
    # is bounded by kappa(M) times the 1e-14 residual of M z = 1
    D = np.abs(pos[:, None] - pos[None, :])
    kappa = np.linalg.cond(1.0 - D / (4.0 * pos[-1]))
    tol = max(1e-11, 2e-14 * kappa)
    np.testing.assert_allclose(w0.cpu().numpy(), expect, atol=0.5 * tol)
    assert s == pytest.approx(2.0 / gaps.sum(), rel=tol)
    # centre + regular 12-gon: v = (1 - (2/k) cot(pi/2k), 1/k, ...)
    k = 12
    ang = 2 * np.pi * np.arange(k) / k
    X = np.vstack([[0.0, 0.0], np.stack([np.cos(ang), np.sin(ang)], axis=1)])
    alpha = 1.0 - (2.0 / k) / math.tan(math.pi / (2 * k))
    v = np.concatenate([[alpha], np.full(k, 1.0 / k)])
    w0, s, _ = ctx.scale_zero(_dev(X))
    np.testing.assert_allclose(w0.cpu().numpy(), v / v.sum(), rtol=1e-12, atol=1e-14)
    assert s == pytest.approx(v.sum(), rel=1e-12)


def test_scale_zero_is_the_small_t_limit_of_the_solver(ctx):
    X = np.random.default_rng(45).standard_normal((500, 3))
    w0, _, _ = ctx.scale_zero(_dev(X))
    w, _, _ = ctx.solve(_dev(X), 1e-4)
    w0 = w0.cpu().numpy()
    assert np.abs(w.cpu().numpy() - w0).max() <= 2e-3 * np.abs(w0).max()


def test_scale_zero_rejects_duplicates(ctx):
    X = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 0.0], [2.0, 3.0]])
    with pytest.raises(M.MagnitudeError) as e:
        ctx.scale_zero(_dev(X))
    assert e.value.status == M.MAG_EDUPLICATE


# ------------------------------------------------- AUTO precision probe
# Below the Gershgorin bound the AUTO policy factors the leading 3072 points
# with the one-product FP16 factor, measures the contraction of two refinement
# steps there and extrapolates it to n.  The three branches: FP16 taken,
# FP16X3 taken, and a wrong FP16 prediction replaced by FP16X3.

def test_auto_probe_takes_fp16_when_refinement_contracts_fast(ctx):
    # [0,1]^8 at t = 10: rows of Z sum to several (no Gershgorin bound) while
    # lambda_min(Z) stays near 0.6, so FP16 refines in a few steps
    X = _cloud(32768, 8, 4242)
    w, mag, info = ctx.solve(_dev(X), 10.0)
    assert info["gershgorin_lmin"] < 0.5
    assert 0.0 <= info["probe_rho"] < 1e-2, info["probe_rho"]
    assert info["precision_used"] == M.PREC_FP16
    assert info["fallback"] == 0
    check_solution(X, 10.0, w.cpu().numpy(), mag)


def test_auto_probe_keeps_the_split_factor_when_ill_conditioned(ctx):
    # [0,1]^8 at t = 1: lambda_min(Z) near 0.08 against row sums in the
    # thousands: FP16 refinement would barely contract
    X = _cloud(16384, 8, 4243)
    w, mag, info = ctx.solve(_dev(X), 1.0)
    assert info["probe_rho"] > 1e-2, info["probe_rho"]
    assert info["precision_used"] == M.PREC_FP16X3
    assert info["fallback"] == 0
    check_solution(X, 1.0, w.cpu().numpy(), mag)


def test_auto_probe_misprediction_falls_back_to_the_split_factor(ctx):
    # the leading 3072 points are far apart (their Z block is the identity, so
    # the probe predicts no error at all) while the other 13312 form one dense
    # cube at t = 0.3, where the FP16 factor cannot drive refinement
    rng = np.random.default_rng(4244)
    spread = rng.random((3072, 8)) * 1e4 + 10.0
    cluster = rng.random((13312, 8))
    X = np.vstack([spread, cluster])
    w, mag, info = ctx.solve(_dev(X), 0.3)
    assert info["probe_rho"] < 1e-6, info["probe_rho"]
    assert info["fallback"] == 3
    assert info["precision_used"] == M.PREC_FP16X3
    check_solution(X, 0.3, w.cpu().numpy(), mag)


@pytest.mark.parametrize("resid", ["stored", "matrix_free"])
def test_solve_where_most_entries_are_below_exp_minus_46(ctx, resid):
    # t = 120 on [0,1]^3: t d > 46 (Z below e^-46, evaluated in FP32 by the
    # solve path) for all pairs farther apart than 0.38, i.e. most of them;
    # weights and magnitude still match the FP64 oracle, and the oracle's own
    # FP64 residual of the GPU weighting meets the tolerance
    X = _cloud(2000, 3, 4245)
    t = 120.0
    ctx.set_options(M.Options(residual_mode=resid))
    try:
        w, mag, info = ctx.solve(_dev(X), t)
    finally:
        ctx.set_options(M.Options())
    w_ref, mag_ref, _ = oracle.weighting(X, t)
    check_solution(X, t, w.cpu().numpy(), mag, w_ref, mag_ref)
    # the similarity matrix entry point keeps every entry FP64-exact
    Zg = ctx.similarity_matrix(_dev(X[:300]), t, "fp64").cpu().numpy()
    Zo = oracle.similarity_matrix(X[:300], t)
    td = t * oracle.distance_matrix(X[:300])
    assert np.all(np.abs(Zg - Zo) <= 2e-15 * (1 + td) * Zo + 1e-300)


def test_stored_residual_on_separated_clusters(ctx):
    # six clusters of 256 points (two tiles each), centres 3 apart, radius
    # 0.3, t = 25: every tile between two clusters holds only entries near
    # e^-60 (evaluated in FP32 by the solve path's generator) next to
    # well-coupled diagonal blocks; weights, magnitude and the oracle's FP64
    # residual match
    rng = np.random.default_rng(4246)
    centres = np.array([[3.0 * i, 0.0, 0.0] for i in range(6)])
    pts = []
    for c in centres:
        v = rng.standard_normal((256, 3))
        v *= 0.3 * rng.random((256, 1)) ** (1 / 3) / np.linalg.norm(v, axis=1, keepdims=True)
        pts.append(c + v)
    X = np.vstack(pts)
    t = 25.0
    ctx.set_options(M.Options(residual_mode="stored"))
    try:
        w, mag, info = ctx.solve(_dev(X), t)
    finally:
        ctx.set_options(M.Options())
    assert info["residual_mode"] == M.RESID_STORED
    w_ref, mag_ref, _ = oracle.weighting(X, t)
    check_solution(X, t, w.cpu().numpy(), mag, w_ref, mag_ref)


@pytest.mark.parametrize("n,m,t", [(9000, 8, 1.0), (4500, 3, 0.3), (130, 16, 5.0)])
def test_matrix_free_refinement_over_the_lower_triangle(ctx, n, m, t):
    # the solver's matrix-free residual visits each lower tile once and uses
    # its entries for two row blocks; several row blocks and a ragged tail
    X = _cloud(n, m, seed=n + m)
    ctx.set_options(M.Options(residual_mode="matrix_free"))
    try:
        w, mag, info = ctx.solve(_dev(X), t)
    finally:
        ctx.set_options(M.Options())
    assert info["residual_mode"] == M.RESID_MATRIX_FREE
    w_ref, mag_ref, _ = oracle.weighting(X, t)
    check_solution(X, t, w.cpu().numpy(), mag, w_ref, mag_ref)
    # its ||Z||inf is the oracle's
    _, rs = oracle.residual_rows(X, t, w_ref)
    assert info["z_norm_inf"] == pytest.approx(rs.max(), rel=1e-6)


# ------------------------------------------------- small t: the deflated system
# Near t = 0, Z approaches 1 1^T and kappa(Z) grows like 1/t; mag_solve then
# solves the deflated system A u = 1 (A = (Z - (1 - c t) 1 1^T) / t) and maps u
# back to w = Z^{-1} 1 by Sherman-Morrison.  Closed forms fix w exactly.

def _line(n, seed):
    rng = np.random.default_rng(seed)
    gaps = rng.uniform(0.05, 2.0, size=n - 1)
    s = np.concatenate([[0.0], np.cumsum(gaps)])
    u = rng.standard_normal(3)
    u /= np.linalg.norm(u)
    return s[:, None] * u[None, :], gaps


@pytest.mark.parametrize("t", [1e-2, 1e-3, 1e-5])
@pytest.mark.parametrize("deflate", [0, 1])
def test_deflated_small_t_closed_forms(ctx, t, deflate):
    ctx.set_options(M.Options(deflate=deflate))
    try:
        # two points: w = 1 / (1 + e^{-t d})
        X2 = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
        w, mag, info = ctx.solve(_dev(X2), t)
        assert info["deflation_c"] > 0
        np.testing.assert_allclose(w.cpu().numpy(), 1 / (1 + math.exp(-5 * t)), rtol=1e-13)
        # points on a line: the tanh formula (w_1 = (1 + tanh(t g_1/2))/2, ...)
        X, gaps = _line(300, 7)
        w, mag, info = ctx.solve(_dev(X), t)
        far = gaps.sum()  # max_j ||x_j - x_0||
        # deflated when t max d is small: t far <= 1/8 (AUTO), 4 far t <= 1 (forced)
        assert (info["deflation_c"] > 0) == (t * far <= (0.125 if deflate == 0 else 0.25))
        th = np.tanh(t * gaps / 2)
        exact = np.concatenate([[(1 + th[0]) / 2], (th[:-1] + th[1:]) / 2, [(1 + th[-1]) / 2]])
        # the weighting tolerance (1e-9 of max |w|), or kappa times the
        # residual of the system solved where that is larger: Z (kappa 2.5e5
        # at t = 1e-2, where the line is too long for the deflated form) or
        # the deflated A (kappa 6e6 at t = 1e-5 against 5e8 for Z)
        c = info["deflation_c"]
        D = np.linalg.norm(X[:, None, :] - X[None, :, :], axis=2)
        rel = info["rel_residual"]
        if c > 0:
            ct = c * t
            S = 1 + np.expm1(-t * D) / ct
            zn = info["z_norm_inf"]
            rel = rel * zn / (zn - (1 - ct) * len(X))  # A's own relative residual
        else:
            S = np.exp(-t * D)
        kappa = np.linalg.cond(S)
        err = np.abs(w.cpu().numpy() - exact).max() / np.abs(exact).max()
        assert err <= max(1e-9, 10 * kappa * rel), (err, kappa, rel)
        assert mag == pytest.approx(1 + np.sum(th), rel=max(1e-10, err * X.shape[0]))
        assert info["rel_residual"] <= 1e-14
        assert oracle.relative_residual(X, t, w.cpu().numpy()) <= 1e-14
        # centred regular 12-gon (radius 1): w = (a, b, ..., b)
        k = 12
        ang = 2 * np.pi * np.arange(k) / k
        Xk = np.vstack([[0.0, 0.0], np.stack([np.cos(ang), np.sin(ang)], axis=1)])
        w, mag, info = ctx.solve(_dev(Xk), t)
        S = np.sum(np.exp(-2 * t * np.sin(np.pi * np.arange(k) / k)))
        den = S - k * math.exp(-2 * t)
        wk = w.cpu().numpy()
        assert wk[0] == pytest.approx((S - k * math.exp(-t)) / den, rel=1e-9)
        np.testing.assert_allclose(wk[1:], (1 - math.exp(-t)) / den, rtol=1e-9)
    finally:
        ctx.set_options(M.Options())


@pytest.mark.parametrize("n,m,cov", [(1000, 3, "identity"), (3000, 3, "halving"), (2000, 10, "identity")])
def test_deflated_small_t_against_oracle(ctx, n, m, cov):
    # the paper's runtime workload at the bracket's lower end t = 1e-3: the
    # deflated solve needs no FP64 factor; the oracle's FP64 residual of the
    # GPU weighting and the weighting within kappa times the residuals
    X = workloads.paper_runtime_cloud(n, m, cov, 0)
    t = 1e-3
    w, mag, info = ctx.solve(_dev(X), t)
    assert info["deflation_c"] > 0 and info["fallback"] != 2
    wg = w.cpu().numpy()
    assert oracle.relative_residual(X, t, wg) <= 1e-14
    w_ref, mag_ref, oi = oracle.weighting_lapack(X, t)
    bound = max(1e-9, 10 * oi["kappa1_est"] * (1e-14 + oi["rel_residual"]))
    assert np.abs(wg - w_ref).max() <= bound * np.abs(w_ref).max()
    # the plain solve of Z (FP64 factor fallback) agrees within the same bound
    ctx.set_options(M.Options(deflate=-1))
    try:
        w2, mag2, info2 = ctx.solve(_dev(X), t)
    finally:
        ctx.set_options(M.Options())
    assert info2["deflation_c"] == 0
    assert np.abs(w2.cpu().numpy() - wg).max() <= bound * np.abs(wg).max()


def test_deflated_solve_tends_to_scale_zero(ctx):
    # w(t) -> d^{-1} 1 / 1^T d^{-1} 1 with O(t) error (App. C)
    X = np.random.default_rng(91).standard_normal((500, 3))
    w0, _, _ = ctx.scale_zero(_dev(X))
    w0 = w0.cpu().numpy()
    errs = []
    for t in (1e-3, 1e-4):
        w, _, info = ctx.solve(_dev(X), t)
        assert info["deflation_c"] > 0
        errs.append(np.abs(w.cpu().numpy() - w0).max() / np.abs(w0).max())
    assert errs[1] < errs[0] / 5
