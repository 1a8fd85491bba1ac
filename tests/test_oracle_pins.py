"""Pins for the CPU FP64 oracle: closed forms, invariants, values the paper
prints, and special cases that reduce to library routines.  None of these
re-types the oracle's own formula; each compares against something the
paper or the mathematics fixes independently.
"""
import math

import numpy as np
import pytest
import scipy.linalg
from scipy.optimize import brentq
from scipy.spatial.distance import pdist, squareform

import oracle


def _rot(m, seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).standard_normal((m, m)))
    return q * np.sign(np.diag(r))


def _collinear(n, m, seed):
    """Sorted points on a random line in R^m, with random gaps."""
    rng = np.random.default_rng(seed)
    gaps = rng.uniform(0.05, 2.0, size=n - 1)
    s = np.concatenate([[0.0], np.cumsum(gaps)])
    u = rng.standard_normal(m)
    u /= np.linalg.norm(u)
    x0 = rng.standard_normal(m)
    return x0 + s[:, None] * u[None, :], gaps, u


def _collinear_w(gaps, t):
    th = np.tanh(t * gaps / 2)
    n = len(gaps) + 1
    w = np.empty(n)
    w[0] = (1 + th[0]) / 2
    w[-1] = (1 + th[-1]) / 2
    w[1:-1] = (th[:-1] + th[1:]) / 2
    return w


def _kgon(k, radius=1.0):
    ang = 2 * np.pi * np.arange(k) / k
    pts = np.stack([np.cos(ang), np.sin(ang)], axis=1) * radius
    return np.vstack([[0.0, 0.0], pts])


def _kgon_S(t, k):
    return np.sum(np.exp(-2 * t * np.sin(np.pi * np.arange(k) / k)))


# ---------------------------------------------------------------- distances

def test_distance_pythagorean_exact():
    X = np.array([[0.0, 0, 0], [2, 3, 6], [1, 2, 2], [0, 3, 4], [-4, 4, 7]])
    D = oracle.distance_matrix(X)
    assert D[0, 1] == 7.0 and D[0, 2] == 3.0 and D[0, 3] == 5.0 and D[0, 4] == 9.0
    assert D[1, 0] == 7.0 and np.all(np.diag(D) == 0.0)


def test_distance_matches_pdist():
    X = np.random.default_rng(1).standard_normal((60, 7)) * 3 + 10
    np.testing.assert_allclose(oracle.distance_matrix(X), squareform(pdist(X)), rtol=2e-15, atol=0)


def test_min_distance_and_bound():
    X = np.random.default_rng(2).random((300, 4))
    dmin = pdist(X).min()
    assert oracle.min_distance(X) == pytest.approx(dmin, rel=1e-15)
    assert oracle.tplus_bound(X) == pytest.approx(math.log(299) / dmin, rel=1e-15)


def test_bound_fig1_identity(paper_values):
    # Fig. 1: 740 unique integer points with min distance 1 give t = log(739) ~ 6.605.
    n = int(paper_values["fig1_n"])
    cells = np.array([(i, j) for i in range(28) for j in range(28)], dtype=float)[:n]
    assert oracle.min_distance(cells) == 1.0
    assert round(oracle.tplus_bound(cells), 3) == paper_values["fig1_bound_t"]


def test_distance_spectrum_app_c3(paper_values):
    # App. C.3: points N(0, I/m), m=128, n=512: largest eigenvalue of d ~ 720.
    X = np.random.default_rng(5).standard_normal((512, 128)) / np.sqrt(128)
    lmax = np.linalg.eigvalsh(oracle.distance_matrix(X))[-1]
    assert lmax == pytest.approx(paper_values["lambda_max_d"], rel=0.02)


def test_similarity_structure():
    X = np.random.default_rng(3).standard_normal((80, 5))
    Z = oracle.similarity_matrix(X, 0.7)
    assert np.all(np.diag(Z) == 1.0)
    assert np.array_equal(Z, Z.T)
    assert np.all(Z > 0) and np.all(Z <= 1)
    # 3-4-5: exactly exp(-5 t)
    Z2 = oracle.similarity_matrix(np.array([[0.0, 0.0], [3.0, 4.0]]), 0.3)
    assert Z2[0, 1] == math.exp(-1.5)
    # Z is positive definite for Euclidean d (Sec. 2)
    assert np.linalg.eigvalsh(Z)[0] > 0


# ----------------------------------------------------------- factor/solves

def test_cholesky_matches_numpy_and_reconstructs():
    A = np.random.default_rng(4).standard_normal((150, 150))
    A = A @ A.T + 150 * np.eye(150)
    L = oracle.cholesky(A)
    np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(L @ L.T, A, rtol=1e-13, atol=1e-11)
    assert np.all(np.triu(L, 1) == 0)


def test_cholesky_rejects_non_pd():
    A = np.eye(5)
    A[3, 3] = -1.0
    with pytest.raises(oracle.OracleError) as e:
        oracle.cholesky(A)
    assert e.value.status == oracle.ENOTPD


def test_triangular_solves_match_scipy():
    rng = np.random.default_rng(5)
    L = np.tril(rng.standard_normal((90, 90))) + 10 * np.eye(90)
    b = rng.standard_normal(90)
    np.testing.assert_allclose(oracle.forward(L, b), scipy.linalg.solve_triangular(L, b, lower=True), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(oracle.backward(L, b),
                               scipy.linalg.solve_triangular(L.T, b, lower=False), rtol=1e-12, atol=1e-15)


# ------------------------------------------------------------ closed forms

@pytest.mark.parametrize("t", [0.01, 0.5, 3.0, 40.0])
@pytest.mark.parametrize("m", [1, 5])
def test_two_point_closed_form(t, m):
    rng = np.random.default_rng(int(t * 100) + m)
    X = rng.standard_normal((2, m))
    d = np.linalg.norm(X[0] - X[1])
    w, mag, info = oracle.weighting(X, t)
    np.testing.assert_allclose(w, 1 / (1 + math.exp(-t * d)), rtol=1e-14)
    assert mag == pytest.approx(2 / (1 + math.exp(-t * d)), rel=1e-14)


@pytest.mark.parametrize("t", [0.05, 1.0, 7.0])
@pytest.mark.parametrize("m", [1, 4])
def test_collinear_closed_form(t, m):
    X, gaps, _ = _collinear(40, m, seed=7 + m)
    w, mag, info = oracle.weighting(X, t)
    exact = _collinear_w(gaps, t)
    np.testing.assert_allclose(w, exact, rtol=5e-12 if t < 0.1 else 1e-13, atol=1e-13)
    assert mag == pytest.approx(1 + np.sum(np.tanh(t * gaps / 2)), rel=1e-12)
    assert info["rel_residual"] < 1e-15


@pytest.mark.parametrize("t,delta", [(0.001, 0.01), (0.3, 0.1), (2.0, 0.05), (10.0, 0.01)])
def test_three_point_example_formula(t, delta):
    # Sec. 2, Example: d_12 = d_13 = 1, d_23 = delta.
    th = math.asin(delta / 2)
    X = np.array([[0.0, 0.0], [math.cos(th), math.sin(th)], [math.cos(th), -math.sin(th)]])
    w, mag, _ = oracle.weighting(X, t)
    den = math.exp((delta + 2) * t) - 2 * math.exp(delta * t) + math.exp(2 * t)
    w1 = (math.exp((delta + 2) * t) - 2 * math.exp((delta + 1) * t) + math.exp(2 * t)) / den
    w2 = (math.exp((delta + 2) * t) - math.exp((delta + 1) * t)) / den
    tol = 1e-9 if t < 0.01 else 1e-12
    np.testing.assert_allclose(w, [w1, w2, w2], rtol=tol)


def test_three_point_example_printed_values(paper_values):
    # Sec. 2, Example: the printed approximate weightings (isolated point first,
    # the order the example's formula uses; the text lists it last).
    def w_at(t, delta=0.01):
        th = math.asin(delta / 2)
        X = np.array([[0.0, 0.0], [math.cos(th), math.sin(th)], [math.cos(th), -math.sin(th)]])
        return oracle.weighting(X, t)[0]

    pv = paper_values
    np.testing.assert_allclose(w_at(1e-3), [pv["ex3_small_t_isolated"], pv["ex3_small_t_pair"],
                                            pv["ex3_small_t_pair"]], atol=0.01)
    np.testing.assert_allclose(w_at(10.0), [pv["ex3_mid_t_isolated"], pv["ex3_mid_t_pair"],
                                            pv["ex3_mid_t_pair"]], atol=0.03)
    np.testing.assert_allclose(w_at(1e4), [pv["ex3_large_t"]] * 3, atol=1e-6)
    # "effective number of points" 1 -> 2 -> 3
    assert sum(w_at(1e-3)) == pytest.approx(1.0, abs=0.01)
    assert sum(w_at(10.0)) == pytest.approx(2.0, abs=0.06)
    assert sum(w_at(1e4)) == pytest.approx(3.0, abs=1e-6)


@pytest.mark.parametrize("k", [5, 12])
@pytest.mark.parametrize("t", [0.3, 1.0, 2.5])
def test_centred_regular_polygon_closed_form(k, t):
    X = _kgon(k)
    w, mag, _ = oracle.weighting(X, t)
    S = _kgon_S(t, k)
    a = (S - k * math.exp(-t)) / (S - k * math.exp(-2 * t))
    b = (1 - math.exp(-t)) / (S - k * math.exp(-2 * t))
    np.testing.assert_allclose(w, [a] + [b] * k, rtol=1e-12, atol=1e-14)


def test_scale_zero_limit():
    # App. C.1, Eq. scaleZero: lim_{t->0} Z^{-1} 1 = d^{-1} 1 / (1^T d^{-1} 1), with O(t) error.
    X = np.random.default_rng(9).random((12, 3))
    v = np.linalg.solve(squareform(pdist(X)), np.ones(12))
    v /= v.sum()
    errs = []
    for t in [1e-3, 1e-4, 1e-5]:
        w, mag, _ = oracle.weighting(X, t)
        errs.append(np.abs(w - v).max())
        assert mag == pytest.approx(1.0, abs=10 * t)
    assert errs[-1] < 1e-5
    assert 5 < errs[0] / errs[1] < 20 and 5 < errs[1] / errs[2] < 20


def test_large_t_magnitude_tends_to_n():
    X = np.random.default_rng(10).random((50, 3))
    dmin = pdist(X).min()
    _, mag, _ = oracle.weighting(X, 60.0 / dmin)
    assert mag == pytest.approx(50.0, rel=1e-12)


# ---------------------------------------------------------------- invariants

def test_invariances_permutation_translation_rotation():
    rng = np.random.default_rng(11)
    X = rng.standard_normal((70, 6))
    t = 1.3
    w, mag, _ = oracle.weighting(X, t)
    p = rng.permutation(70)
    wp, magp, _ = oracle.weighting(X[p], t)
    np.testing.assert_allclose(wp, w[p], rtol=1e-11, atol=1e-13)
    wt, _, _ = oracle.weighting(X + rng.standard_normal(6) * 5, t)
    np.testing.assert_allclose(wt, w, rtol=1e-10, atol=1e-12)
    wr, magr, _ = oracle.weighting(X @ _rot(6, 12).T, t)
    np.testing.assert_allclose(wr, w, rtol=1e-10, atol=1e-12)
    assert magp == pytest.approx(mag, rel=1e-13) and magr == pytest.approx(mag, rel=1e-11)


def test_scaling_law_weights():
    # App. C.2: t_+(lambda d) = t_+(d)/lambda follows from w(t; lambda x) = w(lambda t; x).
    X = np.random.default_rng(13).standard_normal((60, 4))
    w1, _, _ = oracle.weighting(2.0 * X, 0.4)
    w2, _, _ = oracle.weighting(X, 0.8)
    np.testing.assert_array_equal(w1, w2)  # scaling by 2 is exact in binary
    w3, _, _ = oracle.weighting(3.0 * X, 0.4)
    w4, _, _ = oracle.weighting(X, 1.2)
    np.testing.assert_allclose(w3, w4, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("seed,t", [(14, 0.2), (15, 2.0), (16, 20.0)])
def test_refined_residual_is_fp64_level(seed, t):
    X = np.random.default_rng(seed).random((400, 8))
    w, _, info = oracle.weighting(X, t)
    assert info["rel_residual"] <= 1e-15


def test_residual_of_exact_two_point_solution():
    X = np.array([[0.0, 0.0], [3.0, 4.0]])
    t = 0.2
    w = np.full(2, 1 / (1 + math.exp(-1.0)))
    r, rs = oracle.residual_rows(X, t, w)
    assert np.abs(r).max() < 3e-16
    np.testing.assert_allclose(rs, 1 + math.exp(-1.0), rtol=1e-16)
    r2, _ = oracle.residual_rows(X, t, np.zeros(2))
    np.testing.assert_array_equal(r2, [1.0, 1.0])


def _exact_residual_norms(Z, w, b=None):
    """||b - Zw||inf, max row sum of Z and ||w||inf in exact rational
    arithmetic on the given FP64 entries (each rounded once at the end)."""
    from fractions import Fraction
    n = len(w)
    wf = [Fraction(float(v)) for v in w]
    rmax, zmax = Fraction(0), Fraction(0)
    for j in range(n):
        row = [Fraction(float(z)) for z in Z[j]]
        bj = Fraction(1) if b is None else Fraction(float(b[j]))
        rmax = max(rmax, abs(bj - sum(z * v for z, v in zip(row, wf))))
        zmax = max(zmax, sum(row))
    return float(rmax), float(zmax), float(max(abs(v) for v in wf))


@pytest.mark.parametrize("a,b", [(0.3, -0.7), (2.5, 1e-3), (-1e-8, 4.0)])
def test_relative_residual_two_point_closed_form(a, b):
    # two points at distance 5, w = (a, b) far from the solution: r and the
    # norms are closed forms, ||Z||inf = 1 + e^{-5t} (diagonal included)
    X = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    t = 0.3
    z = math.exp(-5 * t)
    r1 = abs(1 - a - z * b)
    r2 = abs(1 - z * a - b)
    expect = max(r1, r2) / ((1 + z) * max(abs(a), abs(b)))
    got = oracle.relative_residual(X, t, np.array([a, b]))
    assert got == pytest.approx(expect, rel=1e-14)
    # a general right-hand side enters r, not the normalisation
    bb = np.array([2.0, -3.0])
    expect_b = max(abs(2 - a - z * b), abs(-3 - z * a - b)) / ((1 + z) * max(abs(a), abs(b)))
    assert oracle.relative_residual(X, t, np.array([a, b]), b=bb) == pytest.approx(expect_b, rel=1e-14)


@pytest.mark.parametrize("seed,t,perturb", [(41, 0.7, 1.0), (42, 3.0, 1e-7)])
def test_relative_residual_against_exact_rational_sums(seed, t, perturb):
    # n = 200 in R^3: the norm step against exact sums of the (pinned) FP64
    # entries of Z; w is the solution plus a perturbation, so the residual is
    # large compared with the rounding of any single row sum
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((200, 3))
    Z = np.exp(-t * squareform(pdist(X)))
    w = scipy.linalg.solve(Z, np.ones(200), assume_a="pos") + perturb * rng.standard_normal(200)
    Zo = oracle.similarity_matrix(X, t)
    rmax, zmax, wmax = _exact_residual_norms(Zo, w)
    got = oracle.relative_residual(X, t, w)
    assert got == pytest.approx(rmax / (zmax * wmax), rel=1e-12)
    r, rs = oracle.residual_rows(X, t, w)
    assert np.abs(r).max() == pytest.approx(rmax, rel=1e-12)
    assert rs.max() == pytest.approx(zmax, rel=1e-15)


def test_solve_info_norms_are_the_relative_residual():
    # orc_solve's info: ||Z||inf and ||x||inf exactly, and its relative
    # residual the one of orc_relative_residual (pinned above) for the same x
    X = np.random.default_rng(43).standard_normal((150, 4))
    b = np.random.default_rng(44).standard_normal(150)
    t = 0.6
    for bb in (None, b):
        x, info = oracle.solve(X, t, b=bb, ir_steps=1)
        _, zmax, wmax = _exact_residual_norms(oracle.similarity_matrix(X, t), x, bb)
        assert info["z_norm_inf"] == pytest.approx(zmax, rel=1e-15)
        assert info["x_norm_inf"] == wmax
        assert info["rel_residual"] == pytest.approx(oracle.relative_residual(X, t, x, b=bb), rel=1e-12)
        assert 0 < info["rel_residual"] <= 1e-15
        w, mag, winfo = oracle.weighting(X, t, ir_steps=1) if bb is None else (None, None, None)
        if bb is None:
            assert winfo["rel_residual"] == pytest.approx(oracle.relative_residual(X, t, w), rel=1e-12)


@pytest.mark.parametrize("t", [0.05, 1.0, 7.0])
def test_weighting_lapack_closed_forms_and_agreement(t):
    # the library-factor weighting: two points, points on a line, the centred
    # 12-gon (closed forms), and the plain-loop weighting on a random cloud
    X2 = np.array([[0.0, 0.0], [3.0, 4.0]])
    w2, mag2, _ = oracle.weighting_lapack(X2, t)
    assert mag2 == pytest.approx(2 / (1 + math.exp(-5 * t)), rel=1e-14)
    Xl, gaps, _ = _collinear(40, 3, seed=31)
    wl, _, info = oracle.weighting_lapack(Xl, t)
    np.testing.assert_allclose(wl, _collinear_w(gaps, t), rtol=1e-12, atol=1e-14)
    assert info["rel_residual"] < 1e-15
    k = 12
    S = _kgon_S(t, k)
    wk, _, _ = oracle.weighting_lapack(_kgon(k), t)
    den = S - k * math.exp(-2 * t)
    assert wk[0] == pytest.approx((S - k * math.exp(-t)) / den, rel=1e-11, abs=1e-13)
    np.testing.assert_allclose(wk[1:], (1 - math.exp(-t)) / den, rtol=1e-11, atol=1e-13)
    X = np.random.default_rng(32).random((400, 5))
    wa, ma, ia = oracle.weighting_lapack(X, t)
    wb, mb, ib = oracle.weighting(X, t)
    assert np.abs(wa - wb).max() <= 1e-10 * np.abs(wb).max()
    assert ma == pytest.approx(mb, rel=1e-12)
    assert ia["min_w"] == wa.min() and ia["rel_residual"] <= 1e-15
    # the condition estimate against the exact 1-norm condition number
    Z = oracle.similarity_matrix(X, t)
    k1 = np.linalg.norm(Z, 1) * np.linalg.norm(np.linalg.inv(Z), 1)
    assert k1 / 3 <= ia["kappa1_est"] <= k1 * 1.0000001


def test_general_rhs_solve_matches_dense_library_solve():
    X = np.random.default_rng(17).standard_normal((120, 3))
    b = np.random.default_rng(18).standard_normal(120)
    x, info = oracle.solve(X, 0.9, b=b)
    Z = np.exp(-0.9 * squareform(pdist(X)))
    np.testing.assert_allclose(x, scipy.linalg.solve(Z, b, assume_a="pos"), rtol=1e-9, atol=1e-11)
    assert info["rel_residual"] < 1e-15


def test_kahan_sum():
    v = np.array([1.0, 1e-16, 1e-16, -1.0] * 10)
    assert oracle.kahan_sum(v) == pytest.approx(20e-16, rel=1e-12)


# ------------------------------------------------------------------ cutoff

def test_tplus_regular_polygon_root():
    k = 12
    X = _kgon(k)
    root = brentq(lambda t: _kgon_S(t, k) - k * math.exp(-t), 0.2, 20.0, xtol=1e-15, rtol=1e-15)
    assert root == pytest.approx(1.235133, abs=1e-6)
    r = oracle.tplus(X, 1e-3, 0.0, 1e-6)
    lo, hi = r["bracket"]
    assert lo <= root + 1e-12 and root - 1e-12 <= hi
    assert hi - lo <= 1e-6 * hi
    assert not r["below"]
    assert r["w"].min() >= 0
    assert 20 <= r["probes"] <= 30


def test_tplus_exact_scaling_law():
    X = np.random.default_rng(19).standard_normal((90, 3))
    r1 = oracle.tplus(X, 1e-3, 0.0, 1e-6)
    r2 = oracle.tplus(2.0 * X, 0.5e-3, oracle.tplus_bound(X) / 2, 1e-6)
    assert r2["t_plus"] == r1["t_plus"] / 2
    assert r2["probes"] == r1["probes"]


def test_tplus_collinear_below_bracket():
    X, _, _ = _collinear(30, 3, seed=20)
    r = oracle.tplus(X, 1e-3, 0.0, 1e-6)
    assert r["below"] and r["t_plus"] == 1e-3 and r["probes"] == 2


def test_tplus_no_bracket():
    with pytest.raises(oracle.OracleError) as e:
        oracle.tplus(_kgon(12), 1e-3, 1.0, 1e-6)
    assert e.value.status == oracle.ENOBRACKET


def test_tplus_ridders_regular_polygon_root():
    # Ridders' method (the paper's preferred root-finder) on min_j w_j(t):
    # the same bracket invariant and width, fewer solves than bisection
    k = 12
    X = _kgon(k)
    root = brentq(lambda t: _kgon_S(t, k) - k * math.exp(-t), 0.2, 20.0, xtol=1e-15, rtol=1e-15)
    r = oracle.tplus(X, 1e-3, 0.0, 1e-6, method="ridders")
    lo, hi = r["bracket"]
    assert lo <= root + 1e-12 and root - 1e-12 <= hi
    assert hi - lo <= 1e-6 * hi
    assert not r["below"] and r["w"].min() >= 0
    assert r["probes"] < oracle.tplus(X, 1e-3, 0.0, 1e-6)["probes"]


def test_tplus_ridders_exact_scaling_law():
    # t and d enter only as t d, and every step of the protocol scales exactly by 2
    X = np.random.default_rng(19).standard_normal((90, 3))
    r1 = oracle.tplus(X, 1e-3, 0.0, 1e-6, method="ridders")
    r2 = oracle.tplus(2.0 * X, 0.5e-3, oracle.tplus_bound(X) / 2, 1e-6, method="ridders")
    assert r2["t_plus"] == r1["t_plus"] / 2
    assert r2["probes"] == r1["probes"]


@pytest.mark.parametrize("seed", [31, 32, 33])
def test_tplus_ridders_agrees_with_bisection(seed):
    X = np.random.default_rng(seed).standard_normal((120, 4))
    rb = oracle.tplus(X, 1e-3, 0.0, 1e-6)
    rr = oracle.tplus(X, 1e-3, 0.0, 1e-6, method="ridders")
    # both brackets hold the sign change and are at most 1e-6 wide
    assert abs(rr["t_plus"] - rb["t_plus"]) <= 1e-6 * rb["t_plus"]
    assert max(rr["bracket"][0], rb["bracket"][0]) <= min(rr["bracket"][1], rb["bracket"][1])
    assert rr["probes"] <= rb["probes"]


def test_tplus_ridders_edge_cases():
    X, _, _ = _collinear(30, 3, seed=20)
    r = oracle.tplus(X, 1e-3, 0.0, 1e-6, method="ridders")
    assert r["below"] and r["t_plus"] == 1e-3 and r["probes"] == 2
    with pytest.raises(oracle.OracleError) as e:
        oracle.tplus(_kgon(12), 1e-3, 1.0, 1e-6, method="ridders")
    assert e.value.status == oracle.ENOBRACKET


def test_tplus_rejects_duplicates():
    X = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 0.0]])
    with pytest.raises(oracle.OracleError) as e:
        oracle.tplus(X)
    assert e.value.status == oracle.EDUPLICATE


def test_tplus_gaussian_law(paper_values):
    # App. C.2, Eq. gaussianCutoff: E t_+ ~ gamma_+ m^(-2/3) n^(1/4) (loose).
    g = paper_values["gamma_plus"]
    for n, m in [(512, 8), (1024, 16)]:
        ts = [oracle.tplus(np.random.default_rng(100 + s).standard_normal((n, m)))["t_plus"] for s in range(3)]
        assert np.mean(ts) == pytest.approx(g * m ** (-2 / 3) * n ** 0.25, rel=0.1)


def test_largest_eigenvalue_at_cutoff(paper_values):
    # App. C.3: m=128, n=512, N(0, I/m): largest eigenvalue of Z(t_+) ~ 3.15 (loose, 4 draws).
    vals = []
    for s in range(4):
        X = np.random.default_rng(200 + s).standard_normal((512, 128)) / np.sqrt(128)
        tp = oracle.tplus(X)["t_plus"]
        vals.append(np.linalg.eigvalsh(oracle.similarity_matrix(X, tp))[-1])
    assert np.mean(vals) == pytest.approx(paper_values["lambda_max_Z_tplus"], rel=0.25)


# --------------------------------------------------------------- gradients

@pytest.mark.parametrize("t", [0.1, 1.5])
def test_grad_two_point_closed_form(t):
    X = np.random.default_rng(21).standard_normal((2, 3))
    d = np.linalg.norm(X[0] - X[1])
    e = math.exp(-t * d)
    dt, dx = oracle.grad(X, t)
    assert dt == pytest.approx(2 * d * e / (1 + e) ** 2, rel=1e-13)
    g = 2 * t * e / (1 + e) ** 2 * (X[0] - X[1]) / d
    np.testing.assert_allclose(dx, [g, -g], rtol=1e-13)


@pytest.mark.parametrize("t", [0.3, 2.0])
def test_grad_collinear_closed_form(t):
    X, gaps, u = _collinear(25, 3, seed=22)
    dt, dx = oracle.grad(X, t)
    sech2 = 1 / np.cosh(t * gaps / 2) ** 2
    assert dt == pytest.approx(np.sum(gaps / 2 * sech2), rel=1e-11)
    dm = np.zeros(25)
    dm[1:] += t / 2 * sech2
    dm[:-1] -= t / 2 * sech2
    np.testing.assert_allclose(dx, dm[:, None] * u[None, :], rtol=1e-9, atol=1e-11)


def test_grad_identities_translation_rotation_euler():
    X = np.random.default_rng(23).standard_normal((60, 4))
    t = 0.8
    dt, dx = oracle.grad(X, t)
    scale = np.abs(dx).max()
    assert np.abs(dx.sum(axis=0)).max() < 1e-11 * scale * 60
    A = dx.T @ X
    assert np.abs(A - A.T).max() < 1e-11 * scale * 60
    assert t * dt == pytest.approx(np.sum(X * dx), rel=1e-11)


def test_grad_central_differences():
    X = np.random.default_rng(24).standard_normal((40, 3))
    t, h = 1.1, 1e-6
    dt, dx = oracle.grad(X, t)
    fd_t = (oracle.magnitude(X, t + h) - oracle.magnitude(X, t - h)) / (2 * h)
    assert dt == pytest.approx(fd_t, rel=1e-7, abs=1e-8)
    for i, l in [(0, 0), (7, 2), (39, 1)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[i, l] += h
        Xm[i, l] -= h
        fd = (oracle.magnitude(Xp, t) - oracle.magnitude(Xm, t)) / (2 * h)
        assert dx[i, l] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_grad_general_loss_adjoint_central_differences():
    # L(w) = ||w||^2: dL/dw = 2w, lambda = Z^{-1} 2w.
    X = np.random.default_rng(25).standard_normal((30, 2))
    t, h = 0.9, 1e-6

    def L(Y, tt):
        w = oracle.weighting(Y, tt)[0]
        return float(w @ w)

    w = oracle.weighting(X, t)[0]
    dt, dx = oracle.grad_loss(X, t, 2 * w, w=w)
    assert dt == pytest.approx((L(X, t + h) - L(X, t - h)) / (2 * h), rel=1e-6)
    for i, l in [(0, 1), (17, 0)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[i, l] += h
        Xm[i, l] -= h
        assert dx[i, l] == pytest.approx((L(Xp, t) - L(Xm, t)) / (2 * h), rel=1e-5, abs=1e-8)


# --------------------------------------------------------- scale zero (App. C)

def test_scale_zero_two_points():
    a = 2.5
    X = np.array([[0.0, 0.0], [a, 0.0]])
    w0, s, info = oracle.scale_zero(X)
    np.testing.assert_allclose(w0, [0.5, 0.5], rtol=1e-15)
    assert s == pytest.approx(2.0 / a, rel=1e-15)


def test_scale_zero_collinear_closed_form():
    # d v = 1 on a line: v = (1, 0, ..., 0, 1) / L, so w0 is 1/2 at the two
    # ends and 0 inside, and 1^T d^{-1} 1 = 2 / L
    X, gaps, _ = _collinear(40, 3, seed=41)
    L = gaps.sum()
    w0, s, info = oracle.scale_zero(X)
    expect = np.zeros(40)
    expect[0] = expect[-1] = 0.5
    np.testing.assert_allclose(w0, expect, atol=1e-12)
    assert s == pytest.approx(2.0 / L, rel=1e-12)


def test_scale_zero_centred_polygon_closed_form():
    # centre + regular k-gon of radius 1: v = (alpha, 1/k, ..., 1/k) with
    # alpha = 1 - (2/k) cot(pi / 2k) (the centre row gives k beta = 1, a
    # vertex row alpha + beta sum_j 2 sin(pi j / k) = 1)
    k = 12
    alpha = 1.0 - (2.0 / k) / math.tan(math.pi / (2 * k))
    v = np.concatenate([[alpha], np.full(k, 1.0 / k)])
    w0, s, _ = oracle.scale_zero(_kgon(k))
    assert alpha < 0  # the centre carries a negative weight at scale zero
    np.testing.assert_allclose(w0, v / v.sum(), rtol=1e-12, atol=1e-14)
    assert s == pytest.approx(v.sum(), rel=1e-12)


def test_scale_zero_is_the_small_t_limit():
    # Eq. scaleZero: Z(t)^{-1} 1 -> d^{-1} 1 / 1^T d^{-1} 1 as t -> 0, with O(t)
    # error; the weighting side is the Cholesky path of Z, the limit side the
    # pivoted LU of d
    X = np.random.default_rng(42).standard_normal((60, 3))
    w0, _, _ = oracle.scale_zero(X)
    errs = []
    for t in (1e-3, 1e-4):
        w, _, _ = oracle.weighting(X, t)
        errs.append(np.abs(w - w0).max() / np.abs(w0).max())
    assert errs[1] < 2e-3
    assert errs[0] / errs[1] == pytest.approx(10.0, rel=0.2)


def test_scale_zero_matches_scipy_and_invariances():
    rng = np.random.default_rng(43)
    X = rng.standard_normal((150, 6))
    w0, s, info = oracle.scale_zero(X)
    D = scipy.spatial.distance.cdist(X, X)
    v = scipy.linalg.solve(D, np.ones(150))
    np.testing.assert_allclose(w0, v / v.sum(), rtol=1e-9, atol=1e-12)
    assert info["rel_residual"] < 1e-15
    assert w0.sum() == pytest.approx(1.0, rel=1e-14)
    # permutation, translation + rotation, scaling (w0 is scale-free, s scales as 1/lambda)
    perm = rng.permutation(150)
    np.testing.assert_allclose(oracle.scale_zero(X[perm])[0], w0[perm], rtol=1e-10, atol=1e-13)
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    np.testing.assert_allclose(oracle.scale_zero(X @ Q + 3.0)[0], w0, rtol=1e-9, atol=1e-12)
    w2, s2, _ = oracle.scale_zero(2.0 * X)
    np.testing.assert_allclose(w2, w0, rtol=1e-12, atol=1e-14)
    assert s2 == pytest.approx(s / 2.0, rel=1e-12)


def test_scale_zero_rejects_duplicates():
    X = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 0.0]])
    with pytest.raises(oracle.OracleError) as e:
        oracle.scale_zero(X)
    assert e.value.status == oracle.EDUPLICATE
