"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

None of these re-types the oracle's formula or re-calls its library routine
as the reference: each compares against an independent closed form, an
independent implementation (mpmath, exact rational arithmetic, quadrature),
an invariant, or a hand-written trace of Algorithm 1.
"""
import math
import os
from fractions import Fraction
from itertools import permutations

import mpmath
import numpy as np
import pytest

from oracle import geo_oracle as O
from paper_2003_05324_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ Eq. 1 pins ---
XS = np.concatenate([np.logspace(-6, 0, 25), np.linspace(1.5, 40, 30), [100.0, 300.0, 690.0]])


@pytest.mark.parametrize("nu,closed", [
    (0.5, lambda x: np.exp(-x)),
    (1.5, lambda x: (1 + x) * np.exp(-x)),
    (2.5, lambda x: (1 + x + x * x / 3.0) * np.exp(-x)),
])
def test_matern_half_integer_closed_forms(nu, closed):
    # K_{1/2}, K_{3/2}, K_{5/2} are elementary, so Eq. 1 collapses to these.
    sigma2, beta = 1.7, 0.3
    r = XS * beta
    got = O.matern(r, sigma2, beta, nu)
    want = sigma2 * closed(XS)
    np.testing.assert_allclose(got, want, rtol=2e-13, atol=0)


@pytest.mark.parametrize("nu", [0.3, 1.0, 1.7, 2.2])
def test_matern_general_nu_vs_mpmath(nu):
    sigma2, beta = 1.3, 0.07
    xs = np.array([1e-5, 1e-3, 0.05, 0.4, 1.0, 1.9, 2.1, 5.0, 17.0, 60.0, 300.0])
    got = O.matern(xs * beta, sigma2, beta, nu)
    mpmath.mp.dps = 40
    want = [float(mpmath.mpf(sigma2) / (2 ** (mpmath.mpf(nu) - 1) * mpmath.gamma(nu))
                  * mpmath.mpf(x) ** nu * mpmath.besselk(nu, x)) for x in xs]
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=0)


def _k_quadrature(nu, x):
    # K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt, trapezoid rule in mpmath;
    # the integrand is analytic in a strip, so the rule converges geometrically.
    mpmath.mp.dps = 30
    h = mpmath.mpf(1) / 16
    total = mpmath.mpf(0)
    t = mpmath.mpf(0)
    w = mpmath.mpf(1) / 2
    while True:
        term = mpmath.exp(-x * mpmath.cosh(t)) * mpmath.cosh(nu * t)
        total += w * term
        if t > 2 and term < mpmath.mpf(10) ** -40:
            break
        t += h
        w = 1
    return total * h


@pytest.mark.parametrize("nu", [0.5, 1.0, 1.37])
def test_bessel_k_by_quadrature(nu):
    for x in [0.01, 0.3, 1.0, 2.5, 9.0, 30.0]:
        want = float(_k_quadrature(nu, x))
        # oracle's C(r) at sigma2 = 2^(nu-1) Gamma(nu), beta = 1 is x^nu K_nu(x)
        c = O.matern(np.array([x]), 2 ** (nu - 1) * math.gamma(nu), 1.0, nu)[0]
        assert abs(c / x ** nu - want) <= 1e-13 * want, (nu, x)


@pytest.mark.parametrize("nu", [0.3, 0.5, 1.0, 2.5])
def test_matern_origin_limit(nu):
    # x^nu K_nu(x) -> 2^(nu-1) Gamma(nu) as x -> 0, so C(r) -> theta1; C(0) = theta1.
    s2 = 2.3
    assert O.matern(np.array([0.0]), s2, 0.1, nu)[0] == s2
    small = O.matern(np.array([1e-9]), s2, 0.1, nu)[0]
    assert abs(small - s2) < 1e-3 * s2
    # far field underflows to an exact 0, never NaN
    far = O.matern(np.array([1e6]), s2, 0.1, nu)[0]
    assert far == 0.0


# ------------------------------------------------------------ Eq. 2 pins ---
def _exact_loglik(S, z):
    """Eq. 2 from exact rational det (Gaussian elimination over Q) and exact Z'S^-1 Z."""
    n = len(z)
    M = [[Fraction(float(S[i, j])) for j in range(n)] + [Fraction(float(z[i]))] for i in range(n)]
    det = Fraction(1)
    for c in range(n):
        piv = max(range(c, n), key=lambda r: abs(M[r][c]))
        if piv != c:
            M[c], M[piv] = M[piv], M[c]
            det = -det
        det *= M[c][c]
        for r in range(c + 1, n):
            f = M[r][c] / M[c][c]
            for cc in range(c, n + 1):
                M[r][cc] -= f * M[c][cc]
    sol = [Fraction(0)] * n
    for r in reversed(range(n)):
        acc = M[r][n] - sum(M[r][cc] * sol[cc] for cc in range(r + 1, n))
        sol[r] = acc / M[r][r]
    quad = sum(Fraction(float(z[i])) * sol[i] for i in range(n))
    return -0.5 * n * math.log(2 * math.pi) - 0.5 * math.log(float(det)) - 0.5 * float(quad), det


def _leibniz_det(S):
    n = S.shape[0]
    total = Fraction(0)
    for perm in permutations(range(n)):
        inv = sum(1 for a in range(n) for b in range(a + 1, n) if perm[a] > perm[b])
        prod = Fraction(1)
        for i in range(n):
            prod *= Fraction(float(S[i, perm[i]]))
        total += -prod if inv % 2 else prod
    return total


@pytest.mark.parametrize("n,nu", [(5, 0.5), (6, 1.0), (8, 1.5)])
def test_loglik_brute_force_small(n, nu):
    x, y = inputs.uniform_points(n, seed=11 + n)
    z = inputs.white_noise(n, seed=3)
    th = O.Theta(1.4, 0.25, nu, 1e-3)
    got = O.loglik_dense(x, y, z, th)
    S = O.covariance(x, y, theta=th)
    want, det = _exact_loglik(S, z)
    assert abs(got["loglik"] - want) <= 1e-12 * abs(want)
    if n <= 6:
        assert _leibniz_det(S) == det
    L, info = O.dense_factor(S)
    assert info == 0
    assert np.linalg.norm(L @ L.T - S) / np.linalg.norm(S) <= 1e-15 * n


def _markov_loglik(x, z, sigma2, beta):
    # nu = 1/2 on sorted 1D points is a Markov (AR(1)-type) process:
    # log|S| = log s2 + sum_{i>=2} log(s2 (1 - rho_i^2)),
    # Z'S^-1 Z = Z_1^2/s2 + sum_{i>=2} (Z_i - rho_i Z_{i-1})^2 / (s2 (1 - rho_i^2)),
    # rho_i = exp(-d_i / beta).
    n = len(z)
    d = np.diff(x)
    rho = np.exp(-d / beta)
    one_m = -np.expm1(-2 * d / beta)
    logdet = math.log(sigma2) + math.fsum(np.log(sigma2 * one_m).tolist())
    quad = z[0] ** 2 / sigma2 + math.fsum(((z[1:] - rho * z[:-1]) ** 2 / (sigma2 * one_m)).tolist())
    return -0.5 * n * math.log(2 * math.pi) - 0.5 * logdet - 0.5 * quad, logdet, quad


# --------------------------------------------- Eq. 1 on 2D locations ---
def test_covariance_right_triangle_by_hand():
    """Three points with hand-computed Euclidean distances 3/10, 4/10, 5/10 (a
    3-4-5 right triangle, legs along x and along y): with nu = 1/2 Eq. 1 is
    sigma2 exp(-r/beta).  A dropped or mis-signed dy term, or a distance taken
    as |dx| + |dy|, changes the (1, 2) and (0, 2) entries."""
    x = np.array([0.1, 0.4, 0.1])
    y = np.array([0.2, 0.2, 0.6])
    th = O.Theta(1.7, 0.25, 0.5, 0.0)
    S = O.covariance(x, y, theta=th)
    d01, d02, d12 = 0.3, 0.4, 0.5
    want = np.array([[1.7, 1.7 * math.exp(-d01 / 0.25), 1.7 * math.exp(-d02 / 0.25)],
                     [1.7 * math.exp(-d01 / 0.25), 1.7, 1.7 * math.exp(-d12 / 0.25)],
                     [1.7 * math.exp(-d02 / 0.25), 1.7 * math.exp(-d12 / 0.25), 1.7]])
    assert np.allclose(S, want, rtol=1e-14, atol=0.0)
    # nu = 3/2 closed form on the same triangle
    S32 = O.covariance(x, y, theta=O.Theta(1.0, 0.25, 1.5, 0.0))
    assert S32[1, 2] == pytest.approx((1 + d12 / 0.25) * math.exp(-d12 / 0.25), rel=1e-14)
    assert S32[0, 2] == pytest.approx((1 + d02 / 0.25) * math.exp(-d02 / 0.25), rel=1e-14)


@pytest.mark.parametrize("angle,shift", [(0.7, (0.05, -0.02)), (math.pi / 2, (0.0, 0.0)), (2.2, (-0.1, 0.3))])
def test_covariance_is_invariant_under_rigid_motion(angle, shift):
    """Eq. 1 depends on the locations only through ||s_a - s_b||: rotating and
    translating the point set leaves Sigma unchanged (to rounding).  A wrong
    sign or weight of either coordinate difference breaks the invariance."""
    x, y = inputs.uniform_points(40, seed=41)
    c, s_ = math.cos(angle), math.sin(angle)
    xr = c * x - s_ * y + shift[0]
    yr = s_ * x + c * y + shift[1]
    for th in (O.Theta(1.3, 0.2, 0.5, 0.01), O.Theta(0.8, 0.3, 1.0, 0.0), O.Theta(1.0, 0.1, 2.2, 0.0)):
        a = O.covariance(x, y, theta=th)
        b = O.covariance(xr, yr, theta=th)
        assert np.allclose(a, b, rtol=1e-12, atol=1e-15)
    # and a reflection across the line y = x swaps the coordinates
    th = O.Theta(1.0, 0.15, 1.5, 0.0)
    assert np.allclose(O.covariance(x, y, theta=th), O.covariance(y, x, theta=th), rtol=1e-13, atol=0.0)


def test_covariance_nugget_only_on_the_diagonal():
    """Sigma(theta) - sigma2 R = tau2 I exactly, with R the unit-variance
    correlation of the same points (sigma2 a power of two and tau2 exactly
    representable, so every step is exact): the nugget sits on the diagonal
    only and nowhere else (reading: Sigma + tau2 I)."""
    x, y = inputs.jittered_grid(7, seed=43)
    for nu in (0.5, 1.0, 1.5):
        S = O.covariance(x, y, theta=O.Theta(2.0, 0.2, nu, 0.25))
        R = O.covariance(x, y, theta=O.Theta(1.0, 0.2, nu, 0.0))
        D = S - 2.0 * R
        assert np.array_equal(D, 0.25 * np.eye(len(x))), nu
    # a cross-covariance (two point sets) carries no nugget even where points coincide
    C = O.covariance(x[:5], y[:5], x[:5], y[:5], theta=O.Theta(2.0, 0.2, 0.5, 0.25))
    assert np.array_equal(np.diag(C), np.full(5, 2.0))


def test_loglik_markov_1d_closed_form():
    n = 600
    x, y = inputs.line_points(n, seed=5, min_gap=0.05)
    z = inputs.white_noise(n, seed=6)
    th = O.Theta(1.2, 0.05, 0.5, 0.0)
    got = O.loglik_dense(x, y, z, th)
    want, ld, q = _markov_loglik(x, z, th.sigma2, th.beta)
    assert abs(got["logdet"] - ld) <= 1e-10 * abs(ld)
    assert abs(got["quad"] - q) <= 1e-10 * abs(q)
    assert abs(got["loglik"] - want) <= 1e-11 * abs(want)


def test_loglik_identity_covariance():
    # beta tiny and spacing >= 1e-3: every off-diagonal exp(-r/beta) underflows to 0.
    x, y = inputs.jittered_grid(12, seed=2)
    n = len(x)
    z = inputs.white_noise(n, seed=4)
    th = O.Theta(1.0, 1e-6, 0.5, 0.0)
    S = O.covariance(x, y, theta=th)
    assert np.array_equal(S, np.eye(n))
    got = O.loglik_dense(x, y, z, th)
    want = -0.5 * n * math.log(2 * math.pi) - 0.5 * math.fsum((z * z).tolist())
    assert got["loglik"] == pytest.approx(want, rel=1e-15)


def test_loglik_sigma2_scaling():
    x, y = inputs.jittered_grid(10, seed=8)
    n = len(x)
    z = inputs.white_noise(n, seed=9)
    base = O.loglik_dense(x, y, z, O.Theta(1.0, 0.2, 1.0, 0.0))
    for s2 in [0.3, 2.0, 17.0]:
        got = O.loglik_dense(x, y, z, O.Theta(s2, 0.2, 1.0, 0.0))["loglik"]
        want = (-0.5 * n * math.log(2 * math.pi) - 0.5 * n * math.log(s2)
                - 0.5 * base["logdet"] - 0.5 * base["quad"] / s2)
        assert got == pytest.approx(want, rel=1e-12)


def test_loglik_permutation_invariance():
    x, y = inputs.jittered_grid(9, seed=10)
    z = inputs.white_noise(len(x), seed=12)
    th = O.Theta(1.0, 0.1, 0.5)
    a = O.loglik_dense(x, y, z, th)["loglik"]
    perm = np.random.default_rng(0).permutation(len(x))
    b = O.loglik_dense(x[perm], y[perm], z[perm], th)["loglik"]
    assert abs(a - b) <= 1e-12 * abs(a)


def test_profile_sigma2_is_argmax():
    # theta1_opt = Z'S~^-1 Z / n maximises Eq. 2 over theta1 (text after Eq. 3).
    x, y = inputs.jittered_grid(10, seed=13)
    z = inputs.white_noise(len(x), seed=14) * 1.7
    s2, prof = O.profile_sigma2(x, y, z, 0.15, 0.5)
    at = O.loglik_dense(x, y, z, O.Theta(s2, 0.15, 0.5))["loglik"]
    assert prof == pytest.approx(at, rel=1e-12)
    for f in [0.99, 1.01, 0.8, 1.25]:
        assert O.loglik_dense(x, y, z, O.Theta(s2 * f, 0.15, 0.5))["loglik"] < at


def test_not_spd_reports_first_failing_row():
    S = np.diag([4.0, 1.0, -2.0, 3.0])
    L, info = O.dense_factor(S)
    assert info == 3
    L2, info2 = O.mp_tile_cholesky(S, 2, 1)
    assert info2 == 3


# ------------------------------------------------------ Algorithm 1 pins ---
def test_alg1_trace_5x5_band2_matches_hand_trace():
    S = np.eye(50) * 3.0 + 0.01
    trace = []
    O.mp_tile_cholesky(S, 10, 2, trace=trace)
    step0 = [t for t in trace if t[3] == 0]
    want = []
    with open(os.path.join(GOLDEN, "alg1_5x5_band2_step0.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                op, i, j, k = line.split()
                want.append((op, int(i), int(j), int(k)))
    assert step0 == want
    # precision map: DP tiles are the diagonal and the first sub-diagonal
    dp = {(i, j) for i in range(5) for j in range(i + 1) if O.tile_is_dp(i, j, 2)}
    assert dp == {(0, 0), (1, 1), (2, 2), (3, 3), (4, 4), (1, 0), (2, 1), (3, 2), (4, 3)}
    # every trailing update appears exactly once per step
    for k in range(5):
        ups = [t for t in trace if t[3] == k and t[0] in ("dgemm", "sgemm", "dsyrk")]
        assert len(ups) == (4 - k) * (5 - k) // 2


def test_alg1_full_band_equals_dense_factor():
    x, y = inputs.jittered_grid(16, seed=15)
    th = O.Theta(1.0, 0.1, 0.5)
    S = O.covariance(x, y, theta=th)
    Ld, _ = O.dense_factor(S)
    p = -(-len(x) // 40)
    Lm, info = O.mp_tile_cholesky(S, 40, p)
    assert info == 0
    assert np.max(np.abs(Lm - Ld)) <= 1e-12


def test_alg1_padding_is_exact():
    x, y = inputs.uniform_points(230, seed=16)
    z = inputs.white_noise(230, seed=17)
    th = O.Theta(1.0, 0.1, 1.0, 1e-6)
    d = O.loglik_dense(x, y, z, th)
    m = O.loglik_mp(x, y, z, th, nb=64, band=4)  # p = 4 (padded to 256), all DP
    assert abs(m["loglik"] - d["loglik"]) <= 1e-11 * abs(d["loglik"])


@pytest.mark.parametrize("band", [1, 2])
def test_alg1_mixed_precision_error_is_fp32_level(band):
    x, y = inputs.jittered_grid(24, seed=18)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    z = inputs.matern_field_rff(x, y, 1.0, 0.1, 0.5, seed=19)
    th = O.Theta(1.0, 0.1, 0.5)
    d = O.loglik_dense(x, y, z, th)
    m = O.loglik_mp(x, y, z, th, nb=48, band=band)
    rel = abs(m["loglik"] - d["loglik"]) / abs(d["loglik"])
    assert 0 < rel < 1e-5


# ------------------------------------------------------------ ordering ---
def test_morton_keys_hand_values():
    x = np.array([0.0, 0.5, 0.0, 1.0, 0.75, 1.0 / 65536])
    y = np.array([0.0, 0.0, 0.5, 1.0, 0.25, 0.0])
    k = O.morton_keys(x, y)
    # 0.5 -> q = 0x8000 (bit 15): x bit 15 -> key bit 30, y bit 15 -> key bit 31
    # 1.0 clamps to 0xFFFF: all 32 bits set
    # 0.75 -> 0xC000 (bits 15,14 -> key bits 30,28); 0.25 -> 0x4000 (bit 14 -> key bit 29)
    assert list(k) == [0, 1 << 30, 1 << 31, 0xFFFFFFFF, (1 << 30) | (1 << 28) | (1 << 29), 1]


def test_morton_order_2x2_z_pattern():
    x = np.array([0.75, 0.25, 0.75, 0.25])
    y = np.array([0.75, 0.75, 0.25, 0.25])
    # Z pattern: (lo x, lo y), (hi x, lo y), (lo x, hi y), (hi x, hi y)
    assert list(O.morton_order(x, y)) == [3, 2, 1, 0]
    # ties keep the original order
    assert list(O.morton_order(np.array([0.1, 0.1]), np.array([0.2, 0.2]))) == [0, 1]


# --------------------------------------------------------------- kriging ---
def test_krige_interpolates_observed_points():
    x, y = inputs.uniform_points(80, seed=20)
    z = inputs.white_noise(80, seed=21)
    th = O.Theta(1.0, 0.2, 1.5, 0.0)
    pick = np.array([0, 7, 33, 79])
    zhat = O.krige(x, y, z, th, x[pick], y[pick])
    np.testing.assert_allclose(zhat, z[pick], atol=1e-7)


def test_krige_far_point_predicts_zero_mean():
    x, y = inputs.uniform_points(50, seed=22)
    z = inputs.white_noise(50, seed=23)
    th = O.Theta(1.0, 0.01, 0.5, 0.0)
    zhat = O.krige(x, y, z, th, np.array([50.0]), np.array([50.0]))
    assert zhat[0] == 0.0


def test_krige_dst_interpolates_and_reduces_to_full_kriging():
    """DST kriging: a new location on an observed one returns its observation
    for every d; with d covering every tile it is plain kriging."""
    x, y = inputs.uniform_points(90, seed=24)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    z = inputs.white_noise(90, seed=25)
    th = O.Theta(1.0, 0.05, 0.5, 0.0)
    pick = np.array([0, 11, 45, 89])
    for d in (1, 2, 3):
        np.testing.assert_allclose(O.krige_dst(x, y, z, th, x[pick], y[pick], 30, d), z[pick], atol=1e-9)
    xn, yn = inputs.uniform_points(7, seed=26)
    np.testing.assert_allclose(O.krige_dst(x, y, z, th, xn, yn, 30, 3), O.krige(x, y, z, th, xn, yn),
                               rtol=1e-12, atol=1e-14)


def test_krige_dst_d1_is_kriging_from_the_home_block():
    """With d = 1 (independent blocks) the prediction at s is ordinary kriging
    from the observations of the block that holds s's nearest observed point
    alone."""
    x, y = inputs.uniform_points(120, seed=27)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    z = inputs.white_noise(120, seed=28)
    th = O.Theta(1.3, 0.1, 1.5, 1e-6)
    nb = 40
    xn, yn = inputs.uniform_points(9, seed=29)
    got = O.krige_dst(x, y, z, th, xn, yn, nb, 1)
    for q in range(9):
        a = int(np.argmin((x - xn[q]) ** 2 + (y - yn[q]) ** 2))
        b = slice((a // nb) * nb, (a // nb + 1) * nb)
        want = O.krige(x[b], y[b], z[b], th, xn[q:q + 1], yn[q:q + 1])[0]
        assert abs(got[q] - want) <= 1e-10 * max(1.0, abs(want)), (q, got[q], want)


# ------------------------------------------- MLE: the Nelder-Mead simplex ---
def test_nelder_mead_convex_quadratic():
    a = np.array([0.7, -1.3, 2.1])
    w = np.array([1.0, 4.0, 0.25])
    u, f, evals, iters = O.nelder_mead(lambda u: float(np.sum(w * (u - a) ** 2)), [0.0, 0.0, 0.0],
                                       step=0.5, max_evals=2000, xtol=1e-10)
    assert np.max(np.abs(u - a)) <= 1e-6 and f <= 1e-11 and evals <= 2000 and iters > 0


def test_nelder_mead_rosenbrock():
    def rosen(u):
        return float(100.0 * (u[1] - u[0] ** 2) ** 2 + (1.0 - u[0]) ** 2)
    u, f, evals, _ = O.nelder_mead(rosen, [-1.2, 1.0], step=0.5, max_evals=5000, xtol=1e-12)
    assert np.max(np.abs(u - 1.0)) <= 1e-5 and f <= 1e-10


def test_nelder_mead_bounds_and_budget():
    # the unconstrained minimum (3, -3) lies outside the box: the result is its corner
    calls = []
    def f(u):
        calls.append(u.copy())
        return float((u[0] - 3.0) ** 2 + (u[1] + 3.0) ** 2)
    u, _, evals, _ = O.nelder_mead(f, [0.0, 0.0], step=0.3, max_evals=400, xtol=1e-9, lo=[-1, -1], hi=[1, 1])
    assert np.allclose(u, [1.0, -1.0], atol=1e-7)
    assert all(np.all(c >= -1) and np.all(c <= 1) for c in calls)
    # a budget is never exceeded, and the best point seen is returned
    calls.clear()
    u, fb, evals, _ = O.nelder_mead(f, [0.0, 0.0], step=0.3, max_evals=7)
    assert evals == len(calls) == 7 and fb == min(f(c) for c in calls[:7])


def _ar1_field(x, sigma2, beta, seed):
    # exact simulation of the nu = 1/2 (exponential) process on sorted 1D points
    w = inputs.white_noise(len(x), seed)
    z = np.empty(len(x))
    z[0] = math.sqrt(sigma2) * w[0]
    rho = np.exp(-np.diff(x) / beta)
    for i in range(1, len(x)):
        z[i] = rho[i - 1] * z[i - 1] + math.sqrt(sigma2 * (1.0 - rho[i - 1] ** 2)) * w[i]
    return z


def _markov_argmax(x, z):
    # theta-hat of the 1D Markov likelihood without any simplex: for fixed beta
    # the maximising sigma2 is Q_1(beta)/n, and the profile in log beta is
    # maximised by a grid search refined with bounded Brent.
    from scipy.optimize import minimize_scalar
    n = len(z)
    def neg_profile(lb):
        _, ld1, q1 = _markov_loglik(x, z, 1.0, math.exp(lb))
        return -(-0.5 * n * math.log(2 * math.pi) - 0.5 * n - 0.5 * n * math.log(q1 / n) - 0.5 * ld1)
    grid = np.linspace(math.log(1e-4), math.log(2.0), 400)
    vals = [neg_profile(g) for g in grid]
    j = int(np.argmin(vals))
    res = minimize_scalar(neg_profile, bounds=(grid[max(j - 1, 0)], grid[min(j + 1, len(grid) - 1)]),
                          method="bounded", options={"xatol": 1e-12})
    beta = math.exp(res.x)
    _, _, q1 = _markov_loglik(x, z, 1.0, beta)
    return q1 / n, beta


@pytest.mark.parametrize("profile", [False, True])
def test_mle_markov_1d_matches_closed_form_argmax(profile):
    n = 2000
    x, y = inputs.line_points(n, seed=21, min_gap=0.02)
    z = _ar1_field(x, 1.3, 0.08, seed=22)
    s2_hat, b_hat = _markov_argmax(x, z)
    def evaluate(th):
        _, ld, q = _markov_loglik(x, z, th.sigma2, th.beta)
        return ld, q
    res = O.mle(x, y, z, O.Theta(0.5, 0.05, 0.5), max_evals=400, xtol=1e-9, profile=profile, fix_nu=True,
                evaluate=evaluate)
    assert abs(res["theta"].beta - b_hat) <= 1e-6 * b_hat
    assert abs(res["theta"].sigma2 - s2_hat) <= 1e-6 * s2_hat


def test_mle_dense_objective_follows_the_same_path():
    # the dense definition of Eq. 2 and the Markov closed form agree to ~1e-12,
    # so the simplex takes the same steps with either objective
    n = 240
    x, y = inputs.line_points(n, seed=23, min_gap=0.02)
    z = _ar1_field(x, 0.9, 0.1, seed=24)
    def markov(th):
        _, ld, q = _markov_loglik(x, z, th.sigma2, th.beta)
        return ld, q
    th0 = O.Theta(0.5, 0.05, 0.5)
    a = O.mle(x, y, z, th0, max_evals=60, fix_nu=True)
    b = O.mle(x, y, z, th0, max_evals=60, fix_nu=True, evaluate=markov)
    assert a["evals"] == b["evals"] and a["iterations"] == b["iterations"]
    assert abs(a["theta"].beta - b["theta"].beta) <= 1e-9 * b["theta"].beta
    assert abs(a["theta"].sigma2 - b["theta"].sigma2) <= 1e-9 * b["theta"].sigma2


def test_nelder_mead_hand_traced_steps():
    # f = u0^2 + 2 u1^2 from (1, 1), step 0.5 (worked by hand):
    # simplex (1,1) 3, (1.5,1) 4.25, (1,1.5) 5.5; centroid (1.25,1);
    # reflection (1.5,0.5) 2.75 beats the best, expansion (1.75,0) 3.0625 does
    # not beat it -> keep the reflection.  Next: centroid of (1.5,.5),(1,1) is
    # (1.25,.75), worst (1.5,1): reflection (1,.5) 1.5, expansion (.75,.25)
    # 0.6875 -> keep the expansion.  Seven evaluations.
    u, f, evals, iters = O.nelder_mead(lambda u: float(u[0] ** 2 + 2 * u[1] ** 2), [1.0, 1.0], step=0.5,
                                       max_evals=7)
    assert evals == 7 and iters == 2
    assert np.allclose(u, [0.75, 0.25], rtol=0, atol=1e-15) and abs(f - 0.6875) <= 1e-15
    # 1D, f = u^2 from 0.2, step 1: simplex 0.2 (.04), 1.2 (1.44); reflection
    # -0.8 (.64) -> outside contraction -0.3 (.09), accepted; then reflection
    # 0.7 (.49) is worse than the worst -> inside contraction -0.05 (.0025).
    u, f, evals, iters = O.nelder_mead(lambda u: float(u[0] ** 2), [0.2], step=1.0, max_evals=6)
    assert evals == 6 and iters == 2
    assert abs(u[0] + 0.05) <= 1e-15 and abs(f - 0.0025) <= 1e-16


# ---- DST / IND approximation (Section V-B) --------------------------------
def _dst_problem(m=18, seed=31):
    x, y = inputs.jittered_grid(m, seed=seed)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    z = inputs.white_noise(len(x), seed=seed + 1)
    return x, y, z


def test_dst_band1_is_independent_blocks():
    # d = 1 keeps only the diagonal tiles: Eq. 2 then splits into the blocks'
    # own Eq. 2 (log-det, quadratic form and the n/2 log 2 pi term are additive)
    x, y, z = _dst_problem()
    nb, th = 64, O.Theta(1.0, 0.1, 1.0, 0.0)
    n = len(z)                                     # 324: five full tiles and one of 4 rows
    got = O.loglik_dst(x, y, z, th, nb, 1)
    parts = [O.loglik_dense(x[a:a + nb], y[a:a + nb], z[a:a + nb], th) for a in range(0, n, nb)]
    assert got["logdet"] == pytest.approx(math.fsum(p["logdet"] for p in parts), rel=1e-12)
    assert got["quad"] == pytest.approx(math.fsum(p["quad"] for p in parts), rel=1e-12)
    assert got["loglik"] == pytest.approx(math.fsum(p["loglik"] for p in parts), rel=1e-12)


def test_dst_band2_matches_block_tridiagonal_recursion():
    # d = 2 leaves a block-tridiagonal matrix: block LDL' by the recursion
    # D_k = A_kk - A_k,k-1 D_k-1^-1 A_k-1,k, w_k = z_k - A_k,k-1 D_k-1^-1 w_k-1,
    # log|A| = sum log|D_k| and Z'A^-1 Z = sum w_k' D_k^-1 w_k
    x, y, z = _dst_problem(m=16, seed=41)
    nb, th = 48, O.Theta(1.3, 0.04, 0.5, 0.0)   # short range: the truncated matrix stays SPD
    n = len(z)
    S = O.covariance(x, y, theta=th)
    cuts = list(range(0, n, nb)) + [n]
    blk = [slice(cuts[t], cuts[t + 1]) for t in range(len(cuts) - 1)]
    logdet, quad = 0.0, 0.0
    D = w = None
    for t, b in enumerate(blk):
        A = S[b, b].copy()
        v = z[b].copy()
        if t > 0:
            C = S[b, blk[t - 1]]
            A -= C @ np.linalg.solve(D, C.T)
            v -= C @ np.linalg.solve(D, w)
        D, w = A, v
        logdet += np.linalg.slogdet(D)[1]
        quad += float(w @ np.linalg.solve(D, w))
    got = O.loglik_dst(x, y, z, th, nb, 2)
    assert got["info"] == 0
    assert got["logdet"] == pytest.approx(logdet, rel=1e-11)
    assert got["quad"] == pytest.approx(quad, rel=1e-10)


def test_dst_full_reach_is_the_dense_likelihood():
    x, y, z = _dst_problem(m=12, seed=51)
    nb, th = 40, O.Theta(0.9, 0.2, 1.5, 0.0)
    p = -(-len(z) // nb)
    want = O.loglik_dense(x, y, z, th)["loglik"]
    for d in (p, p + 3):
        assert O.loglik_dst(x, y, z, th, nb, d)["loglik"] == want
    # one tile diagonal fewer changes the value
    assert O.loglik_dst(x, y, z, th, nb, p - 1)["loglik"] != want


# ----------------------------------- far tier (Section IX extension) pins ---
def test_far_product_hand_values():
    """Slices by hand: row a = (0.3, -0.1): max 0.3 = 0.6 2^-1 -> e = 0,
    t = (76.8, -25.6), a0 = (77, -26), a1 = rint(4096 (-0.2, 0.4)) =
    (-819, 1638).  Row b = (0.75, 0.5): max 0.75 = 0.75 2^0 -> e = 1,
    t = (96, 64) exactly, b0 = (96, 64), b1 = (0, 0)."""
    A = np.array([[0.3, -0.1]])
    B = np.array([[0.75, 0.5]])
    a0, a1 = np.array([77.0, -26.0]), np.array([-819.0, 1638.0])
    b0 = np.array([96.0, 64.0])
    scale = 2.0 ** (0 + 1 - 16)
    want3 = scale * (a0 @ b0 + (a1 @ b0) / 4096.0)
    want1 = scale * (a0 @ b0)
    assert O.far_product(A, B, 3)[0, 0] == want3
    assert O.far_product(A, B, 1)[0, 0] == want1
    # the exact product here differs from the 3-product form only by the
    # rounding of a1 (b1 = 0): |0.3*0.75 - 0.1*0.5 - want3| <= 2 * 2^-13 * 96 * scale
    assert abs((0.3 * 0.75 - 0.1 * 0.5) - want3) <= 2 * 2 ** -13 * 96 * scale


@pytest.mark.parametrize("products,bound_units", [(3, 0.25 + 2 * 128.5 * 2 ** -13 + 2 ** -26),
                                                  (1, 2 * 128.5 * 0.5 + 0.25 + 2 * 128.5 * 2 ** -13)])
def test_far_product_error_bound(products, bound_units):
    """With t = t0 + t1 2^-12 + d, |d| <= 2^-13, and |t0| <= 128, |t1| <= 2048,
    each dropped term is bounded: per contraction index the error of the
    3-product form is at most |t1 2^-12||u1 2^-12| + |t||d_u| + |u||d_t|
    <= 1/4 + 2 (128.5) 2^-13 (+ d d) in units of 2^(e_r + e_c - 16); the
    1-product form also drops t0 u1 2^-12 + t1 2^-12 u0 (<= 128.5 each).  The
    bound holds element by element and is reached to within a factor of a few."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((20, 64)) * np.exp(rng.uniform(-3, 3, size=(20, 1)))
    B = rng.standard_normal((17, 64)).astype(np.float32).astype(np.float64)
    P = O.far_product(A, B, products)
    exact = A @ B.T

    def ex(X):
        m = np.max(np.abs(X.astype(np.float32)), axis=1).astype(np.float64)
        return np.frexp(m)[1] + 1
    unit = np.ldexp(1.0, ex(A)[:, None] + ex(B)[None, :] - 16)
    err = np.abs(P - exact) / unit
    assert np.all(err <= 64 * bound_units)
    assert err.max() >= bound_units / 8          # the dropped terms are really there


def test_far_product_full_tier_would_be_exact_to_fp32_level():
    """Keeping every slice pair makes the product the exact one up to the
    second rounding only: a check that the slices carry the value (the a1
    slice is the next 12 bits, not a lost term)."""
    rng = np.random.default_rng(4)
    A = rng.standard_normal((8, 32))
    a = O.far_product(A, np.eye(32), 3)                 # B = I: b0 = 128 on its unit, b1 = 0
    assert np.allclose(a, A, rtol=0, atol=np.max(np.abs(A)) * 2 ** -18)


def test_far_tile_mask_band_and_distance():
    # 3 tiles of 2 points on a line: boxes [0, .1], [.5, .6], [.9, 1.0]
    x = np.array([0.0, 0.1, 0.5, 0.6, 0.9, 1.0])
    y = np.zeros(6)
    m = O.far_tile_mask(x, y, 2, far_band=2)
    assert m.tolist() == [[False, False, False], [False, False, False], [True, False, False]]
    d = O.far_tile_mask(x, y, 2, far_dist=0.35)        # gaps: (1,0) 0.4, (2,1) 0.3, (2,0) 0.8
    assert d.tolist() == [[False, False, False], [True, False, False], [True, False, False]]
    assert not O.far_tile_mask(x, y, 2, far_dist=0.9).any()


def test_far_tier_in_algorithm1():
    """Algorithm 1 with far tiles: no far tile leaves the factor unchanged bit
    for bit; a far tier moves it by more than the FP32 tier's rounding but
    stays within its own per-product bound (3 products: ~2^-16 relative)."""
    x, y = inputs.jittered_grid(16, seed=5)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    S = O.covariance(x, y, theta=O.Theta(1.0, 0.1, 0.5, 1e-3))
    L64, _ = O.dense_factor(S)
    L1, _ = O.mp_tile_cholesky(S, 32, 1)
    none = np.zeros((8, 8), dtype=bool)
    L1b, _ = O.mp_tile_cholesky(S, 32, 1, far=none)
    assert np.array_equal(L1, L1b)
    far = O.far_tile_mask(x, y, 32, far_band=3)
    L3, info = O.mp_tile_cholesky(S, 32, 1, far=far, far_products=3)
    assert info == 0
    e1 = np.max(np.abs(L1 - L64))
    e3 = np.max(np.abs(L3 - L64))
    assert e1 < e3 < 2 ** -10


# --------------------------- the mixed-precision MLE tolerance (Section IV-C) ---
def test_algorithm1_mle_deviation_golden():
    """tests/golden/mle_alg1.json (written by make_mle_alg1.py from oracle calls
    only) holds, for the datasets of the GPU MLE test, the FP64 estimate and the
    estimate on the oracle's own Algorithm 1 likelihood (band 1).  Checked here:
    each stored optimum is an optimum of its own objective against the other's
    point (recomputed at n = 1,600 for two datasets), and the oracle's
    Algorithm 1 itself moves theta-hat along the sigma2-beta ridge by more than
    1e-3 on single datasets (the median stays near 1e-3 at n = 1,600 and grows at
    n = 6,400): the reason the GPU test compares its deviation dataset by
    dataset with the oracle's."""
    import json
    g = json.load(open(os.path.join(GOLDEN, "mle_alg1.json")))
    cases = g["cases"]
    assert {(c["n"], c["profile"]) for c in cases} == {(1600, False), (1600, True), (6400, False)}
    dev = {(c["n"], c["profile"], c["seed"]): max(c["rel_dev"]) for c in cases}
    assert max(v for k, v in dev.items() if k[0] == 1600) > 1e-3
    assert np.median([v for k, v in dev.items() if k[:2] == (1600, False)]) <= 1e-3
    assert np.median([v for k, v in dev.items() if k[0] == 6400]) > 1e-3
    for c in cases:   # the deviation lies along the ridge: sigma2 and beta move together, nu much less
        s2, b, nu = c["rel_dev"]
        assert nu <= max(s2, b)
    for seed in (5, 8):
        c = next(c for c in cases if c["n"] == 1600 and not c["profile"] and c["seed"] == seed)
        x, y = inputs.jittered_grid(40, seed=seed)
        perm = O.morton_order(x, y)
        x, y = x[perm], y[perm]
        z = inputs.matern_field_rff(x, y, 1.0, 0.1, 0.5, seed=seed + 1)
        t64, t1 = O.Theta(*c["fp64"]["theta"]), O.Theta(*c["alg1"]["theta"])
        assert O.loglik_dense(x, y, z, t64)["loglik"] == pytest.approx(c["fp64"]["loglik"], rel=1e-12)
        assert O.loglik_dense(x, y, z, t64)["loglik"] >= O.loglik_dense(x, y, z, t1)["loglik"]
        assert O.loglik_mp(x, y, z, t1, 200, 1)["loglik"] == pytest.approx(c["alg1"]["loglik"], rel=1e-12)
        assert O.loglik_mp(x, y, z, t1, 200, 1)["loglik"] >= O.loglik_mp(x, y, z, t64, 200, 1)["loglik"]
