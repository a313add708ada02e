"""Plain CPU oracle for the mixed-precision Gaussian log-likelihood.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
module: only the tests, the package smoke check and the CPU-baseline leg of
the benchmark use it.  It shares no code with the CUDA path (the seeded input
draws come from a separate module that holds none of the arithmetic below).

Everything is float64 unless a step of Algorithm 1 fixes single precision.
Library primitives (LAPACK's potrf and triangular solves through scipy,
BLAS matrix products through numpy, the modified Bessel function K_nu from
scipy.special) serve as steps; there is no blocking, fusion or reordering
beyond what the paper's definitions and Algorithm 1 state.

Paper: Abdulah, Ltaief, Sun, Genton, Keyes, "Geostatistical Modeling and
Prediction Using Mixed-Precision Tile Cholesky Factorization" (2019).

Function -> paper passage -> what pins it (tests/test_oracle_pins.py):
  morton_keys / morton_order   "appropriate ordering" (Section VI, mixed-
                               precision Cholesky); Z-order reading    hand-worked
                                                                        keys, 2x2 grid
  matern                       Eq. 1                                    closed forms
                                                                        nu=1/2,3/2,5/2,
                                                                        mpmath K_nu,
                                                                        quadrature, r->0
  covariance                   Eq. 1 with Sigma_ij = C(||s_i-s_j||)     symmetry, diag
  loglik_dense                 Eq. 2                                    n<=8 exact
                                                                        rational det and
                                                                        solve; 1D Markov
                                                                        closed form;
                                                                        Sigma=I; sigma2
                                                                        scaling
  mp_tile_cholesky             Algorithm 1                              band=p equals the
                                                                        dense factor;
                                                                        Fig. 2 op trace
  far_product / far_tile_mask  three-precision extension (Section IX,  exact integer
                               future work): reduced products for far   slices (hand
                               tiles (reading: 8/12-bit row-scaled      values), error
                               slices, 1 or 3 products)                 bounds vs sgemm
  loglik_mp                    Eq. 2 on the Algorithm 1 factor          within FP32-level
                                                                        error of dense
  dst_covariance / loglik_dst   DST / IND approximation (Section V-B)  d = 1: sum of the
                                                                        blocks' own Eq. 2;
                                                                        d >= p: dense Eq. 2
  krige                        prediction (Section VIII-D); simple       interpolation at
                               kriging reading                          observed points
  profile_sigma2               Eq. 3 and theta1_opt = Z'S~^-1 Z / n     argmax of Eq. 2
                                                                        over theta1
  nelder_mead                  the MLE's optimizer (Section IV-C: the  convex quadratic,
                               paper uses NLopt with tolerance 1e-3;    Rosenbrock, 1D
                               reading: Nelder & Mead 1965 simplex)     Markov MLE vs a
                                                                        grid search
  mle                          the estimator theta-hat maximising Eq. 2 1D Markov MLE vs
                               (all three parameters, or Eq. 3's two    a grid search of
                               with theta1 profiled)                    the closed form
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.special as sps

__all__ = [
    "morton_keys", "morton_order", "matern", "covariance", "loglik_dense",
    "dense_factor", "mp_tile_cholesky", "loglik_mp", "factor_logdet_quad",
    "krige", "profile_sigma2", "Theta", "tile_is_dp", "nelder_mead", "mle", "profile_loglik",
    "far_tile_mask", "far_product",
]

LOG_2PI = math.log(2.0 * math.pi)


@dataclass(frozen=True)
class Theta:
    """theta1 (variance sigma2), theta2 (range beta), theta3 (smoothness nu) of Eq. 1,
    plus a nugget tau2 added to the diagonal (reading: Sigma + tau2 I)."""
    sigma2: float
    beta: float
    nu: float
    nugget: float = 0.0


# ---------------------------------------------------------------- ordering ---
def morton_keys(x, y):
    """Z-order key of each location (reading of the paper's 'appropriate ordering').

    Each coordinate c in [0,1] is quantised to q = clamp(floor(c * 2^16), 0, 2^16-1);
    the key interleaves the 16 bits of qx (even bit positions) with those of qy
    (odd bit positions).  Bit by bit, plainly.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    keys = np.empty(x.shape[0], dtype=np.uint64)
    for idx in range(x.shape[0]):
        qx = min(max(int(math.floor(x[idx] * 65536.0)), 0), 65535)
        qy = min(max(int(math.floor(y[idx] * 65536.0)), 0), 65535)
        k = 0
        for b in range(16):
            k |= ((qx >> b) & 1) << (2 * b)
            k |= ((qy >> b) & 1) << (2 * b + 1)
        keys[idx] = k
    return keys


def morton_order(x, y):
    """Permutation perm (new position -> old index) sorting by (key, old index)."""
    keys = morton_keys(x, y)
    return np.array(sorted(range(len(keys)), key=lambda i: (int(keys[i]), i)), dtype=np.int64)


# ------------------------------------------------------------------ Eq. 1 ---
def matern(r, sigma2, beta, nu):
    """Eq. 1: C(r) = theta1 / (2^(theta3-1) Gamma(theta3)) (r/theta2)^theta3 K_theta3(r/theta2).

    C(0) = theta1 (the limit of x^nu K_nu(x) at 0 is 2^(nu-1) Gamma(nu)); where
    K_nu underflows to 0 the product is 0.
    """
    r = np.asarray(r, dtype=np.float64)
    xr = r / beta
    out = np.empty_like(xr)
    zero = xr == 0.0
    xs = xr[~zero]
    kv = sps.kv(nu, xs)
    with np.errstate(invalid="ignore", over="ignore"):
        val = sigma2 / (2.0 ** (nu - 1.0) * sps.gamma(nu)) * np.power(xs, nu) * kv
    val = np.where(kv == 0.0, 0.0, val)
    out[~zero] = val
    out[zero] = sigma2
    return out


def covariance(xa, ya, xb=None, yb=None, theta: Theta = None):
    """Sigma_ab = C(||s_a - s_b||_2) by Eq. 1.  With one set of points the
    nugget is added on the diagonal (a == b); a cross-covariance gets none."""
    xa = np.asarray(xa, dtype=np.float64)
    ya = np.asarray(ya, dtype=np.float64)
    same = xb is None
    if same:
        xb, yb = xa, ya
    dx = xa[:, None] - np.asarray(xb, dtype=np.float64)[None, :]
    dy = ya[:, None] - np.asarray(yb, dtype=np.float64)[None, :]
    r = np.sqrt(dx * dx + dy * dy)
    S = matern(r, theta.sigma2, theta.beta, theta.nu)
    if same:
        S[np.diag_indices_from(S)] = theta.sigma2 + theta.nugget
    return S


# ------------------------------------------------------------------ Eq. 2 ---
def dense_factor(S):
    """Lower Cholesky factor by LAPACK dpotrf; info>0 is the 1-based order of
    the first leading minor that is not positive definite."""
    c, info = sla.lapack.dpotrf(np.asarray(S, dtype=np.float64), lower=1, clean=1)
    return np.tril(c), int(info)


def factor_logdet_quad(L, z):
    """log|Sigma| = 2 sum log L_ii and Q = Z' Sigma^-1 Z = ||L^-1 Z||^2 (Eq. 2)."""
    d = np.diag(L)
    logdet = 2.0 * math.fsum(np.log(d).tolist())
    yv = sla.solve_triangular(L, np.asarray(z, dtype=np.float64), lower=True)
    quad = math.fsum((yv * yv).tolist())
    return logdet, quad


def _assemble(n, logdet, quad):
    return -0.5 * n * LOG_2PI - 0.5 * logdet - 0.5 * quad


def loglik_dense(x, y, z, theta: Theta):
    """Eq. 2 in float64 on the dense covariance: l = -n/2 log 2pi - 1/2 log|S| - 1/2 Z'S^-1 Z."""
    n = len(z)
    S = covariance(x, y, theta=theta)
    L, info = dense_factor(S)
    if info != 0:
        return dict(loglik=float("nan"), logdet=float("nan"), quad=float("nan"), info=info)
    logdet, quad = factor_logdet_quad(L, z)
    return dict(loglik=_assemble(n, logdet, quad), logdet=logdet, quad=quad, info=0)


# ------------------------------------------------------------ Algorithm 1 ---
def tile_is_dp(i, j, band):
    """Precision map of Algorithm 1: lower tile (i, j), i >= j, is double
    precision iff it lies within `band` (diag_thick) tiles of the diagonal."""
    return abs(i - j) < band


def far_tile_mask(x, y, nb, far_band=None, far_dist=None):
    """Which lower tiles (i, j) fall in the far tier of the three-precision
    extension (Section IX names it as future work; reading: a third tier beyond
    the FP32 one).  A tile is far when i - j >= far_band, or, with far_dist, when
    the smallest distance between the bounding boxes of the two tiles' locations
    (nb consecutive locations each, the last tile possibly short) is at least
    far_dist.  Returns a p x p boolean array (upper triangle False)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = len(x)
    p = -(-n // nb)
    far = np.zeros((p, p), dtype=bool)
    box = []
    for i in range(p):
        sl = slice(i * nb, min(n, (i + 1) * nb))
        box.append((x[sl].min(), x[sl].max(), y[sl].min(), y[sl].max()))
    for j in range(p):
        for i in range(j + 1, p):
            if far_band is not None and i - j >= far_band:
                far[i, j] = True
            if far_dist is not None:
                gx = max(0.0, box[j][0] - box[i][1], box[i][0] - box[j][1])
                gy = max(0.0, box[j][2] - box[i][3], box[i][2] - box[j][3])
                if math.hypot(gx, gy) >= far_dist:
                    far[i, j] = True
    return far


def far_product(Ai, Aj, products=3):
    """The far tier's reduced-precision product Ai Aj' (Section IX extension).

    Each row of a panel tile is scaled by a power of two, 2^-e with e the
    smallest integer such that max|v| 2^-e < 1/2 (the row maximum taken after
    rounding |v| to float32), and cut into an 8-bit integer t0 = rint(t) and a
    12-bit integer t1 = rint(2^12 (t - t0)), t = v 2^(8-e) (round half to
    even).  The product keeps the terms of weight 1 and 2^-12:
        products = 3:  2^(e_r + e_c - 16) [a0 b0' + 2^-12 (a0 b1' + a1 b0')]
        products = 1:  2^(e_r + e_c - 16) a0 b0'
    (every term an exact integer sum, formed here in float64)."""
    def slices(X):
        X = np.asarray(X)
        m = np.max(np.abs(X.astype(np.float32)), axis=1).astype(np.float64)
        e = np.where(m > 0, np.frexp(m)[1] + 1, 0).astype(np.int64)
        t = np.ldexp(np.asarray(X, dtype=np.float64), (8 - e)[:, None])
        s0 = np.rint(t)
        s1 = np.rint((t - s0) * 4096.0)
        return s0, s1, e
    a0, a1, ea = slices(Ai)
    b0, b1, eb = slices(Aj)
    acc = a0 @ b0.T
    if products == 3:
        acc = acc + (a0 @ b1.T + a1 @ b0.T) / 4096.0
    return acc * np.ldexp(1.0, (ea[:, None] + eb[None, :] - 16))


def mp_tile_cholesky(A, nb, band, trace=None, far=None, far_products=3):
    """Algorithm 1 (mixed-precision tile Cholesky, lower case) on a dense SPD A.

    Readings of the printed algorithm: the undefined `m` in the two precision
    tests stands for the row index of the tile being written ((i,k) for the
    triangular solve, (i,j) for the update), the loop bound `r` is p, and
    diag_thick = `band` >= 1.  A is padded to p*nb with an identity block
    (decoupled rows change neither log|A| nor the solve).  Single-precision
    tiles keep only their float32 copy: after a strsm the double copy is the
    exact promotion of the float32 result (sconv2d), so no information lives
    in it beyond the float32 value.

    Returns (L, info): L dense float64 (n x n, lower) with single-precision
    tiles promoted exactly; info = 1-based global row of the first failing
    pivot, 0 on success.  `trace`, if a list, receives (op, i, j, k) tuples
    in execution order, op in {dpotrf, dtrsm, strsm, dsyrk, dconv2s, dgemm, sgemm}.

    far (optional p x p boolean, far_tile_mask): the three-precision extension
    -- an off-band target tile marked far is still stored in FP32 and solved
    by strsm, but its updates use far_product (products = far_products)
    instead of the FP32 sgemm; the rounded result is stored in FP32 as usual.
    """
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    p = -(-n // nb)
    npad = p * nb
    Ap = np.eye(npad, dtype=np.float64)
    Ap[:n, :n] = A
    T = {}
    # lines 2-6: off-band tiles go to single precision (dlag2s)
    for j in range(p):
        for i in range(j, p):
            blk = Ap[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb]
            T[(i, j)] = blk.copy() if tile_is_dp(i, j, band) else blk.astype(np.float32)
    S = {}  # single-precision copies of in-band panel tiles (line 21, dconv2s)

    def rec(*t):
        if trace is not None:
            trace.append(t)

    for k in range(p):
        # line 8: dpotrf
        c, info = sla.lapack.dpotrf(T[(k, k)], lower=1, clean=1)
        rec("dpotrf", k, k, k)
        if info != 0:
            return None, k * nb + int(info)
        Lkk = np.tril(c)
        T[(k, k)] = Lkk
        tmp = Lkk.astype(np.float32)  # line 9: tmp_0k <- dlag2s(A_kk)
        # lines 10-17: triangular solves of column k
        for i in range(k + 1, p):
            if tile_is_dp(i, k, band):
                T[(i, k)] = sla.solve_triangular(Lkk, T[(i, k)].T, lower=True).T
                rec("dtrsm", i, k, k)
            else:
                T[(i, k)] = sla.solve_triangular(tmp, T[(i, k)].T, lower=True).T.astype(np.float32)
                rec("strsm", i, k, k)
        # lines 18-31: updates of the trailing matrix
        for j in range(k + 1, p):
            Ajk = T[(j, k)].astype(np.float64)
            T[(j, j)] = T[(j, j)] - Ajk @ Ajk.T
            rec("dsyrk", j, j, k)
            if tile_is_dp(j, k, band):
                S[(j, k)] = T[(j, k)].astype(np.float32)
                rec("dconv2s", j, k, k)
            for i in range(j + 1, p):
                if tile_is_dp(i, j, band):
                    Aik = T[(i, k)].astype(np.float64)
                    T[(i, j)] = T[(i, j)] - Aik @ Ajk.T
                    rec("dgemm", i, j, k)
                elif far is not None and far[i, j]:
                    # far tier: the reduced product of the operands' own values
                    # (an in-band A_jk is read in its FP64 value, as the slices are)
                    T[(i, j)] = (T[(i, j)].astype(np.float64) -
                                 far_product(T[(i, k)], T[(j, k)], far_products)).astype(np.float32)
                    rec("far", i, j, k)
                else:
                    Aik_s = T[(i, k)]  # off-band whenever (i, j) is off-band
                    Ajk_s = S[(j, k)] if tile_is_dp(j, k, band) else T[(j, k)]
                    T[(i, j)] = (T[(i, j)] - np.matmul(Aik_s, Ajk_s.T)).astype(np.float32)
                    rec("sgemm", i, j, k)
    L = np.zeros((npad, npad), dtype=np.float64)
    for (i, j), blk in T.items():
        L[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb] = blk.astype(np.float64)
    return L[:n, :n], 0


def loglik_mp(x, y, z, theta: Theta, nb, band, far=None, far_products=3):
    """Eq. 2 with the covariance factored by Algorithm 1 (float64 log-det and
    solve); far / far_products: the far tier of mp_tile_cholesky."""
    n = len(z)
    S = covariance(x, y, theta=theta)
    L, info = mp_tile_cholesky(S, nb, band, far=far, far_products=far_products)
    if info != 0:
        return dict(loglik=float("nan"), logdet=float("nan"), quad=float("nan"), info=info)
    logdet, quad = factor_logdet_quad(L, z)
    return dict(loglik=_assemble(n, logdet, quad), logdet=logdet, quad=quad, info=0)


# -------------------------------------------- DST / IND (Section V-B) ---
def dst_covariance(S, nb, d):
    """Diagonal Super-Tile approximation (Section V-B): the covariance with
    every tile (i, j) whose tile distance |i - j| is d or more set to zero
    (tiles of nb rows and columns, the last one possibly short).  d = 1 keeps
    the diagonal tiles only: the independent-blocks (IND) method."""
    n = S.shape[0]
    blk = np.arange(n) // nb
    far = np.abs(blk[:, None] - blk[None, :]) >= d
    A = np.array(S, dtype=np.float64, copy=True)
    A[far] = 0.0
    return A


def loglik_dst(x, y, z, theta: Theta, nb, d):
    """Eq. 2 for the DST covariance, which the method keeps in full (double)
    precision: dense float64 Cholesky of the zeroed matrix."""
    n = len(z)
    S = dst_covariance(covariance(x, y, theta=theta), nb, d)
    L, info = dense_factor(S)
    if info != 0:
        return dict(loglik=float("nan"), logdet=float("nan"), quad=float("nan"), info=info)
    logdet, quad = factor_logdet_quad(L, z)
    return dict(loglik=_assemble(n, logdet, quad), logdet=logdet, quad=quad, info=0)


# --------------------------------------------------------------- kriging ---
def krige(xo, yo, z, theta: Theta, xn, yn):
    """Simple (zero-mean) kriging predictor Z_new = Sigma_new,obs Sigma_obs^-1 Z.

    The paper predicts missing values with the fitted model and scores them by
    the prediction mean square error without printing the predictor; this is
    the reading used.  Sigma_obs^-1 Z is formed by the two triangular solves
    with the float64 factor.
    """
    S = covariance(xo, yo, theta=theta)
    L, info = dense_factor(S)
    if info != 0:
        raise np.linalg.LinAlgError(f"covariance not positive definite (info={info})")
    yv = sla.solve_triangular(L, np.asarray(z, dtype=np.float64), lower=True)
    alpha = sla.solve_triangular(L.T, yv, lower=False)
    C = covariance(xn, yn, xo, yo, theta=theta)
    return C @ alpha


def krige_dst(xo, yo, z, theta: Theta, xn, yn, nb, d):
    """Simple kriging under the DST approximation (Section V-B), read so that
    the new locations are treated like the observed ones: the covariance
    between a new location s and an observed one is C(||s - s_a||) when the
    tile of s -- the tile of its nearest observed location (the lowest index
    on a tie) -- is within d tiles of a's tile, else 0, exactly as
    dst_covariance truncates the observed covariance.  Z_new = C_dst
    Sigma_dst^-1 Z with the float64 factor of the truncated matrix.  A new
    location that coincides with an observed one (no nugget) gets its
    observation back, for every d."""
    xo = np.asarray(xo, dtype=np.float64)
    yo = np.asarray(yo, dtype=np.float64)
    S = dst_covariance(covariance(xo, yo, theta=theta), nb, d)
    L, info = dense_factor(S)
    if info != 0:
        raise np.linalg.LinAlgError(f"truncated covariance not positive definite (info={info})")
    yv = sla.solve_triangular(L, np.asarray(z, dtype=np.float64), lower=True)
    alpha = sla.solve_triangular(L.T, yv, lower=False)
    xn = np.asarray(xn, dtype=np.float64)
    yn = np.asarray(yn, dtype=np.float64)
    C = covariance(xn, yn, xo, yo, theta=theta)
    r2 = (xn[:, None] - xo[None, :]) ** 2 + (yn[:, None] - yo[None, :]) ** 2
    home = np.argmin(r2, axis=1) // nb              # argmin takes the lowest index on a tie
    blk = np.arange(len(xo)) // nb
    C[np.abs(home[:, None] - blk[None, :]) >= d] = 0.0
    return C @ alpha


# ------------------------------------------------------- profile (Eq. 3) ---
def profile_sigma2(x, y, z, beta, nu, nugget_ratio=0.0):
    """theta1_opt = Z' S~^-1 Z / n with S~ the covariance at unit variance
    (Eq. 3 and the expression for theta1 following it).  Returns
    (theta1_opt, profile loglik) where the profile loglik is Eq. 2 at theta1_opt,
    i.e. -n/2 log 2pi - n/2 - n/2 log(Q/n) - 1/2 log|S~| (reading of the garbled
    Eq. 3: its quadratic term at the optimum equals n)."""
    n = len(z)
    th = Theta(1.0, beta, nu, nugget_ratio)
    S = covariance(x, y, theta=th)
    L, info = dense_factor(S)
    logdet, quad = factor_logdet_quad(L, z)
    s2 = quad / n
    prof = -0.5 * n * LOG_2PI - 0.5 * n - 0.5 * n * math.log(s2) - 0.5 * logdet
    return s2, prof


# ------------------------------------------------------- MLE (Section IV-C) ---
# The estimator theta-hat maximises Eq. 2.  The paper drives it with NLopt at an
# optimisation tolerance of 1e-3 without naming the method; the reading here is
# the Nelder-Mead simplex (Nelder & Mead, 1965) over log-parameters with the
# classic coefficients (reflection 1, expansion 2, contraction 1/2, shrink 1/2),
# box bounds by clamping, a fixed budget of objective evaluations and a
# simplex-size stopping rule at the tolerance.
NM_LO = (1e-3, 1e-4, 0.05)   # sigma2, beta, nu
NM_HI = (1e2, 2.0, 3.0)


def nelder_mead(f, u0, step=0.1, max_evals=60, xtol=1e-3, lo=None, hi=None):
    """Minimise f over R^d from u0.

    Simplex u0, u0 + step e_i.  Each iteration orders the vertices by f (ties:
    the earlier position first), stops when every vertex is within xtol (max
    norm) of the best, and replaces the worst by the reflection, expansion,
    outside or inside contraction, or shrinks towards the best.  Trial points
    are clamped to [lo, hi] before evaluation.  An evaluation is made only while
    fewer than max_evals have been made; the best point evaluated is returned as
    (u, f(u), evaluations, iterations).
    """
    d = len(u0)
    lo = np.full(d, -np.inf) if lo is None else np.asarray(lo, dtype=np.float64)
    hi = np.full(d, np.inf) if hi is None else np.asarray(hi, dtype=np.float64)
    state = {"evals": 0, "best_u": None, "best_f": math.inf}

    def clamp(u):
        return np.minimum(np.maximum(np.asarray(u, dtype=np.float64), lo), hi)

    def ev(u):
        if state["evals"] >= max_evals:
            return None
        state["evals"] += 1
        v = f(u)
        v = v if (v is not None and math.isfinite(v)) else math.inf
        if v < state["best_f"]:
            state["best_f"], state["best_u"] = v, u.copy()
        return v

    verts, fv = [], []
    for i in range(d + 1):
        u = np.array(u0, dtype=np.float64)
        if i > 0:
            u[i - 1] += step
        u = clamp(u)
        v = ev(u)
        if v is None:
            break
        verts.append(u)
        fv.append(v)
    iters = 0   # completed iterations
    while len(verts) == d + 1:
        order = sorted(range(d + 1), key=lambda q: (fv[q], q))
        verts = [verts[q] for q in order]
        fv = [fv[q] for q in order]
        if max(np.max(np.abs(verts[q] - verts[0])) for q in range(1, d + 1)) <= xtol:
            break
        c = np.mean(verts[:d], axis=0)
        worst = verts[d]
        r = clamp(c + (c - worst))
        fr = ev(r)
        if fr is None:
            break
        if fr < fv[0]:
            e = clamp(c + 2.0 * (c - worst))
            fe = ev(e)
            if fe is None:
                break
            verts[d], fv[d] = (e, fe) if fe < fr else (r, fr)
            iters += 1
            continue
        if fr < fv[d - 1]:
            verts[d], fv[d] = r, fr
            iters += 1
            continue
        if fr < fv[d]:
            oc = clamp(c + 0.5 * (r - c))
            fo = ev(oc)
            if fo is None:
                break
            if fo <= fr:
                verts[d], fv[d] = oc, fo
                iters += 1
                continue
        else:
            ic = clamp(c + 0.5 * (worst - c))
            fi = ev(ic)
            if fi is None:
                break
            if fi < fv[d]:
                verts[d], fv[d] = ic, fi
                iters += 1
                continue
        for q in range(1, d + 1):          # shrink towards the best vertex
            verts[q] = clamp(verts[0] + 0.5 * (verts[q] - verts[0]))
            v = ev(verts[q])
            if v is None:
                verts = verts[:q]          # out of budget mid-shrink
                break
            fv[q] = v
        else:
            iters += 1
    return state["best_u"], state["best_f"], state["evals"], iters


def profile_loglik(n, logdet, quad):
    """Eq. 3 at theta1 = quad / n (reading R9): -n/2 log 2pi - n/2 - n/2 log(quad/n) - 1/2 logdet."""
    return -0.5 * n * LOG_2PI - 0.5 * n - 0.5 * n * math.log(quad / n) - 0.5 * logdet


def mle(x, y, z, theta0: Theta, max_evals=60, xtol=1e-3, profile=False, fix_nu=False, evaluate=None):
    """theta-hat maximising Eq. 2 (profile=False: over log sigma2, log beta,
    log nu) or Eq. 3 (profile=True: over log beta, log nu, with theta1 = Q/n and
    the nugget taken relative to theta1).  fix_nu keeps nu at theta0.nu.
    evaluate(theta) -> (logdet, quad) of Sigma(theta), or None when it is not
    positive definite (default: the dense FP64 definition).  Returns
    dict(theta, loglik, evals, iterations)."""
    n = len(z)
    if evaluate is None:
        def evaluate(th):
            L, info = dense_factor(covariance(x, y, theta=th))
            return None if info != 0 else factor_logdet_quad(L, z)
    names = ([] if profile else [0]) + [1] + ([] if fix_nu else [2])
    base = [theta0.sigma2, theta0.beta, theta0.nu]
    lo = [math.log(NM_LO[q]) for q in names]
    hi = [math.log(NM_HI[q]) for q in names]

    def unpack(u):
        t = list(base)
        for q, v in zip(names, u):
            t[q] = math.exp(v)
        return t

    def objective(u):
        t = unpack(u)
        r = evaluate(Theta(1.0 if profile else t[0], t[1], t[2], theta0.nugget))
        if r is None:
            return math.inf
        logdet, quad = r
        return -(profile_loglik(n, logdet, quad) if profile else _assemble(n, logdet, quad))

    u0 = [math.log(base[q]) for q in names]
    ub, fb, evals, iters = nelder_mead(objective, u0, max_evals=max_evals, xtol=xtol, lo=lo, hi=hi)
    t = unpack(ub)
    if profile:
        logdet, quad = evaluate(Theta(1.0, t[1], t[2], theta0.nugget))
        t[0] = quad / n
    return dict(theta=Theta(t[0], t[1], t[2], theta0.nugget), loglik=-fb, evals=evals, iterations=iters)
