"""Chebyshev-filtered subspace iteration on (H, M_D), plain FP64 (oracle).

Test infrastructure only (see ``oracle/__init__``).

Follows Sec. III.B.2 of the paper (subspace iteration for the linear
eigenproblem):
  * Eq. chebfilt -- three-term Chebyshev recurrence on H~ = M_D^-1 H with the
    unwanted interval [lambda_T, lambda_max] mapped to [-1, 1]; the "scaled"
    polynomial is read as the sigma-scaled recurrence normalised at lambda_min.
  * generalised Lanczos estimate of lambda_min / lambda_max.
  * Rayleigh-Ritz: X^H H X Q = X^H M X Q Lambda, U = X Q; here preceded by a
    Cholesky-Gram-Schmidt orthonormalisation in the M_D inner product so the
    projected problem is a standard Hermitian one.
  * the residual-based reformulation of the filter (X_k = X T_k(Lambda^) + Z_k).
"""
from __future__ import annotations

import math

import numpy as np


# ----------------------------------------------------------------------------
# scalar Chebyshev helpers
# ----------------------------------------------------------------------------
def cheb_T(m: int, x):
    """T_m(x) in closed form: cos(m arccos x) on [-1, 1], cosh(m arccosh|x|) sign(x)^m outside."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1.0
    out[inside] = np.cos(m * np.arccos(x[inside]))
    xo = x[~inside]
    out[~inside] = np.cosh(m * np.arccosh(np.abs(xo))) * np.sign(xo) ** m
    return out


def filter_scalar(m: int, lam, lT: float, lmax: float, lmin: float):
    """rho_m(lam) = T_m((lam - c)/e) / T_m((lmin - c)/e), c, e from [lT, lmax]."""
    c = 0.5 * (lmax + lT)
    e = 0.5 * (lmax - lT)
    return cheb_T(m, (np.asarray(lam) - c) / e) / cheb_T(m, np.array((lmin - c) / e))


def sigma_sequence(m: int, lT: float, lmax: float, lmin: float):
    """sigma_1 = e/(lmin - c), sigma_{k+1} = 1/(2/sigma_1 - sigma_k), k = 1..m-1."""
    c = 0.5 * (lmax + lT)
    e = 0.5 * (lmax - lT)
    s = [e / (lmin - c)]
    for _ in range(m - 1):
        s.append(1.0 / (2.0 / s[0] - s[-1]))
    return c, e, s


# ----------------------------------------------------------------------------
# the filter
# ----------------------------------------------------------------------------
def cheb_filter(apply_htilde, X, m: int, lT: float, lmax: float, lmin: float):
    """sigma-scaled Chebyshev filter of degree m (Eq. chebfilt):

      X_1     = (sigma_1/e) (H~ - c) X_0
      X_{k+1} = (2 sigma_{k+1}/e) (H~ - c) X_k - sigma_k sigma_{k+1} X_{k-1}

    which equals T_m((H~ - c)/e) X_0 / T_m((lmin - c)/e).
    """
    c, e, s = sigma_sequence(m, lT, lmax, lmin)
    Xprev = X
    Xcur = (s[0] / e) * (apply_htilde(X) - c * X)
    for k in range(1, m):
        Xnext = (2.0 * s[k] / e) * (apply_htilde(Xcur) - c * Xcur) - s[k - 1] * s[k] * Xprev
        Xprev, Xcur = Xcur, Xnext
    return Xcur


def cheb_filter_split(apply_htilde, X, ritz, m: int, lT: float, lmax: float, lmin: float,
                      HtX=None):
    """Residual form of the same filter for a block of Ritz pairs (X, Lambda):

    with H^ = (H~ - c)/e, Lambda^ = (Lambda - c)/e, R = H^ X - X Lambda^ and
    D_k = T_k(Lambda^)/T_k(tau) (tau = (lmin - c)/e),
      Z_1 = sigma_1 R,
      Z_{k+1} = 2 sigma_{k+1} H^ Z_k - sigma_k sigma_{k+1} Z_{k-1} + 2 sigma_{k+1} R D_k,
      X_m = X D_m + Z_m.
    Exactly equal to ``cheb_filter`` (the operator only ever acts on Z).
    """
    c, e, s = sigma_sequence(m, lT, lmax, lmin)
    lam_hat = (np.asarray(ritz, np.float64) - c) / e
    if HtX is None:
        HtX = apply_htilde(X)
    R = (HtX - c * X) / e - X * lam_hat[None, None, :]
    # scalar recurrence for D_k (same sigma scaling)
    Dprev = np.ones_like(lam_hat)
    Dcur = s[0] * lam_hat
    Zprev = np.zeros_like(X)
    Zcur = s[0] * R
    for k in range(1, m):
        HZ = (apply_htilde(Zcur) - c * Zcur) / e
        Znext = 2 * s[k] * HZ - s[k - 1] * s[k] * Zprev + 2 * s[k] * R * Dcur[None, None, :]
        Dnext = 2 * s[k] * lam_hat * Dcur - s[k - 1] * s[k] * Dprev
        Zprev, Zcur = Zcur, Znext
        Dprev, Dcur = Dcur, Dnext
    return X * Dcur[None, None, :] + Zcur


# ----------------------------------------------------------------------------
# inner products in the M_D metric
# ----------------------------------------------------------------------------
def gram(X, md, Y=None):
    """S = X^H M_D Y for blocks X[M][2][n] (both spins weighted by M_D[I])."""
    if Y is None:
        Y = X
    M = X.shape[0]
    Xw = X * md[:, None, None]
    return Xw.reshape(2 * M, -1).conj().T @ Y.reshape(2 * M, -1)


# ----------------------------------------------------------------------------
# dense helpers written out (own Jacobi eigensolver, own Cholesky)
# ----------------------------------------------------------------------------
def cholesky(S):
    """Lower-triangular L with S = L L^H (plain column-by-column algorithm).
    Raises ValueError if S is not positive definite."""
    n = S.shape[0]
    L = np.zeros_like(S, dtype=np.complex128)
    for j in range(n):
        d = S[j, j].real - np.sum(np.abs(L[j, :j]) ** 2)
        if not d > 0:
            raise ValueError("matrix not positive definite")
        L[j, j] = math.sqrt(d)
        L[j + 1:, j] = (S[j + 1:, j] - L[j + 1:, :j] @ L[j, :j].conj()) / L[j, j]
    return L


def jacobi_eigh(A, tol=1e-15, max_sweeps=60):
    """Cyclic Jacobi for a complex Hermitian matrix.

    Each (p, q) rotation: a unitary diag(1, e^{-i phi}) turns a_pq into
    |a_pq|, then a real Jacobi rotation (t = sgn(tau)/(|tau| + sqrt(1+tau^2)),
    tau = (a_qq - a_pp)/(2|a_pq|)) annihilates it.  Returns ascending
    eigenvalues and the unitary whose columns are the eigenvectors.
    """
    A = np.array(A, dtype=np.complex128)
    n = A.shape[0]
    V = np.eye(n, dtype=np.complex128)
    scale = np.linalg.norm(A)
    for _ in range(max_sweeps):
        off = np.linalg.norm(A - np.diag(np.diag(A)))
        if off <= tol * max(scale, 1e-300):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                mag = abs(apq)
                if mag <= 1e-300 or mag <= 1e-18 * scale:
                    continue
                ph = apq / mag
                tau = (A[q, q].real - A[p, p].real) / (2.0 * mag)
                t = (1.0 if tau >= 0 else -1.0) / (abs(tau) + math.sqrt(1.0 + tau * tau))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = t * c
                G = np.array([[c, s], [-s * ph.conjugate(), c * ph.conjugate()]])
                idx = [p, q]
                A[:, idx] = A[:, idx] @ G
                A[idx, :] = G.conj().T @ A[idx, :]
                A[p, q] = 0.0
                A[q, p] = 0.0
                V[:, idx] = V[:, idx] @ G
    w = np.real(np.diag(A)).copy()
    order = np.argsort(w, kind="stable")
    return w[order], V[:, order]


# ----------------------------------------------------------------------------
# block operations of the ChFSI cycle
# ----------------------------------------------------------------------------
def cholgs(X, md):
    """S = X^H M_D X = L L^H, X <- X L^-H (Cholesky-Gram-Schmidt)."""
    S = gram(X, md)
    L = cholesky(S)
    M, _, n = X.shape
    Linvh = np.linalg.inv(L).conj().T
    return (X.reshape(2 * M, n) @ Linvh).reshape(M, 2, n)


def rayleigh_ritz(apply_h, X, md=None, HX=None):
    """Hp = X^H H X (X M_D-orthonormal), Hp Q = Q Lambda, X <- X Q.
    Returns (ritz ascending, X Q, (H X) Q)."""
    if HX is None:
        HX = apply_h(X)
    M, _, n = X.shape
    Hp = X.reshape(2 * M, n).conj().T @ HX.reshape(2 * M, n)
    Hp = 0.5 * (Hp + Hp.conj().T)
    w, Q = jacobi_eigh(Hp)
    Xn = (X.reshape(2 * M, n) @ Q).reshape(M, 2, n)
    HXn = (HX.reshape(2 * M, n) @ Q).reshape(M, 2, n)
    return w, Xn, HXn


def lanczos_bounds(apply_htilde, md, v0, steps: int):
    """Generalised Lanczos on H~ = M_D^-1 H in the M_D inner product with full
    reorthogonalisation.  Returns (lambda_min, lambda_max) with
    lambda_min = smallest Ritz value of T_k and lambda_max = largest + |beta_k|."""
    def ip(a, b):
        return np.sum(md[:, None] * a.conj() * b)

    v = v0 / math.sqrt(ip(v0, v0).real)
    Vs = [v]
    alpha, beta = [], []
    for j in range(steps):
        w = apply_htilde(Vs[-1][:, :, None])[:, :, 0]
        a = ip(Vs[-1], w).real
        alpha.append(a)
        w = w - a * Vs[-1]
        if j > 0:
            w = w - beta[-1] * Vs[-2]
        for _ in range(2):
            for u in Vs:
                w = w - ip(u, w) * u
        b = math.sqrt(ip(w, w).real)
        beta.append(b)
        Vs.append(w / b)
    T = np.diag(alpha) + np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1)
    theta, _ = jacobi_eigh(T)
    return float(theta[0]), float(theta[-1] + abs(beta[-1]))


def chfsi(apply_h, md, X0, cycles: int, degree: int, lmin: float, lmax: float):
    """Cycle 0 = CholGS + RR on X0 (sets lambda_T = max Ritz value); then
    ``cycles`` x (filter -> CholGS -> RR), lambda_T updated after each RR.
    The filter is normalised at min(lmin, lowest Ritz value of the previous RR):
    a few Lanczos steps do not bound the spectrum from below, and the
    normalisation point must lie below the damped interval [lambda_T, lmax].
    Returns (list of Ritz-value arrays, final X)."""
    def apply_ht(Z):
        return apply_h(Z) / md[:, None, None]

    X = cholgs(X0, md)
    ritz, X, _ = rayleigh_ritz(apply_h, X)
    history = [ritz]
    for _ in range(cycles):
        lT = float(ritz[-1])
        X = cheb_filter(apply_ht, X, degree, lT, lmax, min(lmin, float(ritz[0])))
        X = cholgs(X, md)
        ritz, X, _ = rayleigh_ritz(apply_h, X)
        history.append(ritz)
    return history, X


def generalized_eigs(H, md):
    """Dense brute force: eigenvalues of M_D^-1/2 H M_D^-1/2 (own Jacobi)."""
    d = np.repeat(1.0 / np.sqrt(md), 2)
    A = d[:, None] * H * d[None, :]
    return jacobi_eigh(0.5 * (A + A.conj().T))
