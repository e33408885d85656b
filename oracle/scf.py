"""Self-consistent-field pieces around the eigensolver, plain FP64 (oracle).

Test infrastructure only (see ``oracle/__init__``).

* Exchange-correlation stand-in: the paper uses PBE with the White-Bird treatment (Sec. III,
  Eqs. disvxc / disbxc); the closed-form stand-in here is exchange-only local spin density
  (Dirac-Slater) for a noncollinear density.  With rho_up/dn = (rho +- |m|) / 2,
      e(rho, m) = -(3/4) (6/pi)^(1/3) (rho_up^(4/3) + rho_dn^(4/3))      (energy per volume),
      V_xc = de/drho = (v_up + v_dn) / 2,   B_xc = de/dm = (v_up - v_dn) / 2 * m/|m|,
      v_s = -(6/pi)^(1/3) rho_s^(1/3),
  the point-wise form of Eqs. disvxc / disbxc for a functional without gradients (the
  1/(w_q J) there cancels the quadrature weight of E_xc = sum_q w_q J e).  m = 0 reduces to
  Dirac exchange -(3/4)(3/pi)^(1/3) rho^(4/3).
* Inner product of density pairs (Eq. innerPdt): <(r1, m1), (r2, m2)> = (1/2)(int r1 r2 +
  int m1.m2), by the Gauss quadrature of the mesh.
* Anderson mixing (Sec. III.B.1): next input = sum_j b_j (x_j + alpha r_j), sum_j b_j = 1,
  b minimising || sum_j b_j r_j || in that inner product: b = G^-1 1 / (1^T G^-1 1) with
  G_jk = <r_j, r_k>.
"""
from __future__ import annotations

import numpy as np

CX = (6.0 / np.pi) ** (1.0 / 3.0)


def lsda_exchange(rho, m):
    """Energy density e, V_xc and B_xc [3, ...] at each point from rho [...] and m [3, ...]."""
    rho = np.asarray(rho, np.float64)
    m = np.asarray(m, np.float64)
    am = np.sqrt((m * m).sum(0))
    up = np.maximum(0.5 * (rho + am), 0.0)
    dn = np.maximum(0.5 * (rho - am), 0.0)
    e = -0.75 * CX * (up ** (4.0 / 3.0) + dn ** (4.0 / 3.0))
    vu, vd = -CX * np.cbrt(up), -CX * np.cbrt(dn)
    V = 0.5 * (vu + vd)
    with np.errstate(invalid="ignore", divide="ignore"):
        mhat = np.where(am > 0, m / np.where(am > 0, am, 1.0), 0.0)
    B = 0.5 * (vu - vd) * mhat
    return e, V, B


def inner(W, x1, x2):
    """<x1, x2> of density pairs stored as [E, 4, q] (rho, m_x, m_y, m_z) with the
    quadrature weights W [q] * J already in W ([q] or [E, q])."""
    W = np.asarray(W, np.float64)
    Wq = W[:, None, :] if W.ndim == 2 else W[None, None, :]
    return 0.5 * float((Wq * x1 * x2).sum())


def anderson(W, xs, rs, alpha):
    """Next input from the histories xs[j], rs[j] (arrays [E, 4, q]); returns (x_next, b)."""
    n = len(xs)
    G = np.array([[inner(W, rs[j], rs[k]) for k in range(n)] for j in range(n)])
    y = np.linalg.solve(G, np.ones(n))
    b = y / y.sum()
    x = sum(b[j] * (xs[j] + alpha * rs[j]) for j in range(n))
    return x, b


def _pack(rho, m):
    return np.concatenate([rho[:, None], np.moveaxis(m, 0, 1)], 1)      # [E, 4, q]


def scf_loop(prob, X0, v0, nelec, kT, degree, lanczos_steps, alpha, nhist, iters, eig="chfsi"):
    """The SCF iteration of Sec. III.B.1 on one k-point (see ``scf_loop_k``)."""
    res, x, ritz = scf_loop_k([prob], [X0], [v0], [1.0], nelec, kT, degree, lanczos_steps, alpha,
                              nhist, iters, eig)
    return res, x, ritz[0]


def scf_loop_k(probs, X0s, v0s, kweights, nelec, kT, degree, lanczos_steps, alpha, nhist, iters,
               eig="chfsi"):
    """The SCF iteration of Sec. III.B.1 over k-points with the exchange stand-in.

    probs[k] differ only in the k-point; their veff is the external potential and their
    bx/by/bz must be zero: the first block of each k-point comes from CholGS + Rayleigh-Ritz
    of X0s[k] under H[V_ext] (the cycle 0 of the eigensolver).  Each step builds V_eff =
    V_ext + V_xc and B_xc from the input densities (the same fields at every k-point), runs
    one ChFSI cycle per k-point on its carried-over block (Lanczos bounds from v0s[k], the
    sigma-scaled filter normalised at min(lambda_min, lowest Ritz value), CholGS,
    Rayleigh-Ritz; ``eig='dense'`` takes the exact lowest eigenpairs instead), forms
    Fermi-Dirac occupations with one chemical potential over all k-points, sums the output
    densities over k with the Brillouin-zone weights, and mixes.  Returns (residual norms
    ||F(x) - x||, final input densities, final Ritz values [nk, nv])."""
    from . import chfsi as oc
    from . import density as od
    from . import fe
    nk = len(probs)
    w = np.asarray(kweights, np.float64)
    vext = np.asarray(probs[0].veff, np.float64)
    ds = [fe.Discretisation(pr) for pr in probs]
    md = ds[0].md
    nv = X0s[0].shape[2]
    Xs, ritz = [], []
    for d, X0 in zip(ds, X0s):
        r, X, _ = oc.rayleigh_ritz(d.apply_h, oc.cholgs(X0, md))
        Xs.append(X)
        ritz.append(r)

    def densities(ds, ritz):
        f, _ = od.fermi_occupations(np.array(ritz), w, nelec, kT)
        return sum(w[k] * _pack(*od.densities(ds[k], Xs[k], f[k])) for k in range(nk))

    x_in = densities(ds, ritz)
    W = ds[0].tab.W
    xs, fs, res = [], [], []
    for _ in range(iters):
        _, V, B = lsda_exchange(x_in[:, 0], np.moveaxis(x_in[:, 1:], 1, 0))
        ds = [fe.Discretisation(pr.with_(veff=vext + V, bx=B[0], by=B[1], bz=B[2]))
              for pr in probs]
        for k, d in enumerate(ds):
            if eig == "chfsi":
                def apply_ht(Z, d=d):
                    return d.apply_h(Z) / md[:, None, None]
                lo, hi = oc.lanczos_bounds(apply_ht, md, v0s[k], lanczos_steps)
                X = oc.cheb_filter(apply_ht, Xs[k], degree, float(ritz[k][-1]), hi,
                                   min(lo, float(ritz[k][0])))
                ritz[k], Xs[k], _ = oc.rayleigh_ritz(d.apply_h, oc.cholgs(X, md))
            else:                                # exact eigenpairs of M_D^-1/2 H M_D^-1/2
                dm = np.repeat(1.0 / np.sqrt(md), 2)
                H = d.dense_h()
                ev, Q = np.linalg.eigh(dm[:, None] * (0.5 * (H + H.conj().T)) * dm[None, :])
                ritz[k] = ev[:nv]
                Xs[k] = (dm[:, None] * Q[:, :nv]).reshape(-1, 2, nv)
        x_out = densities(ds, ritz)
        xs, fs = (xs + [x_in])[-nhist:], (fs + [x_out])[-nhist:]
        res.append(np.sqrt(inner(W, x_out - x_in, x_out - x_in)))
        x_in, _ = anderson(W, xs, [b - a for a, b in zip(xs, fs)], alpha)
    return np.array(res), x_in, np.array(ritz)
