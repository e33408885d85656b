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
