"""Electron and magnetisation densities at the Gauss points, plain FP64 (oracle).

Test infrastructure only (see ``oracle/__init__``).

Sec. II (Eqs. rho, mag): with occupations f_n,
    rho(r) = sum_n f_n psi_n(r)^H psi_n(r),
    m(r)   = sum_n f_n psi_n(r)^H sigma psi_n(r),  sigma = (sigma_x, sigma_y, sigma_z),
and psi_n(r) = sum_I N_I(r) X[I, :, n] (Eq. FEWfns), evaluated at the Gauss points r_q of
every cell (the points at which the paper's Eqs. disvxc / disbxc want V_xc and B_xc).
Written out component by component:
    rho = |u|^2 + |d|^2,  m_x = 2 Re(u* d),  m_y = 2 Im(u* d),  m_z = |u|^2 - |d|^2
for psi = (u, d) (spin up, spin down).

Occupations (Sec. II: f_nk with the electron count fixed by the Lagrange multiplier mu;
Sec. V: Fermi-Dirac smearing): f_nk = 1 / (1 + exp((eps_nk - mu) / kT)), one electron per
spinor state, mu the root of sum_k w_k sum_n f_nk = N_e (w_k the Brillouin-zone weights).
"""
from __future__ import annotations

import numpy as np


def spinor_at_gauss(d, X, cells=None):
    """psi[e, q, s, n] = sum_i N_i(r_q) X[I(e, i), s, n], zero for constrained nodes
    (all cells, or the listed ones in that order)."""
    mesh, tab = d.mesh, d.tab
    M, _, nv = X.shape
    cn = mesh.cell_nodes if cells is None else mesh.cell_nodes[np.asarray(cells)]
    sel = np.where(cn >= 0, cn, M)                                 # [E, np^3]
    vals = np.asarray(X)[np.minimum(sel, M - 1)].astype(np.complex128)
    vals[sel == M] = 0.0
    # psi[e, q, s, n] = sum_i N3[i, q] X[sel[e, i], s, n]
    return np.einsum("iq,eisn->eqsn", tab.N3, vals)


def densities(d, X, occ, cells=None):
    """rho[e, q] and m[3, e, q] (Eqs. rho, mag) for the block X[M][2][nv] with
    occupations occ[nv] (all cells, or the listed ones)."""
    occ = np.asarray(occ, np.float64)
    psi = spinor_at_gauss(d, X, cells)
    u, dn = psi[:, :, 0, :], psi[:, :, 1, :]
    uu = (u.conj() * u).real
    dd = (dn.conj() * dn).real
    ud = u.conj() * dn
    rho = (uu + dd) @ occ
    m = np.stack([(2.0 * ud.real) @ occ, (2.0 * ud.imag) @ occ, (uu - dd) @ occ])
    return rho, m


def fermi(x):
    """1 / (1 + e^x), evaluated without overflow."""
    x = np.asarray(x, np.float64)
    out = np.empty_like(x)
    pos = x > 0
    ep = np.exp(-x[pos])
    out[pos] = ep / (1.0 + ep)
    out[~pos] = 1.0 / (1.0 + np.exp(x[~pos]))
    return out


def fermi_occupations(eps, kweights, nelec, kT):
    """f[k, n] and mu with sum_k w_k sum_n f[k, n] = nelec (root by Brent's method)."""
    from scipy.optimize import brentq
    eps = np.atleast_2d(np.asarray(eps, np.float64))
    w = np.asarray(kweights, np.float64)

    def excess(mu):
        return float((w[:, None] * fermi((eps - mu) / kT)).sum()) - nelec

    lo, hi = eps.min() - 60.0 * kT, eps.max() + 60.0 * kT
    for _ in range(100):                     # N(mu) increases with mu: widen the bracket
        if excess(lo) <= 0 <= excess(hi):
            break
        lo, hi = lo - 60.0 * kT, hi + 60.0 * kT
    else:
        raise ValueError("no chemical potential brackets the electron count")
    mu = brentq(excess, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    return fermi((eps - mu) / kT), mu
