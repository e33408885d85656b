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
"""
from __future__ import annotations

import numpy as np


def spinor_at_gauss(d, X):
    """psi[e, q, s, n] = sum_i N_i(r_q) X[I(e, i), s, n], zero for constrained nodes."""
    mesh, tab = d.mesh, d.tab
    M, _, nv = X.shape
    Xp = np.concatenate([np.asarray(X, np.complex128), np.zeros((1, 2, nv), np.complex128)])
    sel = np.where(mesh.cell_nodes >= 0, mesh.cell_nodes, M)      # [E, np^3]
    # psi[e, q, s, n] = sum_i N3[i, q] Xp[sel[e, i], s, n]
    return np.einsum("iq,eisn->eqsn", tab.N3, Xp[sel])


def densities(d, X, occ):
    """rho[e, q] and m[3, e, q] (Eqs. rho, mag) for the block X[M][2][nv] with
    occupations occ[nv]."""
    occ = np.asarray(occ, np.float64)
    psi = spinor_at_gauss(d, X)
    u, dn = psi[:, :, 0, :], psi[:, :, 1, :]
    uu = (u.conj() * u).real
    dd = (dn.conj() * dn).real
    ud = u.conj() * dn
    rho = (uu + dd) @ occ
    m = np.stack([(2.0 * ud.real) @ occ, (2.0 * ud.imag) @ occ, (uu - dd) @ occ])
    return rho, m
