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
