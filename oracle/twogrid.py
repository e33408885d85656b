"""Two-grid transfer of a spinor block from FE order p_c to order p_f >= p_c on the same
mesh, plain FP64 (oracle).

Test infrastructure only (see ``oracle/__init__``).

Sec. IV.A (Eq. FEWfnsCMesh): the early SCF iterations use the basis N^{h,p-1} of the same
triangulation, and the later ones N^{h,p}.  The order-p_c space is contained in the order-p_f
space, so a block expressed in the coarse basis is carried to the fine one exactly by nodal
interpolation: X_f[J] = u_c(r_J) = sum_I N^{h,p_c}_I(r_J) X_c[I] at every free fine node r_J.
Written out: for every cell and every fine local GLL node of it, the coarse Lagrange basis of
that cell is evaluated at the node's reference coordinates and contracted with the cell's coarse
nodal values.
"""
from __future__ import annotations

import numpy as np

from . import fe


def transfer_matrix_1d(pc: int, pf: int) -> np.ndarray:
    """T[j, i] = l^{p_c}_i(x^{p_f}_j): coarse Lagrange basis at the fine GLL nodes."""
    xc, _ = fe.gll(pc)
    xf, _ = fe.gll(pf)
    L, _ = fe.lagrange(xc, xf)          # L[i, j] = l_i(xf_j)
    return np.asarray(L).T


def prolongate(dc, df, Xc, cells=None):
    """X_f [M_f][2][nv] from X_c [M_c][2][nv]; dc, df are Discretisations of the same cells.
    With ``cells``, only the fine nodes of those cells are filled (the rest stay zero)."""
    mc, mf = dc.mesh, df.mesh
    if mc.ncell != mf.ncell or mc.periodic != mf.periodic or not np.allclose(mc.h, mf.h):
        raise ValueError("coarse and fine discretisations must share the mesh")
    nc, nf = mc.np1, mf.np1
    T = transfer_matrix_1d(mc.p, mf.p)                       # [nf, nc]
    # 3-D weights W[(jz, jy, jx), (iz, iy, ix)] = T[jx, ix] T[jy, iy] T[jz, iz]
    W = np.einsum("ad,be,cf->cbafed", T, T, T).reshape(nf ** 3, nc ** 3)
    nv = Xc.shape[2]
    Xf = np.zeros((mf.nnodes, 2, nv), np.complex128)
    for e in (range(mc.ncells) if cells is None else cells):
        ic = mc.cell_nodes[e]
        xe = np.asarray(Xc)[np.maximum(ic, 0)].astype(np.complex128)
        xe[ic < 0] = 0.0
        vals = W @ xe.reshape(nc ** 3, -1)
        jf = mf.cell_nodes[e]
        ok = jf >= 0
        Xf[jf[ok]] = vals.reshape(nf ** 3, 2, nv)[ok]
    return Xf
