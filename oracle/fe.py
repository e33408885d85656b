"""FE discretisation of the spinor Kohn-Sham Hamiltonian, plain FP64 (oracle).

Test infrastructure only (see ``oracle/__init__``).

Follows Sec. III.A of the paper:
  * Eq. FEWfns  -- spinor u = sum_I u^I N_I, N_I tensor-product Lagrange
                   polynomials of degree p on GLL nodes (n_p = p + 1 per dir).
  * Eq. GHEP    -- H^k U = M U Lambda, DOF index 2I + alpha.
  * Eq. FEHloc  -- H^loc entries (kinetic, -i N_I k.grad N_J, |k|^2/2 N_I N_J,
                   V_eff N_I N_J, sum_d B^d N_I N_J sigma^d).
  * Eq. FEHnloc -- H^nloc = sum_a (P_a x I2) Delta_a (P_a x I2)^H, with
                   P^{a,k}_{I chi} = int sum_L e^{-ik.(r-L)} p_chi(r-L-R_a) N_I (Eq.
                   CMat with R_a restored and the index order of Eq.
                   HnlocPeriodic).
  * Eq. cellIntegrals -- integrals cell by cell with tensor Gauss-Legendre
                   quadrature, w_q J^(e).
  * Sec. III.B.2 -- M_D, the GLL-lumped (diagonal) mass.

Two independent H.X forms: ``assemble_local`` + ``NonlocalOp`` (explicit
sparse matrix, form O1a) and ``apply_h`` (element-by-element quadrature apply,
form O1b).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

PAULI = np.array([[[0, 1], [1, 0]],
                  [[0, -1j], [1j, 0]],
                  [[1, 0], [0, -1]]], dtype=np.complex128)


# ----------------------------------------------------------------------------
# 1-D tables
# ----------------------------------------------------------------------------
def gll(p: int):
    """GLL nodes and weights on [-1, 1] for degree p (p + 1 points).

    Nodes: +-1 and the roots of P_p'; weights 2 / (p (p+1) P_p(x_i)^2).
    """
    Pp = np.polynomial.legendre.Legendre.basis(p)
    inner = np.sort(np.real(Pp.deriv().roots())) if p > 1 else np.zeros(0)
    x = np.concatenate([[-1.0], inner, [1.0]])
    w = 2.0 / (p * (p + 1) * Pp(x) ** 2)
    return x, w


def gauss(nq: int):
    """Gauss-Legendre points and weights on [-1, 1] (numpy's leggauss)."""
    return np.polynomial.legendre.leggauss(nq)


def lagrange(nodes: np.ndarray, x: np.ndarray):
    """Values L[i, j] = l_i(x_j) and derivatives D[i, j] = l_i'(x_j).

    l_i(x) = prod_{m != i} (x - x_m) / (x_i - x_m); the derivative is the sum
    over the dropped factor (product rule), written out directly.
    """
    n = len(nodes)
    L = np.ones((n, len(x)))
    D = np.zeros((n, len(x)))
    for i in range(n):
        for m in range(n):
            if m == i:
                continue
            L[i] *= (x - nodes[m]) / (nodes[i] - nodes[m])
        for m in range(n):
            if m == i:
                continue
            term = np.full(len(x), 1.0 / (nodes[i] - nodes[m]))
            for j in range(n):
                if j == i or j == m:
                    continue
                term = term * (x - nodes[j]) / (nodes[i] - nodes[j])
            D[i] += term
    return L, D


# ----------------------------------------------------------------------------
# mesh
# ----------------------------------------------------------------------------
class Mesh:
    """Structured hexahedral mesh with periodic or homogeneous-Dirichlet faces.

    cell e = (cz*ny + cy)*nx + cx; local node i = (iz*np + iy)*np + ix;
    free global node I = (gz*Ny + gy)*Nx + gx over free nodes only.
    """

    def __init__(self, ncell, h, p, periodic):
        self.ncell = tuple(int(n) for n in ncell)
        self.h = np.asarray(h, np.float64)
        self.p = int(p)
        self.np1 = self.p + 1
        self.periodic = tuple(bool(b) for b in periodic)
        self.nfree = [n * self.p if per else n * self.p - 1
                      for n, per in zip(self.ncell, self.periodic)]
        self.nnodes = int(np.prod(self.nfree))
        self.ncells = int(np.prod(self.ncell))
        self.jac = float(np.prod(self.h)) / 8.0
        self.cell_nodes = self._cell_nodes()

    def _free_index_1d(self, d, c, i):
        g = c * self.p + i
        n = self.ncell[d] * self.p
        if self.periodic[d]:
            return g % n
        if g == 0 or g == n:
            return -1
        return g - 1

    def _cell_nodes(self):
        nx, ny, nz = self.ncell
        n1 = self.np1
        Nx, Ny, _ = self.nfree
        out = np.empty((self.ncells, n1 ** 3), np.int64)
        for cz in range(nz):
            for cy in range(ny):
                for cx in range(nx):
                    e = (cz * ny + cy) * nx + cx
                    for iz in range(n1):
                        gz = self._free_index_1d(2, cz, iz)
                        for iy in range(n1):
                            gy = self._free_index_1d(1, cy, iy)
                            for ix in range(n1):
                                gx = self._free_index_1d(0, cx, ix)
                                i = (iz * n1 + iy) * n1 + ix
                                out[e, i] = -1 if min(gx, gy, gz) < 0 else (gz * Ny + gy) * Nx + gx
        return out

    def cell_origin(self, e):
        nx, ny, _ = self.ncell
        cx = e % nx
        cy = (e // nx) % ny
        cz = e // (nx * ny)
        return np.array([cx, cy, cz]) * self.h


class CellTables:
    """Reference-cell tables for one mesh: 3-D Lagrange values and physical
    gradients at the Gauss points (full tensor products, not factorised),
    and w_q J (Eq. cellIntegrals)."""

    def __init__(self, mesh: Mesh, nq: int):
        self.nq = nq
        xg, _ = gll(mesh.p)
        xq, wq = gauss(nq)
        L1, D1 = lagrange(xg, xq)
        n1 = mesh.np1
        # N3[i, q] = l_ix(xq_qx) l_iy(xq_qy) l_iz(xq_qz)
        ii = np.arange(n1 ** 3)
        ix, iy, iz = ii % n1, (ii // n1) % n1, ii // (n1 * n1)
        qq = np.arange(nq ** 3)
        qx, qy, qz = qq % nq, (qq // nq) % nq, qq // (nq * nq)
        Lx, Ly, Lz = L1[ix][:, qx], L1[iy][:, qy], L1[iz][:, qz]
        Dx, Dy, Dz = D1[ix][:, qx], D1[iy][:, qy], D1[iz][:, qz]
        self.N3 = Lx * Ly * Lz
        # d/dx = (2/h_x) d/dxi
        self.D3 = np.stack([(2.0 / mesh.h[0]) * Dx * Ly * Lz,
                            (2.0 / mesh.h[1]) * Lx * Dy * Lz,
                            (2.0 / mesh.h[2]) * Lx * Ly * Dz])
        self.W = wq[qx] * wq[qy] * wq[qz] * mesh.jac
        t = (xq + 1.0) * 0.5
        self.ref = np.stack([t[qx] * mesh.h[0], t[qy] * mesh.h[1], t[qz] * mesh.h[2]], -1)


def lumped_mass(mesh: Mesh) -> np.ndarray:
    """M_D (Sec. III.B.2): diagonal mass from GLL quadrature at the nodes,
    M_D[I] = sum over cells containing I of w^GLL_ix w^GLL_iy w^GLL_iz J."""
    _, wg = gll(mesh.p)
    n1 = mesh.np1
    ii = np.arange(n1 ** 3)
    w3 = wg[ii % n1] * wg[(ii // n1) % n1] * wg[ii // (n1 * n1)] * mesh.jac
    md = np.zeros(mesh.nnodes)
    for e in range(mesh.ncells):
        nodes = mesh.cell_nodes[e]
        ok = nodes >= 0
        np.add.at(md, nodes[ok], w3[ok])
    return md


# ----------------------------------------------------------------------------
# the discrete operator
# ----------------------------------------------------------------------------
class Discretisation:
    """Everything the oracle needs for one synthetic ``Problem``."""

    def __init__(self, prob):
        self.prob = prob
        self.mesh = Mesh(prob.ncell, prob.h, prob.p, prob.periodic)
        self.tab = CellTables(self.mesh, prob.nq)
        self.k = np.asarray(prob.k, np.float64)
        self.md = lumped_mass(self.mesh)
        self.proj = [self._projector(a) for a in prob.atoms]

    # ---- Eq. CMat (with R_a and the Bloch phase of Eq. HnlocPeriodic)
    def _projector(self, atom):
        """Sparse P_a: (node list, values[nodes, npj]) with
        P_{I chi} = sum_(e,L) sum_q w_q J N_I(r_q) e^{-ik.(r_q - L)} p_chi(r_q - L - R_a)."""
        mesh, tab = self.mesh, self.tab
        box = np.array([n * h for n, h in zip(mesh.ncell, mesh.h)])
        acc = {}
        for s, (e, img) in enumerate(zip(atom.supp_cell, atom.supp_img)):
            rq = mesh.cell_origin(int(e)) + tab.ref
            L = np.asarray(img) * box
            phase = np.exp(-1j * ((rq - L) @ self.k))
            f = (tab.W * phase)[:, None] * atom.pvals[s]          # [q, npj]
            Pe = tab.N3 @ f                                        # [i, npj]
            for i, I in enumerate(mesh.cell_nodes[int(e)]):
                if I < 0:
                    continue
                acc[I] = acc.get(I, 0) + Pe[i]
        nodes = np.array(sorted(acc), np.int64)
        vals = np.array([acc[I] for I in nodes]).reshape(len(nodes), atom.npj)
        return nodes, vals

    def projector_dense(self, a):
        nodes, vals = self.proj[a]
        P = np.zeros((self.mesh.nnodes, vals.shape[1]), np.complex128)
        P[nodes] = vals
        return P

    # ---- form O1b: element-by-element quadrature apply
    def apply_local(self, X: np.ndarray, chunk: int = 64, cells=None) -> np.ndarray:
        """Y = H^loc X cell by cell (Eq. FEHloc, Eq. cellIntegrals).

        X[M][2][nv] complex.  For each cell: u, grad u at the Gauss points by
        full Lagrange sums, the pointwise integrand, then the test-function sums
        (N_I and grad N_I) scattered to the global nodes.
        """
        prob, mesh, tab = self.prob, self.mesh, self.tab
        M, _, nv = X.shape
        Y = np.zeros_like(X, dtype=np.complex128)
        Xp = np.concatenate([X.astype(np.complex128), np.zeros((1, 2, nv), np.complex128)])
        k = self.k
        k2 = 0.5 * float(k @ k)
        W = tab.W
        all_cells = np.arange(mesh.ncells) if cells is None else np.asarray(cells)
        for c0 in range(0, len(all_cells), chunk):
            cells = all_cells[c0:c0 + chunk]
            idx = mesh.cell_nodes[cells]                        # [C, n]
            Xc = Xp[np.where(idx >= 0, idx, M)]                 # [C, n, 2, nv]
            C = len(cells)
            Xm = Xc.reshape(C, Xc.shape[1], 2 * nv)
            # u and grad u at the Gauss points (library matmul, full 3-D tables)
            U = (tab.N3.T @ Xm).reshape(C, -1, 2, nv)
            G = [(tab.D3[d].T @ Xm).reshape(C, -1, 2, nv) for d in range(3)]

            def test(B, F):            # sum_q B[i, q] F[c, q, a, v]
                return (B @ F.reshape(C, F.shape[1], 2 * nv)).reshape(C, B.shape[0], 2, nv)
            # kinetic: 1/2 int grad N_I . grad u
            Yc = 0.5 * sum(test(tab.D3[d], W[None, :, None, None] * G[d]) for d in range(3))
            # -i int N_I k . grad u
            kg = sum(k[d] * G[d] for d in range(3))
            # |k|^2/2 + V_eff, and B_xc . sigma
            V = prob.veff[cells][:, :, None, None]
            Bx = prob.bx[cells][:, :, None]
            By = prob.by[cells][:, :, None]
            Bz = prob.bz[cells][:, :, None]
            pt = -1j * kg + (k2 + V) * U
            pt[:, :, 0, :] += Bz * U[:, :, 0, :] + (Bx - 1j * By) * U[:, :, 1, :]
            pt[:, :, 1, :] += (Bx + 1j * By) * U[:, :, 0, :] - Bz * U[:, :, 1, :]
            Yc = Yc + test(tab.N3, W[None, :, None, None] * pt)
            ok = idx >= 0
            np.add.at(Y, idx[ok], Yc[ok])
        return Y

    def apply_nonlocal(self, X: np.ndarray) -> np.ndarray:
        """Y = sum_a (P_a x I2) Delta_a (P_a x I2)^H X (Eq. FEHnloc)."""
        Y = np.zeros_like(X, dtype=np.complex128)
        nv = X.shape[2]
        for (nodes, P), atom in zip(self.proj, self.prob.atoms):
            npj = P.shape[1]
            C = np.einsum("ic,iav->cav", P.conj(), X[nodes])          # [npj, 2, nv]
            Cp = (atom.delta @ C.reshape(2 * npj, nv)).reshape(npj, 2, nv)
            Y[nodes] += np.einsum("ic,cav->iav", P, Cp)
        return Y

    def apply_h(self, X: np.ndarray) -> np.ndarray:
        """H^k X (form O1b): local element-by-element + nonlocal."""
        return self.apply_local(X) + self.apply_nonlocal(X)

    def apply_h_rows(self, X: np.ndarray, nodes) -> np.ndarray:
        """(H^k X)[nodes] only: the element loop runs over the cells that touch
        the requested nodes (the only cells contributing to those rows)."""
        nodes = np.asarray(nodes)
        cells = np.nonzero(np.isin(self.mesh.cell_nodes, nodes).any(axis=1))[0]
        return (self.apply_local(X, cells=cells) + self.apply_nonlocal(X))[nodes]

    def apply_htilde(self, X: np.ndarray) -> np.ndarray:
        """M_D^-1 H X."""
        return self.apply_h(X) / self.md[:, None, None]

    # ---- form O1a: explicit assembled matrix
    def element_matrix(self, e: int) -> np.ndarray:
        """Dense H^loc(e), (2 n_p^3)^2, DOF index 2i + alpha (Eq. FEHloc on one cell)."""
        prob, tab = self.prob, self.tab
        W = tab.W
        k = self.k
        S = 0.5 * sum(tab.D3[d] @ (W[:, None] * tab.D3[d].T) for d in range(3))
        S = S.astype(np.complex128)
        S += -1j * sum(k[d] * (tab.N3 @ (W[:, None] * tab.D3[d].T)) for d in range(3))
        S += tab.N3 @ ((W * (0.5 * float(k @ k) + prob.veff[e]))[:, None] * tab.N3.T)
        H = np.kron(S, np.eye(2))
        for d, B in enumerate((prob.bx, prob.by, prob.bz)):
            Bm = tab.N3 @ ((W * B[e])[:, None] * tab.N3.T)
            H = H + np.kron(Bm, PAULI[d])
        return H

    def assemble_local(self) -> sp.csr_matrix:
        """H^loc = sum_e R^(e)T H^loc(e) R^(e) as a sparse 2M x 2M matrix."""
        mesh = self.mesh
        rows, cols, vals = [], [], []
        for e in range(mesh.ncells):
            He = self.element_matrix(e)
            nodes = mesh.cell_nodes[e]
            dof = np.stack([2 * nodes, 2 * nodes + 1], -1).reshape(-1)
            ok = np.repeat(nodes >= 0, 2)
            d = dof[ok]
            Hs = He[np.ix_(ok, ok)]
            rows.append(np.repeat(d, len(d)))
            cols.append(np.tile(d, len(d)))
            vals.append(Hs.reshape(-1))
        n = 2 * mesh.nnodes
        return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(n, n)).tocsr()

    def dense_h(self) -> np.ndarray:
        """Full dense H^k (tiny meshes only)."""
        H = self.assemble_local().toarray()
        for a, atom in enumerate(self.prob.atoms):
            Pt = np.kron(self.projector_dense(a), np.eye(2))
            H += Pt @ atom.delta @ Pt.conj().T
        return H


class MatrixOp:
    """H applied through the explicit sparse local matrix plus the low-rank
    nonlocal terms (form O1a)."""

    def __init__(self, disc: Discretisation):
        self.disc = disc
        self.Hloc = disc.assemble_local()

    def apply(self, X: np.ndarray) -> np.ndarray:
        M, _, nv = X.shape
        Y = (self.Hloc @ X.reshape(2 * M, nv)).reshape(M, 2, nv)
        for a, atom in enumerate(self.disc.prob.atoms):
            Pt = sp.kron(sp.csr_matrix(self.disc.projector_dense(a)), sp.eye(2)).tocsr()
            Y += (Pt @ (atom.delta @ (Pt.conj().T @ X.reshape(2 * M, nv)))).reshape(M, 2, nv)
        return Y
