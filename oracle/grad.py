"""Reverse-mode gradients through the scaled Chebyshev filter, plain FP64 (oracle).

Test infrastructure only (see ``oracle/__init__``).

Loss (the cube16_p6_grad workload): L = sum_i w_i y_i^H H y_i with Y = rho_m(M_D^-1 H) X_0
(Eq. chebfilt, sigma-scaled), H from Eqs. FEHloc / FEHnloc.  Gradients use the
convention grad = dL/dRe + i dL/dIm for complex quantities, so for a
Hermitian form z^H A z the gradient is 2 A z.

Recurrence X_{k+1} = alpha_k L X_k - beta_k X_{k-1}, L = (M_D^-1 H - c)/e,
alpha_0 = sigma_1, beta_0 = 0, alpha_k = 2 sigma_{k+1}, beta_k = sigma_k sigma_{k+1}.
Adjoint: Lam_k = alpha_k L^H Lam_{k+1} - beta_{k+1} Lam_{k+2}; with
Lt_k = M_D^-1 Lam_k this is Lt_k = alpha_k L Lt_{k+1} - beta_{k+1} Lt_{k+2}
(M_D^-1 L^H M_D = L), Lt_m = M_D^-1 G_Y, and grad_X0 = M_D Lt_0.
Parameters: dL/dtheta = sum_k (alpha_k / e) Re(Lt_{k+1}^H (dH/dtheta) X_k), where
dH/dV_q = w_q J N(r_q) N(r_q)^T x I2 and dH/dB^d_q the same with sigma^d, and
dH/dDelta_a enters through the projector coefficients C = (P_a x I2)^H (.).
"""
from __future__ import annotations

import numpy as np

from . import chfsi as oc


def coefficients(m, lT, lmax, lmin):
    """alpha_k, beta_k (k = 0..m-1) of the sigma-scaled recurrence, and c, e."""
    c, e, s = oc.sigma_sequence(m, lT, lmax, lmin)
    alpha = [s[0]] + [2.0 * s[k] for k in range(1, m)]
    beta = [0.0] + [s[k - 1] * s[k] for k in range(1, m)]
    return c, e, alpha, beta


def quad_products(d, A, B, wv):
    """g[e, c, q] = sum_v wv[v] w_q J Re(a_v(r_q)^H S_c b_v(r_q)), S = (I, sx, sy, sz),
    a_v(r_q) = sum_I A[I, :, v] N_I(r_q) (full Lagrange sums per cell)."""
    mesh, tab = d.mesh, d.tab
    M, _, nv = A.shape
    nq3 = tab.N3.shape[1]
    out = np.zeros((mesh.ncells, 4, nq3))
    Ap = np.concatenate([A, np.zeros((1, 2, nv), A.dtype)])
    Bp = np.concatenate([B, np.zeros((1, 2, nv), B.dtype)])
    wv = np.asarray(wv, np.float64)
    for c0 in range(0, mesh.ncells, 64):
        cells = np.arange(c0, min(mesh.ncells, c0 + 64))
        idx = mesh.cell_nodes[cells]
        sel = np.where(idx >= 0, idx, M)
        C = len(cells)
        ua = (tab.N3.T @ Ap[sel].reshape(C, -1, 2 * nv)).reshape(C, nq3, 2, nv)
        ub = (tab.N3.T @ Bp[sel].reshape(C, -1, 2 * nv)).reshape(C, nq3, 2, nv)
        au, ad, bu, bd = ua[:, :, 0], ua[:, :, 1], ub[:, :, 0], ub[:, :, 1]
        prods = [au.conj() * bu + ad.conj() * bd,
                 au.conj() * bd + ad.conj() * bu,
                 -1j * au.conj() * bd + 1j * ad.conj() * bu,
                 au.conj() * bu - ad.conj() * bd]
        for ci, pr in enumerate(prods):
            out[cells, ci] = (pr.real * wv[None, None, :]).sum(-1) * tab.W[None, :]
    return out


def proj_coeffs(d, A):
    """Per atom C_a = (P_a x I2)^H A, shape [2 npj, nv], row 2 chi + s."""
    out = []
    for nodes, P in d.proj:
        C = np.einsum("ic,iav->cav", P.conj(), A[nodes])
        out.append(C.reshape(-1, A.shape[2]))
    return out


def energy_and_direct_grads(d, Y, w):
    """L = sum_i w_i y_i^H H y_i, G_Y = 2 H Y diag(w), and the direct
    (Y held fixed) gradients with respect to V, B (per quadrature point) and Delta_a."""
    HY = d.apply_h(Y)
    w = np.asarray(w, np.float64)
    L = float(np.real(np.einsum("iav,iav,v->", Y.conj(), HY, w)))
    GY = 2.0 * HY * w[None, None, :]
    g = quad_products(d, Y, Y, w)
    Cs = proj_coeffs(d, Y)
    gD = [(Cy * w[None, :]) @ Cy.conj().T for Cy in Cs]
    return L, GY, g, gD


def filter_vjp(d, X0, GY, m, lT, lmax, lmin):
    """Vector-Jacobian product of Y = filter(X0; H): returns grad_X0, g[E, 4, q]
    (V, Bx, By, Bz at quadrature points) and the Hermitian-projected Delta gradients."""
    c, e, alpha, beta = coefficients(m, lT, lmax, lmin)

    def Lop(Z):
        return (d.apply_htilde(Z) - c * Z) / e

    Xs = [X0]
    for k in range(m):
        nxt = alpha[k] * Lop(Xs[k])
        if k > 0:
            nxt = nxt - beta[k] * Xs[k - 1]
        Xs.append(nxt)
    md = d.md[:, None, None]
    Lt = {m: GY / md, m + 1: np.zeros_like(X0)}
    nv = X0.shape[2]
    g = np.zeros((d.mesh.ncells, 4, d.tab.N3.shape[1]))
    gD = [np.zeros((P.shape[1] * 2, P.shape[1] * 2), complex) for _, P in d.proj]
    for k in range(m - 1, -1, -1):
        f = alpha[k] / e
        g += f * quad_products(d, Lt[k + 1], Xs[k], np.ones(nv))
        Ca, Cx = proj_coeffs(d, Lt[k + 1]), proj_coeffs(d, Xs[k])
        for a in range(len(gD)):
            gD[a] += f * Ca[a] @ Cx[a].conj().T
        nb = beta[k + 1] if k + 1 < m else 0.0
        Lt[k] = alpha[k] * Lop(Lt[k + 1]) - nb * Lt[k + 2]
    gD = [0.5 * (G + G.conj().T) for G in gD]
    return md * Lt[0], g, gD


def total_loss(d, X0, w, m, lT, lmax, lmin):
    Y = oc.cheb_filter(d.apply_htilde, X0, m, lT, lmax, lmin)
    HY = d.apply_h(Y)
    return float(np.real(np.einsum("iav,iav,v->", Y.conj(), HY, np.asarray(w))))
