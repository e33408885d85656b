"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each checks a closed form, an
invariant, a textbook special case, a library routine used as an independent
reference, or brute force on a tiny problem.
"""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import chfsi as oc
from oracle import fe


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------
def tiny(ncell=(2, 2, 2), p=2, k=(0.0, 0.0, 0.0), natoms=2, h=(1.5, 1.5, 1.5), seed=3,
         periodic=(1, 1, 1), **kw):
    return syn.make_problem(ncell=ncell, h=h, p=p, periodic=periodic, k=k, natoms=natoms,
                            rc=1.2, seed=seed, **kw)


def const_fields(prob, V0=0.0, b=(0.0, 0.0, 0.0)):
    return prob.with_(veff=np.full_like(prob.veff, V0), bx=np.full_like(prob.bx, b[0]),
                      by=np.full_like(prob.by, b[1]), bz=np.full_like(prob.bz, b[2]))


def gen_eigs_numpy(H, md):
    d = np.repeat(1 / np.sqrt(md), 2)
    A = d[:, None] * H * d[None, :]
    return np.linalg.eigvalsh(0.5 * (A + A.conj().T))


# ----------------------------------------------------------------------------
# PIN-11: quadrature and Lagrange basis
# ----------------------------------------------------------------------------
def test_gll_textbook_values():
    x, w = fe.gll(2)
    assert np.allclose(x, [-1, 0, 1]) and np.allclose(w, [1 / 3, 4 / 3, 1 / 3])
    x, w = fe.gll(3)
    s = 1 / math.sqrt(5)
    assert np.allclose(x, [-1, -s, s, 1]) and np.allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6])


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 7])
def test_gll_gauss_exactness(p):
    x, w = fe.gll(p)
    assert abs(w.sum() - 2) < 1e-13
    for deg in range(2 * p):            # GLL exact to degree 2p - 1
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(np.sum(w * x ** deg) - exact) < 1e-12
    nq = p + 2
    xq, wq = fe.gauss(nq)
    for deg in range(2 * nq):           # Gauss exact to degree 2nq - 1
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(np.sum(wq * xq ** deg) - exact) < 1e-12
    # GLL is not exact at degree 2p (checks the rule is GLL, not Gauss)
    assert abs(np.sum(w * x ** (2 * p)) - 2.0 / (2 * p + 1)) > 1e-6


@pytest.mark.parametrize("p", [2, 4, 6])
def test_lagrange_cardinal_and_derivative(p):
    x, _ = fe.gll(p)
    L, D = fe.lagrange(x, x)
    assert np.allclose(L, np.eye(p + 1), atol=1e-13)
    t = np.linspace(-1, 1, 37)
    L, D = fe.lagrange(x, t)
    assert np.allclose(L.sum(0), 1.0, atol=1e-12)           # partition of unity
    assert np.allclose(D.sum(0), 0.0, atol=1e-10)
    eps = 1e-6
    Lp, _ = fe.lagrange(x, t + eps)
    Lm, _ = fe.lagrange(x, t - eps)
    assert np.allclose((Lp - Lm) / (2 * eps), D, atol=1e-6)
    # derivative of the interpolant of x^p is p x^(p-1)
    assert np.allclose((x ** p) @ D, p * t ** (p - 1), atol=1e-10)


# ----------------------------------------------------------------------------
# mesh and lumped mass
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("periodic", [(1, 1, 1), (1, 1, 0), (0, 0, 0)])
def test_mesh_node_map(periodic):
    m = fe.Mesh((3, 2, 4), (1.0, 1.3, 0.7), 3, periodic)
    nodes = m.cell_nodes
    used = np.unique(nodes[nodes >= 0])
    assert len(used) == m.nnodes and used[0] == 0 and used[-1] == m.nnodes - 1
    expect = [n * 3 if per else n * 3 - 1 for n, per in zip((3, 2, 4), periodic)]
    assert m.nnodes == int(np.prod(expect))
    # cell-interior nodes belong to exactly one cell
    cnt = np.bincount(nodes[nodes >= 0], minlength=m.nnodes)
    n1 = 4
    ii = np.arange(n1 ** 3)
    inner = ((ii % n1 > 0) & (ii % n1 < 3) & ((ii // n1) % n1 > 0) & ((ii // n1) % n1 < 3)
             & (ii // 16 > 0) & (ii // 16 < 3))
    assert np.all(cnt[nodes[:, inner]] == 1)


def test_lumped_mass_volume():
    m = fe.Mesh((3, 2, 4), (1.0, 1.3, 0.7), 4, (1, 1, 1))
    md = fe.lumped_mass(m)
    assert abs(md.sum() - 3 * 1.0 * 2 * 1.3 * 4 * 0.7) < 1e-12
    assert np.all(md > 0)


# ----------------------------------------------------------------------------
# PIN-1: Hermiticity (k != 0, SOC, B)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("k", [(0, 0, 0), (0.31, -0.2, 0.45)])
def test_hermitian_assembled(k):
    prob = tiny(k=k)
    d = fe.Discretisation(prob)
    H = d.dense_h()
    assert np.linalg.norm(H - H.conj().T) <= 1e-13 * np.linalg.norm(H)


def test_hermitian_elementwise_form():
    prob = tiny(ncell=(3, 2, 2), p=3, k=(0.2, 0.1, -0.3), natoms=3)
    d = fe.Discretisation(prob)
    M = d.mesh.nnodes
    Y1 = syn.random_block(M, 3, 1)
    Y2 = syn.random_block(M, 4, 2)
    a = Y1.reshape(2 * M, -1).conj().T @ d.apply_h(Y2).reshape(2 * M, -1)
    b = (Y2.reshape(2 * M, -1).conj().T @ d.apply_h(Y1).reshape(2 * M, -1)).conj().T
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_dirichlet_hermitian_and_positive_kinetic():
    prob = tiny(periodic=(1, 0, 1), k=(0.2, 0.0, 0.1), natoms=0, bmax=0.0)
    prob = const_fields(prob)
    d = fe.Discretisation(prob)
    H = d.dense_h()
    assert np.linalg.norm(H - H.conj().T) <= 1e-13 * np.linalg.norm(H)
    assert np.linalg.eigvalsh(H).min() > 0          # Dirichlet kills the constant mode


# ----------------------------------------------------------------------------
# PIN-2: exact constant mode
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("b,chi,sign", [
    ((0.0, 0.07, 0.0), (1, 1j), +1),        # sigma_y eigenvector (1, i)/sqrt2 -> +|b|
    ((0.0, 0.07, 0.0), (1, -1j), -1),
    ((0.05, 0.0, 0.0), (1, 1), +1),
    ((0.0, 0.0, 0.05), (0, 1), -1),
])
@pytest.mark.parametrize("form", ["O1a", "O1b"])
def test_constant_mode(b, chi, sign, form):
    k = np.array([0.13, -0.27, 0.4])
    V0 = -0.7
    prob = const_fields(tiny(p=3, k=k, natoms=0), V0, b)
    d = fe.Discretisation(prob)
    M = d.mesh.nnodes
    chi = np.array(chi, np.complex128) / np.linalg.norm(chi)
    U = np.zeros((M, 2, 1), np.complex128)
    U[:, :, 0] = chi[None, :]
    HU = d.apply_h(U) if form == "O1b" else fe.MatrixOp(d).apply(U)
    lam = 0.5 * k @ k + V0 + sign * np.linalg.norm(b)
    assert np.abs(HU - lam * d.md[:, None, None] * U).max() < 1e-13


# ----------------------------------------------------------------------------
# PIN-3: free particle -> 1/2 |k + G|^2, converging with p
# ----------------------------------------------------------------------------
def test_free_particle_convergence():
    L = 4.0
    k = np.array([0.3, 0.0, -0.1])
    G = [np.array(g) * 2 * np.pi / L for g in np.ndindex(5, 5, 5)]
    G = [g - 2 * 2 * np.pi / L for g in G]
    exact = np.sort(np.repeat([0.5 * np.sum((k + g) ** 2) for g in G], 2))[:14]
    errs = []
    for p in (2, 3, 4, 5):
        prob = const_fields(tiny(h=(2.0, 2.0, 2.0), p=p, k=k, natoms=0))
        d = fe.Discretisation(prob)
        ev = gen_eigs_numpy(d.dense_h(), d.md)[:14]
        errs.append(np.abs(ev - exact).max())
    assert errs[-1] < 1e-3
    assert all(errs[i + 1] < errs[i] for i in range(3))


# ----------------------------------------------------------------------------
# PIN-4: SOC off and B = 0 -> exact 2-fold degeneracy
# ----------------------------------------------------------------------------
def test_spin_degeneracy_without_soc():
    prob = tiny(p=3, k=(0.1, 0.2, 0.0), natoms=2)
    prob = prob.with_(bx=0 * prob.bx, by=0 * prob.by, bz=0 * prob.bz)
    rng = np.random.default_rng(7)
    for a in prob.atoms:
        dd = rng.normal(0, 0.1, (a.npj, a.npj))
        a.delta = np.kron(dd + dd.T, np.eye(2)).astype(np.complex128)
    d = fe.Discretisation(prob)
    ev = gen_eigs_numpy(d.dense_h(), d.md)
    assert np.abs(ev[0::2] - ev[1::2]).max() < 1e-10
    # with SOC on the degeneracy is lifted (guards against a vacuous pass)
    prob2 = tiny(p=3, k=(0.1, 0.2, 0.0), natoms=2)
    prob2 = prob2.with_(bx=0 * prob2.bx, by=0 * prob2.by, bz=0 * prob2.bz)
    d2 = fe.Discretisation(prob2)
    ev2 = gen_eigs_numpy(d2.dense_h(), d2.md)
    assert np.abs(ev2[0::2] - ev2[1::2]).max() > 1e-6


# ----------------------------------------------------------------------------
# PIN-5: SU(2) invariance
# ----------------------------------------------------------------------------
def test_su2_invariance():
    prob = tiny(p=3, k=(0.1, -0.2, 0.3), natoms=2, bmax=0.3)
    n = np.array([0.3, -0.5, 0.8])
    n /= np.linalg.norm(n)
    th = 0.9
    U = math.cos(th / 2) * np.eye(2) - 1j * math.sin(th / 2) * np.einsum("d,dab->ab", n, fe.PAULI)
    # adjoint representation R_ij = 1/2 tr(sigma_i U sigma_j U^H)
    R = np.array([[0.5 * np.trace(fe.PAULI[i] @ U @ fe.PAULI[j] @ U.conj().T).real
                   for j in range(3)] for i in range(3)])
    B = np.stack([prob.bx, prob.by, prob.bz], -1) @ R.T
    atoms2 = []
    for a in prob.atoms:
        W = np.kron(np.eye(a.npj), U)
        atoms2.append(syn.Atom(a.pos, a.npj, a.supp_cell, a.supp_img, a.pvals, W @ a.delta @ W.conj().T))
    prob2 = prob.with_(bx=B[..., 0].copy(), by=B[..., 1].copy(), bz=B[..., 2].copy(), atoms=atoms2)
    e1 = gen_eigs_numpy(fe.Discretisation(prob).dense_h(), fe.Discretisation(prob).md)
    d2 = fe.Discretisation(prob2)
    e2 = gen_eigs_numpy(d2.dense_h(), d2.md)
    assert np.abs(e1 - e2).max() < 1e-10
    # rotating only B (not Delta) must change the spectrum when SOC is on
    prob3 = prob.with_(bx=B[..., 0].copy(), by=B[..., 1].copy(), bz=B[..., 2].copy())
    d3 = fe.Discretisation(prob3)
    assert np.abs(e1 - gen_eigs_numpy(d3.dense_h(), d3.md)).max() > 1e-8


# ----------------------------------------------------------------------------
# PIN-6: Kramers pairs and the L.S 4 + 2 split of a p manifold
# ----------------------------------------------------------------------------
def _ls_delta(xi):
    """Delta = xi L.S in the real-harmonic (y, z, x) x spin basis, index 2*chi+alpha."""
    # complex l=1 basis |m>, real harmonics: Y_y = i/sqrt2 (Y_1,-1 + Y_1,1),
    # Y_z = Y_1,0, Y_x = 1/sqrt2 (Y_1,-1 - Y_1,1)
    s2 = 1 / math.sqrt(2)
    C = np.array([[1j * s2, 0, 1j * s2], [0, 1, 0], [s2, 0, -s2]])   # rows: real fn in |m=-1,0,1>
    Lz = np.diag([-1.0, 0, 1.0]).astype(complex)
    Lp = np.zeros((3, 3), complex)
    Lp[1, 0] = Lp[2, 1] = math.sqrt(2)
    Lm = Lp.conj().T
    Lx, Ly = 0.5 * (Lp + Lm), -0.5j * (Lp - Lm)
    Lr = [C.conj() @ Lk @ C.T for Lk in (Lx, Ly, Lz)]                # in the real basis
    S = [0.5 * s for s in fe.PAULI]
    return xi * sum(np.kron(Lr[d], S[d]) for d in range(3))


def test_kramers_and_ls_split():
    """Atom at the centre of a cubic-symmetric periodic mesh, deep well, B = 0:
    every level is a Kramers pair, and xi L.S splits the 6-fold p-like level
    into a doublet (j = 1/2, shift -xi w) and a quartet (j = 3/2, +xi w / 2),
    the Lande interval ratio -2 to first order."""
    def spectrum(xi):
        prob = syn.make_problem(ncell=(3, 3, 3), h=(1.4, 1.4, 1.4), p=3, k=(0, 0, 0),
                                atom_pos=[[2.1, 2.1, 2.1]], channels=((0.45, 1),), bmax=0.0,
                                rc=1.6, seed=11, well_depth=6.0)
        prob.atoms[0].delta = _ls_delta(xi)
        d = fe.Discretisation(prob)
        return gen_eigs_numpy(d.dense_h(), d.md)

    ev0, ev = spectrum(0.0), spectrum(0.1)
    assert np.abs(ev[0::2] - ev[1::2]).max() < 1e-9            # Kramers pairs
    p0 = ev0[2:8]
    assert np.ptp(p0) < 1e-9                                    # 6-fold p level without SOC
    d2, q4 = ev[2:4], ev[4:8]
    assert np.ptp(d2) < 1e-9 and np.ptp(q4) < 1e-9              # 2 + 4 split (Gamma6 + Gamma8)
    assert q4[0] - d2[0] > 1e-3
    ratio = (d2[0] - p0[0]) / (q4[0] - p0[0])
    assert abs(ratio + 2.0) < 0.15


# ----------------------------------------------------------------------------
# PIN-7: Chebyshev closed form
# ----------------------------------------------------------------------------
def test_chebyshev_scalar_recurrence():
    x = np.linspace(-3, 3, 61)
    T0, T1 = np.ones_like(x), x.copy()
    for m in range(2, 31):
        T0, T1 = T1, 2 * x * T1 - T0
        assert np.allclose(oc.cheb_T(m, x), T1, rtol=1e-11, atol=1e-11)
    # sigma-scaled scalar recurrence equals rho_m
    lT, lmax, lmin = 1.0, 9.0, -2.0
    lam = np.linspace(-2, 9, 23)
    c, e, s = oc.sigma_sequence(20, lT, lmax, lmin)
    y0 = np.ones_like(lam)
    y1 = s[0] / e * (lam - c) * y0
    for k in range(1, 20):
        y0, y1 = y1, 2 * s[k] / e * (lam - c) * y1 - s[k - 1] * s[k] * y0
    assert np.allclose(y1, oc.filter_scalar(20, lam, lT, lmax, lmin), rtol=1e-12)


def test_filter_on_exact_eigenvectors():
    prob = tiny(p=2, k=(0.2, 0, 0), natoms=1)
    d = fe.Discretisation(prob)
    H = d.dense_h()
    w, V = np.linalg.eigh((lambda dd: dd[:, None] * H * dd[None, :])(np.repeat(d.md ** -0.5, 2)))
    X = (np.repeat(d.md ** -0.5, 2)[:, None] * V[:, :6]).reshape(-1, 2, 6)   # generalised eigvecs
    lT, lmax, lmin = float(w[10]), float(w[-1]) + 0.1, float(w[0]) - 0.05
    Y = oc.cheb_filter(d.apply_htilde, X, 12, lT, lmax, lmin)
    rho = oc.filter_scalar(12, w[:6], lT, lmax, lmin)
    assert np.abs(Y - X * rho[None, None, :]).max() <= 1e-11 * np.abs(X * rho).max()


# ----------------------------------------------------------------------------
# PIN-8: ChFSI converges to the dense lowest eigenvalues
# ----------------------------------------------------------------------------
def test_chfsi_matches_brute_force():
    prob = tiny(ncell=(2, 2, 2), p=3, k=(0.15, -0.1, 0.05), natoms=2, h=(1.3, 1.3, 1.3))
    d = fe.Discretisation(prob)
    exact = gen_eigs_numpy(d.dense_h(), d.md)
    M = d.mesh.nnodes
    nwant, nblk = 8, 14
    lmin, lmax = oc.lanczos_bounds(d.apply_htilde, d.md, syn.random_start(M, 1), 30)
    assert lmax >= exact[-1] - 1e-9
    hist, X = oc.chfsi(d.apply_h, d.md, syn.random_block(M, nblk, 2), cycles=25, degree=12,
                       lmin=lmin, lmax=lmax)
    assert np.abs(hist[-1][:nwant] - exact[:nwant]).max() < 1e-9


def test_lanczos_full_dimension_is_exact():
    prob = tiny(ncell=(2, 1, 1), p=2, natoms=0, h=(1.0, 1.0, 1.0))
    d = fe.Discretisation(prob)
    exact = gen_eigs_numpy(d.dense_h(), d.md)
    n = 2 * d.mesh.nnodes
    lmin, lmax = oc.lanczos_bounds(d.apply_htilde, d.md, syn.random_start(d.mesh.nnodes, 3), n - 1)
    assert abs(lmin - exact[0]) < 1e-9
    assert lmax >= exact[-1] - 1e-9


# ----------------------------------------------------------------------------
# PIN-9: identities
# ----------------------------------------------------------------------------
def test_matrix_and_elementwise_forms_agree():
    prob = tiny(ncell=(3, 2, 2), p=3, k=(0.2, -0.3, 0.1), natoms=3, periodic=(1, 1, 0))
    d = fe.Discretisation(prob)
    X = syn.random_block(d.mesh.nnodes, 5, 4)
    Y1 = fe.MatrixOp(d).apply(X)
    Y2 = d.apply_h(X)
    assert np.abs(Y1 - Y2).max() <= 1e-13 * np.abs(Y1).max()


def test_md_self_adjoint():
    prob = tiny(ncell=(2, 3, 2), p=3, k=(0.1, 0.2, -0.2), natoms=2)
    d = fe.Discretisation(prob)
    M = d.mesh.nnodes
    X, Y = syn.random_block(M, 3, 5), syn.random_block(M, 3, 6)
    a = oc.gram(Y, d.md, d.apply_htilde(X))
    b = oc.gram(d.apply_htilde(Y), d.md, X)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_cholgs_orthonormal_and_cholesky():
    prob = tiny(ncell=(2, 2, 2), p=3, natoms=1)
    d = fe.Discretisation(prob)
    X = syn.random_block(d.mesh.nnodes, 16, 8)
    Q = oc.cholgs(X, d.md)
    assert np.abs(oc.gram(Q, d.md) - np.eye(16)).max() < 1e-12
    S = oc.gram(X, d.md)
    L = oc.cholesky(S)
    assert np.abs(L @ L.conj().T - S).max() < 1e-12 * np.abs(S).max()
    assert np.allclose(np.triu(L, 1), 0)
    with pytest.raises(ValueError):
        oc.cholesky(np.diag([1.0, -1.0]).astype(complex))


def test_jacobi_matches_library():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(20, 20)) + 1j * rng.normal(size=(20, 20))
    A = A + A.conj().T
    A[3, :] = A[:, 3] = 0
    A[3, 3] = 1.0                       # exact degeneracy handling
    w, V = oc.jacobi_eigh(A)
    assert np.allclose(w, np.linalg.eigvalsh(A), atol=1e-12)
    assert np.abs(V.conj().T @ V - np.eye(20)).max() < 1e-13
    assert np.abs(A @ V - V * w).max() < 1e-12


def test_residual_split_equals_direct():
    prob = tiny(ncell=(2, 2, 2), p=3, k=(0.1, 0, 0.2), natoms=2)
    d = fe.Discretisation(prob)
    M = d.mesh.nnodes
    X = oc.cholgs(syn.random_block(M, 6, 9), d.md)
    ritz, X, HX = oc.rayleigh_ritz(d.apply_h, X)
    lT, lmax, lmin = float(ritz[-1]), 60.0, float(ritz[0]) - 0.1
    A = oc.cheb_filter(d.apply_htilde, X, 15, lT, lmax, lmin)
    B = oc.cheb_filter_split(d.apply_htilde, X, ritz, 15, lT, lmax, lmin,
                             HtX=HX / d.md[:, None, None])
    assert np.abs(A - B).max() <= 1e-12 * np.abs(A).max()


# ----------------------------------------------------------------------------
# planted mistakes: each must be caught by one of the pins above
# ----------------------------------------------------------------------------
def test_planted_sigma_y_sign_is_caught(monkeypatch):
    """Flip the sign of the B_y sigma_y term in the element-wise apply: PIN-2 fails."""
    prob = const_fields(tiny(p=2, natoms=0), -0.3, (0.0, 0.07, 0.0))
    d = fe.Discretisation(prob)
    M = d.mesh.nnodes
    U = np.zeros((M, 2, 1), complex)
    U[:, 0, 0], U[:, 1, 0] = 1 / math.sqrt(2), 1j / math.sqrt(2)
    d.prob = d.prob.with_(by=-d.prob.by)       # the planted mistake
    lam = -0.3 + 0.07
    assert np.abs(d.apply_h(U) - lam * d.md[:, None, None] * U).max() > 1e-3


def _k_shift_gap(p, planted=False):
    """max |eig(H^k) - eig(H^(k+G))| over the lowest levels; G a reciprocal vector."""
    L = 3.0
    k = np.array([0.25, 0.1, 0.0])
    out = []
    for kk in (k, k + np.array([2 * np.pi / L, 0, 0])):
        prob = syn.make_problem(ncell=(2, 2, 2), h=(1.5, 1.5, 1.5), p=p, k=kk, natoms=2, rc=1.2,
                                seed=3, channels=((0.5, 0), (0.5, 1)), delta_std=0.5)
        d = fe.Discretisation(prob)
        if planted:                       # the mistake: conj(P) Delta P^T
            d.proj = [(n, v.conj()) for n, v in d.proj]
        out.append(gen_eigs_numpy(d.dense_h(), d.md)[:6])
    return np.abs(out[0] - out[1]).max()


def test_bloch_phase_convention_k_periodicity():
    """Continuum H^(k+G) = e^{-iG.r} H^k e^{iG.r}: the discrete spectra at k and
    k+G converge to each other with p only if local k-terms and the projector
    Bloch phases (Eq. HnlocPeriodic) use consistent conventions."""
    g3, g5 = _k_shift_gap(3), _k_shift_gap(5)
    assert g5 < 0.05 and g5 < g3 / 5
    assert _k_shift_gap(5, planted=True) > 0.3
