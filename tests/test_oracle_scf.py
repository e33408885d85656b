"""PIN-14: the oracle's SCF pieces against what the mathematics fixes.

* exchange stand-in: m = 0 gives Dirac exchange -(3/4)(3/pi)^(1/3) rho^(4/3) and
  V = -(3/pi)^(1/3) rho^(1/3); |m| = rho gives -(3/4)(6/pi)^(1/3) rho^(4/3); V and B equal
  central finite differences of the energy density in rho and in each m_d; a rotation of m
  rotates B and leaves e and V unchanged;
* inner product (Eq. innerPdt): constant fields give (a^2 + |b|^2)/2 times the box volume;
* Anderson mixing: one history entry is linear mixing; the optimal coefficients satisfy the
  constrained minimum's conditions (G b = lambda 1, sum b = 1); on a linear contraction of
  dimension n it reaches the fixed point within n + 1 steps (its GMRES equivalence).
"""
import numpy as np

import synthetic as syn
from oracle import fe
from oracle import scf


def test_exchange_closed_forms():
    rho = np.array([1e-3, 0.2, 1.0, 7.5])
    e, V, B = scf.lsda_exchange(rho, np.zeros((3, 4)))
    np.testing.assert_allclose(e, -0.75 * (3 / np.pi) ** (1 / 3) * rho ** (4 / 3), rtol=1e-14)
    np.testing.assert_allclose(V, -(3 / np.pi) ** (1 / 3) * np.cbrt(rho), rtol=1e-14)
    assert not B.any()
    m = np.stack([rho * 0.6, -rho * 0.8, 0 * rho])             # |m| = rho
    e, V, B = scf.lsda_exchange(rho, m)
    np.testing.assert_allclose(e, -0.75 * (6 / np.pi) ** (1 / 3) * rho ** (4 / 3), rtol=1e-14)


def test_exchange_derivatives_by_finite_differences():
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.1, 2.0, 50)
    m = rng.normal(size=(3, 50))
    m *= (rng.uniform(0.05, 0.95, 50) * rho / np.sqrt((m * m).sum(0)))[None]
    e, V, B = scf.lsda_exchange(rho, m)
    h = 1e-6
    ep = scf.lsda_exchange(rho + h, m)[0]
    em = scf.lsda_exchange(rho - h, m)[0]
    np.testing.assert_allclose((ep - em) / (2 * h), V, rtol=1e-7)
    for d in range(3):
        dm = np.zeros_like(m)
        dm[d] = h
        fd = (scf.lsda_exchange(rho, m + dm)[0] - scf.lsda_exchange(rho, m - dm)[0]) / (2 * h)
        np.testing.assert_allclose(fd, B[d], rtol=1e-6, atol=1e-9)


def test_exchange_rotation_covariance():
    rng = np.random.default_rng(4)
    rho = rng.uniform(0.1, 2.0, 20)
    m = rng.normal(size=(3, 20)) * 0.3 * rho[None]
    t = 0.9
    R = np.array([[np.cos(t), -np.sin(t), 0], [np.sin(t), np.cos(t), 0], [0, 0, 1.0]])
    R = R @ np.array([[1, 0, 0], [0, np.cos(0.4), -np.sin(0.4)], [0, np.sin(0.4), np.cos(0.4)]])
    e, V, B = scf.lsda_exchange(rho, m)
    e2, V2, B2 = scf.lsda_exchange(rho, R @ m)
    np.testing.assert_allclose(e2, e, rtol=1e-13)
    np.testing.assert_allclose(V2, V, rtol=1e-13)
    np.testing.assert_allclose(B2, R @ B, rtol=1e-12, atol=1e-15)


def test_inner_product_constant_fields():
    prob = syn.make_problem(ncell=(2, 3, 2), h=(1.1, 0.9, 1.3), p=3, natoms=0, seed=1)
    d = fe.Discretisation(prob)
    E, nq3 = d.mesh.ncells, d.tab.W.size
    x = np.zeros((E, 4, nq3))
    x[:, 0], x[:, 1], x[:, 2], x[:, 3] = 0.7, -0.2, 0.5, 0.1
    vol = float(np.prod(prob.box))
    np.testing.assert_allclose(scf.inner(d.tab.W, x, x), 0.5 * (0.49 + 0.04 + 0.25 + 0.01) * vol,
                               rtol=1e-13)


def test_anderson_single_history_and_optimality():
    rng = np.random.default_rng(5)
    W = rng.uniform(0.5, 1.5, 6)
    xs = [rng.normal(size=(2, 4, 6)) for _ in range(4)]
    rs = [rng.normal(size=(2, 4, 6)) for _ in range(4)]
    x1, b1 = scf.anderson(W, xs[:1], rs[:1], 0.3)
    assert np.array_equal(b1, [1.0])
    np.testing.assert_allclose(x1, xs[0] + 0.3 * rs[0], rtol=1e-15)
    x, b = scf.anderson(W, xs, rs, 0.3)
    assert abs(b.sum() - 1) < 1e-14
    rmix = sum(bj * rj for bj, rj in zip(b, rs))
    lam = [scf.inner(W, rj, rmix) for rj in rs]
    np.testing.assert_allclose(lam, lam[0], rtol=1e-10)


def test_anderson_finite_termination_on_linear_map():
    rng = np.random.default_rng(6)
    n = 8                                           # x is [1, 4, 2]: dimension 8
    W = np.array([0.7, 1.3])
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    A = Q @ np.diag(rng.uniform(-0.6, 0.6, n)) @ Q.T  # contraction
    c = rng.normal(size=n)
    F = lambda x: (A @ x.reshape(-1) + c).reshape(1, 4, 2)
    xstar = np.linalg.solve(np.eye(n) - A, c)
    x = np.zeros((1, 4, 2))
    xs, rs = [], []
    for it in range(n + 2):
        r = F(x) - x
        xs.append(x)
        rs.append(r)
        x, _ = scf.anderson(W, xs, rs, 1.0)
    assert np.abs(x.reshape(-1) - xstar).max() < 1e-8


def test_scf_loop_reaches_the_eigensolver_independent_fixed_point():
    """The SCF loop with one ChFSI cycle per step and with exact eigenpairs converge to the
    same self-consistent densities (the fixed point does not depend on the eigensolver)."""
    z = np.zeros((8, 4 ** 3))
    prob = syn.make_problem(ncell=(2, 2, 2), h=(1.0, 1.0, 1.0), p=2, natoms=2, rc=1.0, seed=9,
                            well_depth=3.0, bmax=0.0).with_(bx=z, by=z, bz=z)
    M = prob.nnodes
    X0 = syn.random_block(M, 12, 3)               # 3 electrons, 9 buffer states
    v0 = syn.random_start(M, 3)
    args = dict(nelec=3.0, kT=0.05, degree=16, lanczos_steps=12, alpha=0.5, nhist=4, iters=30)
    r_c, x_c, e_c = scf.scf_loop(prob, X0, v0, eig="chfsi", **args)
    r_d, x_d, e_d = scf.scf_loop(prob, X0, v0, eig="dense", **args)
    assert r_c[-1] < 1e-7 * r_c[0] and r_d[-1] < 1e-8 * r_d[0]
    np.testing.assert_allclose(x_c, x_d, rtol=0, atol=1e-7 * np.abs(x_d).max())
    np.testing.assert_allclose(e_c[:3], e_d[:3], rtol=0, atol=1e-8)


def _two_atom_problem(k=(0.0, 0.0, 0.0)):
    z = np.zeros((8, 4 ** 3))
    return syn.make_problem(ncell=(2, 2, 2), h=(1.0, 1.0, 1.0), p=2, k=k, natoms=2, rc=1.0,
                            seed=9, well_depth=3.0, bmax=0.0).with_(bx=z, by=z, bz=z)


def test_scf_k_loop_weights():
    """Two copies of one k-point with weights 0.3 / 0.7 reproduce the single-k loop."""
    prob = _two_atom_problem()
    M = prob.nnodes
    X0, v0 = syn.random_block(M, 12, 3), syn.random_start(M, 3)
    args = dict(nelec=3.0, kT=0.05, degree=16, lanczos_steps=12, alpha=0.5, nhist=4, iters=6)
    r1, x1, e1 = scf.scf_loop(prob, X0, v0, **args)
    r2, x2, e2 = scf.scf_loop_k([prob, prob], [X0, X0], [v0, v0], [0.3, 0.7], **args)
    # 0.3 f + 0.7 f rounds differently from f, and each step's filter amplifies rounding-level
    # differences of its input (~1e-10 relative after 6 steps): equal up to rounding
    np.testing.assert_allclose(r2, r1, rtol=1e-8)
    np.testing.assert_allclose(x2, x1, rtol=0, atol=1e-9 * np.abs(x1).max())
    np.testing.assert_allclose(e2[1], e1, rtol=1e-8)


def test_scf_k_loop_eigensolver_independent():
    """Two distinct k-points: one ChFSI cycle per step and exact eigenpairs reach the same
    Brillouin-zone-summed fixed point."""
    probs = [_two_atom_problem((0.3, 0.0, 0.0)), _two_atom_problem((-0.2, 0.4, 0.1))]
    M = probs[0].nnodes
    X0s = [syn.random_block(M, 12, 3 + i) for i in range(2)]
    v0s = [syn.random_start(M, 3 + i) for i in range(2)]
    args = dict(nelec=3.0, kT=0.05, degree=16, lanczos_steps=12, alpha=0.5, nhist=4, iters=30)
    r_c, x_c, e_c = scf.scf_loop_k(probs, X0s, v0s, [0.5, 0.5], eig="chfsi", **args)
    r_d, x_d, e_d = scf.scf_loop_k(probs, X0s, v0s, [0.5, 0.5], eig="dense", **args)
    assert r_c[-1] < 1e-7 * r_c[0] and r_d[-1] < 1e-8 * r_d[0]
    np.testing.assert_allclose(x_c, x_d, rtol=0, atol=1e-7 * np.abs(x_d).max())
    np.testing.assert_allclose(e_c[:, :3], e_d[:, :3], rtol=0, atol=1e-8)
