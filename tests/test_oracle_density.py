"""PIN-12: the oracle's densities rho and m at the Gauss points (Eqs. rho, mag) against
what the mathematics fixes independently of its formula:

* polynomial reproduction + the Bloch sphere: nodal values X = (a_n, b_n) phi(r_I) of a
  polynomial phi of degree <= p vanishing on the Dirichlet faces give psi_n(r_q) =
  (a_n, b_n) phi(r_q) exactly, so rho = sum f (|a|^2 + |b|^2) phi^2 and m = sum f |a, b|^2
  n(theta, varphi) phi^2 with the textbook Bloch vector n of (cos theta/2, e^{i varphi}
  sin theta/2) -- pins the gather order, the Gauss-point coordinates and each sigma
  (a sign error in m_y or a swapped u/d fails it);
* the quadrature integrals: sum_q w_q J rho_q = sum_n f_n x_n^H (H[V+1] - H[V]) x_n and
  sum_q w_q J m^d_q = sum_n f_n x_n^H (H[B^d+1] - H[B^d]) x_n, with the oracle's element
  apply of Eq. FEHloc (a second, independently pinned code path);
* |m| = rho for one spinor, |m| <= rho for non-negative occupations (Cauchy-Schwarz);
* an SU(2) rotation U of every spinor leaves rho unchanged and rotates m by the SO(3)
  matrix R_ij = tr(sigma_i U sigma_j U^H) / 2.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import density as od
from oracle import fe

PAULI = [np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]]),
         np.array([[1, 0], [0, -1]], complex)]


@pytest.fixture(scope="module")
def disc():
    prob = syn.make_problem(ncell=(2, 3, 2), h=(1.1, 0.9, 1.3), p=3, k=(0.2, -0.1, 0.15),
                            natoms=0, seed=21, bmax=0.3)
    return fe.Discretisation(prob)


def node_coords(mesh):
    """Coordinates of the free nodes, from the cell -> node map and the GLL nodes."""
    xg, _ = fe.gll(mesh.p)
    n1 = mesh.np1
    out = np.zeros((mesh.nnodes, 3))
    i = np.arange(n1 ** 3)
    loc = np.stack([xg[i % n1], xg[(i // n1) % n1], xg[i // (n1 * n1)]], -1)
    for e in range(mesh.ncells):
        r = mesh.cell_origin(e) + 0.5 * (loc + 1.0) * mesh.h
        ok = mesh.cell_nodes[e] >= 0
        out[mesh.cell_nodes[e][ok]] = r[ok]
    return out


def test_bloch_sphere_polynomial():
    prob = syn.make_problem(ncell=(2, 2, 3), h=(1.0, 1.4, 0.8), p=3, natoms=0, seed=3,
                            periodic=(0, 0, 0))
    d = fe.Discretisation(prob)
    box = prob.box
    phi = lambda r: (r[..., 0] * (box[0] - r[..., 0]) * r[..., 1] * (box[1] - r[..., 1])
                     * r[..., 2] * (box[2] - r[..., 2]) * (1.0 + 0.3 * r[..., 0]))
    rn = node_coords(d.mesh)
    rng = np.random.default_rng(0)
    nv = 4
    th, vp = rng.uniform(0, np.pi, nv), rng.uniform(0, 2 * np.pi, nv)
    amp = rng.uniform(0.5, 2.0, nv)
    gam = rng.uniform(0, 2 * np.pi, nv)                               # a free global phase
    a = amp * np.cos(th / 2) * np.exp(1j * gam)
    b = amp * np.sin(th / 2) * np.exp(1j * (gam + vp))
    X = np.zeros((d.mesh.nnodes, 2, nv), complex)
    X[:, 0, :] = phi(rn)[:, None] * a[None, :]
    X[:, 1, :] = phi(rn)[:, None] * b[None, :]
    f = rng.uniform(0.1, 1.0, nv)
    rho, m = od.densities(d, X, f)
    rq = np.stack([d.mesh.cell_origin(e) + d.tab.ref for e in range(d.mesh.ncells)])
    p2 = phi(rq) ** 2
    nvec = np.stack([np.sin(th) * np.cos(vp), np.sin(th) * np.sin(vp), np.cos(th)])
    w = f * amp ** 2
    np.testing.assert_allclose(rho, p2 * w.sum(), rtol=1e-11, atol=1e-12)
    for c in range(3):
        np.testing.assert_allclose(m[c], p2 * (nvec[c] * w).sum(), rtol=1e-10, atol=1e-11)


def test_quadrature_integrals_match_hamiltonian_difference(disc):
    prob = disc.prob
    nv = 3
    X = syn.random_block(disc.mesh.nnodes, nv, 4)
    f = np.array([1.0, 0.4, 0.75])
    rho, m = od.densities(disc, X, f)
    W = disc.tab.W[None, :]
    base = disc.apply_local(X)

    def quad_form(prob2):
        dY = fe.Discretisation(prob2).apply_local(X) - base
        return float(np.real(np.einsum("isn,isn,n->", X.conj(), dY, f)))

    np.testing.assert_allclose((W * rho).sum(), quad_form(prob.with_(veff=prob.veff + 1.0)),
                               rtol=1e-11)
    for c, key in enumerate(("bx", "by", "bz")):
        shifted = prob.with_(**{key: getattr(prob, key) + 1.0})
        np.testing.assert_allclose((W * m[c]).sum(), quad_form(shifted), rtol=1e-10,
                                   atol=1e-10 * abs((W * rho).sum()))


def test_single_spinor_is_fully_polarised(disc):
    X = syn.random_block(disc.mesh.nnodes, 1, 8)
    rho, m = od.densities(disc, X, [0.7])
    np.testing.assert_allclose(np.sqrt((m ** 2).sum(0)), rho, rtol=1e-12, atol=1e-14)
    X = syn.random_block(disc.mesh.nnodes, 5, 9)
    rho, m = od.densities(disc, X, [1.0, 0.2, 0.0, 0.9, 0.5])
    assert np.all(np.sqrt((m ** 2).sum(0)) <= rho * (1 + 1e-12))
    assert np.all(rho >= 0)


def test_su2_rotation_covariance(disc):
    X = syn.random_block(disc.mesh.nnodes, 4, 10)
    f = np.array([1.0, 0.3, 0.6, 0.05])
    rho, m = od.densities(disc, X, f)
    ax = np.array([0.3, -0.8, 0.5])
    ax /= np.linalg.norm(ax)
    t = 1.1
    U = np.cos(t / 2) * np.eye(2) - 1j * np.sin(t / 2) * sum(a * s for a, s in zip(ax, PAULI))
    XU = np.einsum("st,itn->isn", U, X)
    rho2, m2 = od.densities(disc, XU, f)
    R = np.array([[0.5 * np.trace(si @ U @ sj @ U.conj().T).real for sj in PAULI] for si in PAULI])
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
    np.testing.assert_allclose(rho2, rho, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(m2, np.einsum("ij,jeq->ieq", R, m), rtol=1e-11, atol=1e-12)


# ---- Fermi-Dirac occupations (Sec. II electron-count constraint, Sec. V smearing) -------
KT = 500.0 * 3.166811563e-6          # 500 K in Ha


def test_fermi_count_and_bounds():
    rng = np.random.default_rng(3)
    eps = np.sort(rng.uniform(-1.0, 2.0, (3, 40)), axis=1)
    w = np.array([0.25, 0.5, 0.25])
    f, mu = od.fermi_occupations(eps, w, 17.3, KT)
    assert abs((w[:, None] * f).sum() - 17.3) < 1e-11
    assert np.all((f >= 0) & (f <= 1))
    # decreasing in eps within every k-point, and 1/2 at eps = mu
    assert np.all(np.diff(f, axis=1) <= 0)
    np.testing.assert_allclose(od.fermi(np.zeros(1)), [0.5])


def test_fermi_closed_forms():
    # one state holding a fraction q: mu = eps + kT ln(q / (1 - q))
    for q in (0.1, 0.5, 0.93):
        f, mu = od.fermi_occupations([[0.3]], [1.0], q, KT)
        np.testing.assert_allclose(mu, 0.3 + KT * np.log(q / (1 - q)), rtol=0, atol=1e-14)
        np.testing.assert_allclose(f[0, 0], q, rtol=1e-12)
    # a spectrum symmetric about c at half filling: mu = c (f(-x) = 1 - f(x))
    half = np.random.default_rng(4).uniform(0.001, 0.01, 12)
    eps = np.concatenate([0.2 - half, 0.2 + half])[None, :]
    f, mu = od.fermi_occupations(eps, [1.0], 12.0, KT)
    assert abs(mu - 0.2) < 1e-13


def test_fermi_aufbau_limit():
    # a gap much larger than kT: the N_e lowest states (over all k-points) are full
    eps = np.array([[-0.5, -0.2, 0.4, 0.9], [-0.45, 0.5, 0.6, 1.0]])
    f, mu = od.fermi_occupations(eps, [0.5, 0.5], 1.5, KT)
    full = np.array([[1, 1, 0, 0], [1, 0, 0, 0]], float)
    np.testing.assert_allclose(f, full, atol=1e-12)
    assert -0.2 < mu < 0.4
