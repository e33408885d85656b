"""PIN-10: the oracle's reverse-mode gradients through the scaled Chebyshev
filter agree with central finite differences of the loss itself
(L = sum_i w_i y_i^H H y_i, Y = filter(X0; H)), along seeded random
directions in V_eff, B_xc (quadrature points), the Hermitian Delta_a and X0."""
import numpy as np
import pytest

import synthetic as syn
from oracle import fe
from oracle import grad as og

M_DEG, LT, LMAX, LMIN = 5, 2.0, 60.0, -2.0


@pytest.fixture(scope="module")
def setup():
    prob = syn.make_problem(ncell=(2, 2, 2), h=(1.3, 1.3, 1.3), p=2, k=(0.2, -0.1, 0.15),
                            natoms=2, rc=1.2, seed=12, bmax=0.3)
    d = fe.Discretisation(prob)
    rng = np.random.default_rng(5)
    X0 = syn.random_block(d.mesh.nnodes, 3, 7)
    w = rng.uniform(0, 1, 3)
    from oracle import chfsi as oc
    Y = oc.cheb_filter(d.apply_htilde, X0, M_DEG, LT, LMAX, LMIN)
    L, GY, gdir, gDdir = og.energy_and_direct_grads(d, Y, w)
    gX, gf, gDf = og.filter_vjp(d, X0, GY, M_DEG, LT, LMAX, LMIN)
    g = gdir + gf
    gD = [a + b for a, b in zip(gDdir, gDf)]
    return prob, X0, w, L, gX, g, gD, rng


def loss(prob, X0, w):
    return og.total_loss(fe.Discretisation(prob), X0, w, M_DEG, LT, LMAX, LMIN)


def fd(f, h=1e-4):
    return (f(h) - f(-h)) / (2 * h)


def test_loss_value_matches(setup):
    prob, X0, w, L, *_ = setup
    assert abs(L - loss(prob, X0, w)) < 1e-12 * abs(L)


@pytest.mark.parametrize("comp", [0, 1, 2, 3])
def test_field_gradients_vs_fd(setup, comp):
    prob, X0, w, L, gX, g, gD, rng = setup
    names = ["veff", "bx", "by", "bz"]
    for trial in range(3):
        dirn = rng.normal(size=prob.veff.shape)
        base = getattr(prob, names[comp])
        f = lambda h: loss(prob.with_(**{names[comp]: base + h * dirn}), X0, w)
        num = fd(f)
        ana = float(np.sum(g[:, comp] * dirn))
        assert abs(num - ana) <= 1e-6 * max(abs(num), 1e-3 * abs(L)), (comp, num, ana)


def test_delta_gradients_vs_fd(setup):
    prob, X0, w, L, gX, g, gD, rng = setup
    for a in range(len(prob.atoms)):
        n = prob.atoms[a].delta.shape[0]
        for trial in range(3):
            E = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
            E = 0.5 * (E + E.conj().T)

            def f(h):
                atoms = [syn.Atom(x.pos, x.npj, x.supp_cell, x.supp_img, x.pvals,
                                  x.delta + (h * E if i == a else 0)) for i, x in enumerate(prob.atoms)]
                return loss(prob.with_(atoms=atoms), X0, w)
            num = fd(f)
            ana = float(np.real(np.sum(gD[a].conj() * E)))
            assert abs(num - ana) <= 1e-6 * max(abs(num), 1e-3 * abs(L)), (a, num, ana)


def test_input_block_gradient_vs_fd(setup):
    prob, X0, w, L, gX, g, gD, rng = setup
    d = fe.Discretisation(prob)
    for trial in range(3):
        D = rng.normal(size=X0.shape) + 1j * rng.normal(size=X0.shape)
        f = lambda h: og.total_loss(d, X0 + h * D, w, M_DEG, LT, LMAX, LMIN)
        num = fd(f)
        ana = float(np.real(np.sum(gX.conj() * D)))
        assert abs(num - ana) <= 1e-6 * max(abs(num), 1e-3 * abs(L)), (num, ana)


def test_planted_adjoint_mistake_is_caught(setup, monkeypatch):
    """Drop the beta (three-term) coefficients inside the VJP: the X0 gradient
    no longer matches finite differences."""
    prob, X0, w, L, gX, g, gD, rng = setup
    d = fe.Discretisation(prob)
    from oracle import chfsi as oc
    Y = oc.cheb_filter(d.apply_htilde, X0, M_DEG, LT, LMAX, LMIN)
    _, GY, _, _ = og.energy_and_direct_grads(d, Y, w)
    good = og.coefficients
    monkeypatch.setattr(og, "coefficients",
                        lambda *a: (lambda c, e, al, be: (c, e, al, [0.0] * len(be)))(*good(*a)))
    wrong, _, _ = og.filter_vjp(d, X0, GY, M_DEG, LT, LMAX, LMIN)
    D = rng.normal(size=X0.shape) + 1j * rng.normal(size=X0.shape)
    num = fd(lambda h: og.total_loss(d, X0 + h * D, w, M_DEG, LT, LMAX, LMIN))
    gdx = 0.0   # the direct term has no X0 dependence beyond Y
    ana_wrong = float(np.real(np.sum(wrong.conj() * D))) + gdx
    assert abs(num - ana_wrong) > 1e-3 * abs(num)


def test_fifty_joint_directions_fourth_order(setup):
    """50 seeded joint directions (V_eff, B_x, B_y, B_z at every quadrature point, every
    Hermitian Delta_a, the input block X0 -- all perturbed together): the gradient's
    directional derivative agrees with the fourth-order central difference
    (8 (L(h) - L(-h)) - (L(2h) - L(-2h))) / 12h to 1e-7 relative.  The loss is a
    polynomial in the parameters, so the O(h^4) truncation at h = 1e-3 is far below the
    bound and rounding contributes ~eps |L| / h."""
    prob, X0, w, L, gX, g, gD, rng = setup
    rng = np.random.default_rng(2024)
    names = ["veff", "bx", "by", "bz"]
    base = [np.array(getattr(prob, n)) for n in names]
    worst = 0.0
    for trial in range(50):
        df = [rng.normal(size=b.shape) for b in base]
        E = []
        for a in prob.atoms:
            n = a.delta.shape[0]
            B = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
            E.append(0.5 * (B + B.conj().T))
        D = rng.normal(size=X0.shape) + 1j * rng.normal(size=X0.shape)

        def f(h):
            atoms = [syn.Atom(x.pos, x.npj, x.supp_cell, x.supp_img, x.pvals, x.delta + h * E[i])
                     for i, x in enumerate(prob.atoms)]
            p = prob.with_(atoms=atoms, **{n: b + h * d for n, b, d in zip(names, base, df)})
            return og.total_loss(fe.Discretisation(p), X0 + h * D, w, M_DEG, LT, LMAX, LMIN)

        h = 1e-3
        num = (8 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12 * h)
        ana = (sum(float(np.sum(g[:, c] * df[c])) for c in range(4))
               + sum(float(np.real(np.sum(gD[a].conj() * E[a]))) for a in range(len(E)))
               + float(np.real(np.sum(gX.conj() * D))))
        err = abs(num - ana) / max(abs(num), 1e-3 * abs(L))
        worst = max(worst, err)
    print(f"  PIN-10: 50 joint directions, worst relative error {worst:.2e}")
    assert worst <= 1e-7, worst
