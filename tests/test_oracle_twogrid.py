"""PIN-13: the oracle's two-grid transfer (order p_c -> p_f on the same mesh, Eq.
FEWfnsCMesh) against what the mathematics fixes:

* polynomial reproduction: nodal values of a polynomial of degree <= p_c in each coordinate
  (vanishing on the Dirichlet faces) are carried to its exact values at the fine nodes --
  pins the 1-D transfer matrix, the tensor order and the cell -> node maps of both orders;
* p_f = p_c is the identity;
* the FE function is unchanged, so its mass form and its kinetic + Bloch form are the same
  under the coarse and the fine element apply of Eq. FEHloc (Gauss n_q = p + 2 integrates both
  exactly at either order): a dropped or misplaced entry changes them.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import fe
from oracle import twogrid as tg


def node_coords(mesh):
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


def pair(pc, pf, **kw):
    base = syn.make_problem(p=pc, natoms=0, **kw)
    return fe.Discretisation(base), fe.Discretisation(base.with_(p=pf, nq=pf + 2,
                                                                  veff=None, bx=None, by=None,
                                                                  bz=None)), base


@pytest.mark.parametrize("pc,pf", [(3, 4), (3, 6), (4, 5)])
def test_polynomial_reproduction(pc, pf):
    kw = dict(ncell=(2, 3, 2), h=(1.0, 0.8, 1.3), periodic=(0, 0, 0), seed=2)
    dc, df, base = pair(pc, pf, **kw)
    box = base.box
    phi = lambda r: (r[..., 0] * (box[0] - r[..., 0]) * r[..., 1] * (box[1] - r[..., 1])
                     * r[..., 2] * (box[2] - r[..., 2]) * (1.0 - 0.4 * r[..., 0] + 0.2 * r[..., 2]))
    ab = np.array([[1.0 + 0.5j, -0.3j], [0.2, 0.7 - 0.1j]])           # [spin, vector]
    Xc = phi(node_coords(dc.mesh))[:, None, None] * ab[None]
    Xf = tg.prolongate(dc, df, Xc)
    ref = phi(node_coords(df.mesh))[:, None, None] * ab[None]
    np.testing.assert_allclose(Xf, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_same_order_is_identity():
    prob = syn.make_problem(ncell=(2, 2, 2), p=3, natoms=0, seed=4, periodic=(1, 0, 1))
    d = fe.Discretisation(prob)
    X = syn.random_block(d.mesh.nnodes, 3, 5)
    assert np.array_equal(tg.prolongate(d, d, X), X)


@pytest.mark.parametrize("pc,pf", [(3, 4), (2, 5)])
def test_mass_and_kinetic_forms_preserved(pc, pf):
    prob_c = syn.make_problem(ncell=(2, 2, 3), h=(1.1, 0.9, 1.0), p=pc, k=(0.2, -0.1, 0.3),
                              natoms=0, seed=6, periodic=(1, 1, 0))
    E = prob_c.ncells

    def zero_fields(prob, nq):
        z = np.zeros((E, nq ** 3))
        return prob.with_(veff=z, bx=z, by=z, bz=z)

    pk_c = zero_fields(prob_c, pc + 2)
    pk_f = zero_fields(prob_c.with_(p=pf, nq=pf + 2), pf + 2)
    dc, df = fe.Discretisation(pk_c), fe.Discretisation(pk_f)
    Xc = syn.random_block(dc.mesh.nnodes, 2, 7)
    Xf = tg.prolongate(dc, df, Xc)

    def forms(prob, d, X, nq):
        kin = np.einsum("isn,isn->n", X.conj(), d.apply_local(X)).real
        one = np.ones((E, nq ** 3))
        dm = fe.Discretisation(prob.with_(veff=one)).apply_local(X) - d.apply_local(X)
        mass = np.einsum("isn,isn->n", X.conj(), dm).real
        return kin, mass

    kc, mc = forms(pk_c, dc, Xc, pc + 2)
    kf, mf = forms(pk_f, df, Xf, pf + 2)
    np.testing.assert_allclose(kf, kc, rtol=1e-11)
    np.testing.assert_allclose(mf, mc, rtol=1e-11)
