"""Densities summed over k-points on the GPU: the accumulate mode of gbc_density_dev and
kpoints.sharded_density / sharded_occupations in one process (two k-points, Fermi-Dirac
occupations with a common chemical potential) against the FP64 oracle."""
import numpy as np
import pytest

import synthetic as syn
from oracle import density as od
from oracle import fe

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import __graft_entry__ as ge
    ge.build()
    import paper_2410_02754_gb300 as pkg
    return pkg


@pytest.mark.parametrize("prec", [0, 1])
def test_accumulate_adds_exactly(g, prec):
    """accumulate = 1 adds the same sums: twice the overwrite result, bit for bit."""
    prob = syn.make_problem(ncell=(3, 2, 2), h=(1.1, 0.9, 1.2), p=3, natoms=1, rc=1.0, seed=43)
    c = g.Context(0)
    c.set_problem(prob)
    c.set_precision(prec)
    dt = torch.complex128 if prec == 0 else torch.complex64
    X = torch.from_numpy(syn.random_block(prob.nnodes, 7, 9)).to(dt).cuda()
    occ = torch.from_numpy(np.linspace(1.0, 0.1, 7)).cuda()
    out = torch.empty((prob.ncells, 4, prob.nq ** 3), dtype=torch.float64, device="cuda")
    c.density_dev(X, occ, out)
    torch.cuda.synchronize()
    once = out.cpu().numpy()
    c.density_dev(X, occ, out, accumulate=True)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), 2.0 * once)
    c.close()


def test_brillouin_zone_density_two_kpoints(g):
    """rho, m summed over two k-points with Fermi-Dirac occupations of common chemical
    potential (gbc_fermi_occupations + gbc_density_dev accumulate, single process)
    against the oracle's weighted sum."""
    from paper_2410_02754_gb300 import kpoints
    base = syn.make_problem(ncell=(2, 2, 3), h=(1.0, 1.1, 0.9), p=3, natoms=1, rc=1.0, seed=71,
                            bmax=0.2)
    ks = [(0.1, 0.0, -0.2), (-0.1, 0.25, 0.05)]
    w = np.array([0.4, 0.6])
    nv, kT = 6, 0.05
    eps = np.sort(np.random.default_rng(5).uniform(-1.0, 1.0, (2, nv)), axis=1)
    occ, mu = kpoints.sharded_occupations(eps, w, 4.2, kT)
    f_o, mu_o = od.fermi_occupations(eps, w, 4.2, kT)
    assert abs(mu - mu_o) < 1e-12
    ctxs, blocks, ref = [], [], 0.0
    for i, k in enumerate(ks):
        prob = base.with_(k=np.asarray(k))
        d = fe.Discretisation(prob)
        X = syn.random_block(d.mesh.nnodes, nv, 80 + i)
        r, mm = od.densities(d, X, w[i] * f_o[i])
        ref = ref + np.concatenate([r[:, None], np.moveaxis(mm, 0, 1)], 1)
        c = g.Context(0)
        c.set_problem(prob)
        ctxs.append(c)
        blocks.append(torch.from_numpy(X).cuda())
    out = torch.full((base.ncells, 4, base.nq ** 3), float("nan"), dtype=torch.float64,
                     device="cuda")
    kpoints.sharded_density(ctxs, blocks, occ, w, out)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    for c in ctxs:
        c.close()
