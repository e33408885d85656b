"""Densities rho and m at the Gauss points on the GPU (gbc_density, gbc_density_dev;
Eqs. rho and mag) against the FP64 oracle.

* small meshes, element by element: p = 2..6, periodic and Dirichlet faces, k != 0,
  ragged vector counts (the FP32 kernel takes two vectors per CTA), padded columns
  filled with NaN (never read), zero and negative occupations;
* the device-output form equals the host-output form bit for bit;
* the full cube16_p6 mesh (16^3 cells, p = 6, 884,736 nodes) on sampled cells, FP64 and
  FP32, and there the quadrature integral sum_q w_q J rho_q = sum_n f_n x_n^H
  (H[V+1] - H[V]) x_n through the GPU's own H.X (FP64).

Tolerances (relative to max rho, which bounds |m|): FP64 forms products and sums in
FP64, 1e-12.  FP32 interpolates in FP32 (3 sum-factorised stages of p + 1 terms on O(1)
values, ~1e-7 each) and forms the per-vector products in FP32 before the FP64 sum:
2e-6.
"""
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


def padded_block(X, ldx, dt):
    M, _, nv = X.shape
    out = torch.full((M, 2, ldx), complex(float("nan"), float("nan")), dtype=dt)
    out[:, :, :nv] = torch.from_numpy(X).to(dt)
    return out.cuda()


CASES = [
    # p, periodic, k, nvec, ldx, prec
    (2, (1, 1, 1), (0.2, -0.1, 0.3), 5, 8, 0),
    (3, (0, 1, 0), (0.0, 0.0, 0.0), 3, 3, 1),
    (4, (1, 1, 1), (0.1, 0.25, -0.2), 7, 9, 1),
    (5, (1, 0, 1), (0.3, 0.0, 0.1), 4, 6, 1),
    (6, (1, 0, 1), (0.0, 0.2, 0.0), 4, 4, 0),
    (6, (1, 1, 1), (0.15, 0.1, -0.05), 9, 12, 1),
]


@pytest.mark.parametrize("p,periodic,k,nvec,ldx,prec", CASES)
def test_density_matches_oracle(g, p, periodic, k, nvec, ldx, prec):
    prob = syn.make_problem(ncell=(3, 2, 2), h=(1.1, 0.9, 1.2), p=p, k=k, periodic=periodic,
                            natoms=1, rc=1.0, seed=40 + p, bmax=0.2)
    d = fe.Discretisation(prob)
    X = syn.random_block(d.mesh.nnodes, nvec, 50 + p)
    occ = np.random.default_rng(p).uniform(0.0, 1.0, nvec)
    occ[0] = 0.0
    occ[-1] = -0.3
    rho_o, m_o = od.densities(d, X, occ)
    c = g.Context(0)
    c.set_problem(prob)
    c.set_precision(prec)
    dt = torch.complex128 if prec == 0 else torch.complex64
    Xd = padded_block(X, ldx, dt)
    rho, m = c.density(Xd, occ, nvec=nvec)
    tol = 1e-12 if prec == 0 else 2e-6
    scale = np.abs(rho_o).max()
    assert np.all(np.isfinite(rho)) and np.all(np.isfinite(m))
    np.testing.assert_allclose(rho, rho_o, rtol=0, atol=tol * scale)
    np.testing.assert_allclose(m, m_o, rtol=0, atol=tol * scale)
    # device form: same kernel, same bits
    out = torch.full((d.mesh.ncells, 4, prob.nq ** 3), float("nan"), dtype=torch.float64,
                     device="cuda")
    occ_d = torch.from_numpy(occ).cuda()
    c.density_dev(Xd, occ_d, out, nvec=nvec)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.array_equal(o[:, 0], rho)
    assert np.array_equal(np.moveaxis(o[:, 1:], 1, 0), m)
    c.close()


def test_density_argument_errors(g):
    prob = syn.make_problem(ncell=(2, 2, 2), p=2, natoms=0, seed=1)
    c = g.Context(0)
    c.set_problem(prob)
    Xd = torch.zeros((prob.nnodes, 2, 4), dtype=torch.complex128, device="cuda")
    with pytest.raises(g.GbcError):
        c.density(Xd, np.ones(4), nvec=5)          # nvec > ldx
    with pytest.raises(g.GbcError):
        c.density(Xd, np.ones(4), nvec=0)
    rho, m = c.density(Xd, np.ones(4))             # the context is still usable
    assert not rho.any() and not m.any()
    c.close()


@pytest.fixture(scope="module")
def cube16():
    prob = syn.config("cube16_p6", kindex=1)
    d = fe.Discretisation(prob)
    X = syn.random_block(d.mesh.nnodes, 32, 61)
    occ = np.random.default_rng(7).uniform(0.0, 1.0, 32)
    cells = np.unique(np.concatenate([[0, d.mesh.ncells - 1],
                                      np.random.default_rng(8).integers(0, d.mesh.ncells, 22)]))
    rho_o, m_o = od.densities(d, X, occ, cells=cells)
    return prob, d, X, occ, cells, rho_o, m_o


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-6)])
def test_density_full_mesh_sampled_cells(g, cube16, prec, tol):
    prob, d, X, occ, cells, rho_o, m_o = cube16
    c = g.Context(0)
    c.set_problem(prob)
    c.set_precision(prec)
    dt = torch.complex128 if prec == 0 else torch.complex64
    Xd = torch.from_numpy(X).to(dt).cuda()
    rho, m = c.density(Xd, occ)
    scale = np.abs(rho_o).max()
    np.testing.assert_allclose(rho[cells], rho_o, rtol=0, atol=tol * scale)
    np.testing.assert_allclose(m[:, cells], m_o, rtol=0, atol=tol * scale)
    assert np.all(np.sqrt((m ** 2).sum(0)) <= rho * (1 + 1e-5) + 1e-6 * scale)
    if prec == 0:
        # sum_q w_q J rho_q against the V-shift of the GPU H.X at the full size
        HX = torch.empty_like(Xd)
        c.apply_h(Xd, HX)
        c.set_fields(prob.veff + 1.0, prob.bx, prob.by, prob.bz)
        HX1 = torch.empty_like(Xd)
        c.apply_h(Xd, HX1)
        f = torch.from_numpy(occ).cuda()
        lhs = float(((Xd.conj() * (HX1 - HX)).real.sum(dim=(0, 1)) * f).sum())
        rhs = float((d.tab.W[None, :] * rho).sum())
        assert abs(lhs - rhs) < 1e-10 * abs(rhs), (lhs, rhs)
    c.close()
