"""H.X at the full size of the semi-periodic slab workload (slab40_p6: 40x40x20 cells, p = 6,
6,854,400 free nodes, periodic in x and y, Dirichlet in z, 640 atoms with 18 SOC projectors)
on sampled rows, FP64 and FP32, against the FP64 oracle.

The oracle evaluates only the sampled rows: the element apply over the cells touching them,
and the nonlocal term of the atoms whose supports contain them (no other atom contributes
to those rows).  Rows are drawn in the bottom vacuum, across the periodic x and y wraps, inside
the slab and on the top Dirichlet face.  8 vectors.  Tolerances as for H.X elsewhere: 1e-12
(FP64) and 1e-5 (FP32) relative over the sampled rows."""
import numpy as np
import pytest

import synthetic as syn
from oracle import fe

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import __graft_entry__ as ge
    ge.build()
    import paper_2410_02754_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def slab():
    prob = syn.config("slab40_p6")
    mesh = fe.Mesh(prob.ncell, prob.h, prob.p, prob.periodic)
    Nx, Ny, Nz = mesh.nfree
    rng = np.random.default_rng(1)

    def node(gx, gy, gz):
        return (gz * Ny + gy) * Nx + gx

    nodes = [node(rng.integers(Nx), rng.integers(Ny), rng.integers(1, 12)) for _ in range(8)]
    nodes += [node(0, rng.integers(Ny), rng.integers(30, 90)) for _ in range(4)]
    nodes += [node(rng.integers(Nx), Ny - 1, rng.integers(30, 90)) for _ in range(4)]
    nodes += [node(rng.integers(Nx), rng.integers(Ny), rng.integers(30, 90)) for _ in range(8)]
    nodes += [node(rng.integers(Nx), rng.integers(Ny), Nz - 1) for _ in range(2)]
    nodes = np.unique(nodes)
    cells = np.nonzero(np.isin(mesh.cell_nodes, nodes).any(axis=1))[0]
    near = [a for a in prob.atoms if np.isin(a.supp_cell, cells).any()]
    d = fe.Discretisation(prob.with_(atoms=near))
    X = syn.random_block(mesh.nnodes, 8, 5)
    ref = d.apply_h_rows(X, nodes)
    return prob, X, nodes, ref


@pytest.fixture(scope="module")
def slab_ctx(g, slab):
    c = g.Context(0)
    c.set_problem(slab[0])            # 640 atoms, 4 GB of projector values: set once
    yield c
    c.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_slab_hx_sampled_rows(g, slab, slab_ctx, prec, tol):
    prob, X, nodes, ref = slab
    c = slab_ctx
    c.set_precision(prec)
    dt = torch.complex128 if prec == 0 else torch.complex64
    Xd = torch.from_numpy(X).to(dt).cuda()
    Yd = torch.empty_like(Xd)
    c.apply_h(Xd, Yd)
    c.sync_status()
    out = Yd[torch.from_numpy(nodes).cuda()].cpu().numpy().astype(np.complex128)
    del Xd, Yd
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert err < tol, err
