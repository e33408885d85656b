"""Two-grid transfer on the GPU (gbc_prolongate, Eq. FEWfnsCMesh) against the FP64 oracle.

* small meshes, element by element, every supported order pair p -> p + 1 (2..7) and p -> p,
  periodic and Dirichlet faces, FP64 and FP32, ragged vector tiles (8 FP32 / 4 FP64 vectors
  per CTA), padded columns: NaN in the coarse padding (never read) and a sentinel in the fine
  padding (never written);
* the full cube16_p6 mesh (16^3 cells) from p = 5 to p = 6 on sampled cells, FP32;
* argument errors, after which the contexts stay usable.

Tolerances (relative to the largest value): FP64 1e-13 (three 1-D stages of <= 7 terms);
FP32 5e-6 (the same stages in FP32 on O(1) values).
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import fe
from oracle import twogrid as tg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import __graft_entry__ as ge
    ge.build()
    import paper_2410_02754_gb300 as pkg
    return pkg


def contexts(g, base, pf, prec):
    cc, cf = g.Context(0), g.Context(0)
    cc.set_problem(base)
    cf.set_mesh(base.ncell, base.h, pf, pf + 2, base.periodic)
    cc.set_precision(prec)
    cf.set_precision(prec)
    return cc, cf


CASES = [(2, 3, (1, 1, 1), 0), (3, 4, (1, 0, 1), 1), (4, 5, (0, 1, 0), 0), (5, 6, (1, 1, 0), 1),
         (6, 7, (0, 0, 1), 1), (3, 3, (1, 0, 0), 0), (6, 6, (1, 1, 1), 1)]


@pytest.mark.parametrize("pc,pf,per,prec", CASES)
def test_prolongate_matches_oracle(g, pc, pf, per, prec):
    base = syn.make_problem(ncell=(2, 2, 3), h=(1.0, 0.9, 1.2), p=pc, natoms=0, seed=5 + pc,
                            periodic=per)
    dc = fe.Discretisation(base)
    df = fe.Discretisation(base.with_(p=pf, nq=pf + 2))
    nv, ldc, ldf = 19, 21, 20
    Xc = syn.random_block(dc.mesh.nnodes, nv, 30 + pc)
    ref = tg.prolongate(dc, df, Xc)
    dt = torch.complex128 if prec == 0 else torch.complex64
    xc = torch.full((dc.mesh.nnodes, 2, ldc), complex(float("nan"), float("nan")), dtype=dt)
    xc[:, :, :nv] = torch.from_numpy(Xc).to(dt)
    xf = torch.full((df.mesh.nnodes, 2, ldf), complex(7.0, -7.0), dtype=dt)
    xc, xf = xc.cuda(), xf.cuda()
    cc, cf = contexts(g, base, pf, prec)
    cf.prolongate_from(cc, xc, xf, nvec=nv)
    torch.cuda.synchronize()
    out = xf.cpu().numpy().astype(np.complex128)
    tol = 1e-13 if prec == 0 else 5e-6
    np.testing.assert_allclose(out[:, :, :nv], ref, rtol=0, atol=tol * np.abs(ref).max())
    assert np.all(out[:, :, nv:] == complex(7.0, -7.0))
    if pc == pf and prec == 0:
        assert np.array_equal(out[:, :, :nv], Xc)          # p -> p is the identity, bit for bit
    cc.close()
    cf.close()


def test_prolongate_full_mesh_sampled_cells(g):
    base = syn.config("cube16_p6", kindex=1).with_(p=5, nq=7, atoms=[])
    E = base.ncells
    z = np.zeros((E, 7 ** 3))
    base = base.with_(veff=z, bx=z, by=z, bz=z)
    dc = fe.Discretisation(base)
    df = fe.Discretisation(base.with_(p=6, nq=8))
    Xc = syn.random_block(dc.mesh.nnodes, 32, 41)
    cells = np.unique(np.concatenate([[0, E - 1], np.random.default_rng(2).integers(0, E, 14)]))
    ref = tg.prolongate(dc, df, Xc, cells=cells)
    nodes = np.unique(np.concatenate([df.mesh.cell_nodes[e] for e in cells]))
    nodes = nodes[nodes >= 0]
    cc, cf = contexts(g, base, 6, 1)
    xc = torch.from_numpy(Xc).to(torch.complex64).cuda()
    xf = torch.empty((df.mesh.nnodes, 2, 32), dtype=torch.complex64, device="cuda")
    cf.prolongate_from(cc, xc, xf)
    torch.cuda.synchronize()
    out = xf.cpu().numpy().astype(np.complex128)[nodes]
    np.testing.assert_allclose(out, ref[nodes], rtol=0, atol=5e-6 * np.abs(ref[nodes]).max())
    cc.close()
    cf.close()


def test_prolongate_argument_errors(g):
    base = syn.make_problem(ncell=(2, 2, 2), p=3, natoms=0, seed=1)
    cc, cf = contexts(g, base, 4, 0)
    xc = torch.zeros((base.nnodes, 2, 4), dtype=torch.complex128, device="cuda")
    mf = fe.Discretisation(base.with_(p=4, nq=6)).mesh.nnodes
    xf = torch.zeros((mf, 2, 4), dtype=torch.complex128, device="cuda")
    with pytest.raises(g.GbcError):
        cf.prolongate_from(cc, xc, xf, nvec=5)               # nvec > ldx
    # the C checks run before any launch; the raw call bypasses the binding's shape checks
    bad = g.Context(0)
    bad.set_mesh((2, 2, 3), base.h, 4, 6, base.periodic)  # another mesh
    far = g.Context(0)
    far.set_mesh(base.ncell, base.h, 5, 7, base.periodic)  # p -> p + 2
    for fine in (bad, far):
        st = fine.lib.gbc_prolongate(cc.h, fine.h, xc.data_ptr(), 4, xf.data_ptr(), 4, 4, None)
        with pytest.raises(g.GbcError):
            fine._chk(st)
    cf.prolongate_from(cc, xc, xf)                           # still usable
    torch.cuda.synchronize()
    assert not xf.abs().max().item()
    for c in (cc, cf, bad, far):
        c.close()
