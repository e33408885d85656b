"""Deterministic mode (gbc_set_deterministic): the FP64 cell apply assembled by a
fixed-order gather of per-cell results, the projection summed per chunk in order, the
energy's column dots and the Lanczos inner products summed block by block in order.
Two runs give identical bits; the results agree with the FP64 oracle and with the
default (atomic) mode to rounding."""
import numpy as np
import pytest

import synthetic as syn
from oracle import chfsi as oc
from oracle import fe

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import __graft_entry__ as ge
    ge.build()
    import paper_2410_02754_gb300 as pkg
    return pkg


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [
    # ncell, p, periodic, natoms, rc: periodic wrap with one cell in x, Dirichlet faces in z,
    # several 1024-node projection chunks per atom
    ((1, 3, 2), 3, (1, 1, 0), 2, 1.2),
    ((5, 4, 4), 4, (1, 1, 1), 3, 2.4),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-p{c[1]}-per{''.join(map(str, c[2]))}")
def test_deterministic_fp64_bits_and_parity(g, case):
    ncell, p, per, natoms, rc = case
    prob = syn.make_problem(ncell=ncell, h=(1.1, 1.0, 0.9), p=p, periodic=per, k=(0.1, -0.2, 0.05),
                            natoms=natoms, rc=rc, seed=41, channels=syn.SPD_CHANNELS)
    d = fe.Discretisation(prob)
    M = d.mesh.nnodes
    X = syn.random_block(M, 6, 3)
    w = np.linspace(0.2, 1.0, 6)
    bounds = (1.0, 90.0, -2.0)
    ref_h = d.apply_h(X)
    ref_f = oc.cheb_filter(d.apply_htilde, X, 4, *bounds)
    v0 = torch.from_numpy(syn.random_start(M, 2)).cuda()

    def run(det):
        c = g.Context(0)
        c.set_problem(prob)
        c.set_deterministic(det)
        assert c.deterministic() == det
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.empty_like(Xd)
        c.apply_h(Xd, Yd)
        Fd = Xd.clone()
        c.filter(Fd, 4, *bounds)
        GY = torch.empty_like(Xd)
        L, gV, gBx, gBy, gBz, gD = c.energy_grad(Xd, w, GY)
        GX = torch.empty_like(Xd)
        fV, *_ = c.filter_vjp(Xd, GY, GX, 4, *bounds, ckpt_every=2)
        lo, hi = c.lanczos_bounds(v0, 12)
        c.sync_status()
        out = dict(h=Yd.cpu().numpy(), f=Fd.cpu().numpy(), L=np.array([L]), gV=np.asarray(gV),
                   gD=np.asarray(gD), gx=GX.cpu().numpy(), fV=np.asarray(fV),
                   lz=np.array([lo, hi]))
        c.close()
        return out

    a, b, atomic = run(True), run(True), run(False)
    for k in a:
        assert np.array_equal(a[k], b[k]), f"{k}: deterministic runs differ"
    assert rel(a["h"], ref_h) < 1e-12
    assert rel(a["f"], ref_f) < 1e-11
    for k in a:
        assert rel(a[k], atomic[k]) < 1e-11, (k, rel(a[k], atomic[k]))
