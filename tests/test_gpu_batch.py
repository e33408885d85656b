"""Batched filtering of uneven systems (one persistent cell-apply launch per
group, CUDA-graph replay) and the tile autotuner, against the FP64 oracle."""
import numpy as np
import pytest

import synthetic as syn
from oracle import chfsi as oc
from oracle import fe

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SYSTEMS = [
    # ncell, p, k, natoms, nvec, ldx, degree, bounds (lT, lmax, lmin)
    ((2, 2, 3), 3, (0.0, 0.0, 0.0), 1, 5, 5, 4, (1.0, 60.0, -2.0)),
    ((3, 2, 2), 3, (0.0, 0.0, 0.0), 2, 3, 4, 7, (0.5, 70.0, -1.5)),
    ((2, 2, 2), 4, (0.1, 0.0, -0.1), 2, 6, 6, 5, (2.0, 90.0, -3.0)),
    ((3, 3, 2), 2, (0.0, 0.0, 0.0), 1, 4, 6, 1, (1.0, 40.0, -1.0)),
]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def g():
    import __graft_entry__ as ge
    ge.build()
    import paper_2410_02754_gb300 as pkg
    return pkg


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-5)])
def test_batch_filter_matches_oracle_and_replays(g, prec, tol):
    dt = torch.complex128 if prec == 0 else torch.complex64
    probs, ctxs, discs = [], [], []
    for i, (nc, p, k, na, nv, ld, m, b) in enumerate(SYSTEMS):
        prob = syn.make_problem(ncell=nc, h=(1.1, 1.1, 1.1), p=p, k=k, natoms=na, rc=1.2, seed=20 + i)
        c = g.Context(0)
        c.set_problem(prob)
        c.set_precision(prec)
        probs.append(prob)
        ctxs.append(c)
        discs.append(fe.Discretisation(prob))
    batch = g.Batch(ctxs)
    stream = torch.cuda.Stream()
    for call in range(2):                    # second call replays the captured graph
        Xs, refs = [], []
        for i, (nc, p, k, na, nv, ld, m, b) in enumerate(SYSTEMS):
            X = syn.random_block(discs[i].mesh.nnodes, nv, 100 * call + i)
            refs.append(oc.cheb_filter(discs[i].apply_htilde, X, m, *b))
            Xd = torch.zeros((X.shape[0], 2, ld), dtype=dt, device="cuda")
            Xd[:, :, :nv] = torch.from_numpy(X).to(dt).cuda()
            Xs.append(Xd)
        if call == 0:
            bufs = Xs
        else:                                # same buffers, new contents
            for dst, src in zip(bufs, Xs):
                dst.copy_(src)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            batch.filter(bufs, [s[6] for s in SYSTEMS], [s[7] for s in SYSTEMS], stream)
        stream.synchronize()
        for i, s in enumerate(SYSTEMS):
            got = bufs[i].cpu().numpy()[:, :, :s[4]]
            assert rel(got, refs[i]) < tol, (call, i, rel(got, refs[i]))
    assert batch.launches() > 0
    batch.close()
    for c in ctxs:
        c.close()


def test_tuner_picks_a_tile_and_keeps_parity(g):
    prob = syn.make_problem(ncell=(3, 3, 2), h=(1.0, 1.0, 1.0), p=5, k=(0.1, 0.0, 0.0), natoms=2,
                            rc=1.2, seed=5)
    d = fe.Discretisation(prob)
    c = g.Context(0)
    c.set_problem(prob)
    c.set_precision(1)
    vb = c.tune(8)
    assert vb in (1, 2)
    X = syn.random_block(d.mesh.nnodes, 8, 3)
    Xd = torch.from_numpy(X).to(torch.complex64).cuda()
    Yd = torch.empty_like(Xd)
    c.apply_h(Xd, Yd)
    torch.cuda.synchronize()
    assert rel(Yd.cpu().numpy(), d.apply_h(X)) < 1e-5
    assert c.tune(8) == vb                   # cached
    c.close()
