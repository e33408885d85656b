"""Batched filtering of uneven systems (one persistent cell-apply launch per group of
systems sharing order, cell edges and k-point; CUDA-graph replay) and the cell-apply
autotuner, against the FP64 oracle."""
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


# a second p = 4 system at another k-point: two table groups of one order
EXTRA = ((2, 2, 2), 4, (0.0, 0.2, 0.0), 1, 4, 4, 3, (1.5, 80.0, -2.0))


@pytest.mark.parametrize("prec,tol,systems", [(0, 1e-11, SYSTEMS), (1, 2e-5, SYSTEMS),
                                              (1, 2e-5, SYSTEMS + [EXTRA])],
                         ids=["fp64", "fp32", "fp32-two-groups-one-order"])
def test_batch_filter_matches_oracle_and_replays(g, prec, tol, systems):
    dt = torch.complex128 if prec == 0 else torch.complex64
    probs, ctxs, discs = [], [], []
    for i, (nc, p, k, na, nv, ld, m, b) in enumerate(systems):
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
        for i, (nc, p, k, na, nv, ld, m, b) in enumerate(systems):
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
            batch.filter(bufs, [s[6] for s in systems], [s[7] for s in systems], stream)
        stream.synchronize()
        for i, s in enumerate(systems):
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
    var, vb2, nt = c.cell_variant()
    assert 0 <= var < 5 and vb2 == vb and (vb, nt) == ((4, 512) if var == 4 else (2, 256))
    X = syn.random_block(d.mesh.nnodes, 8, 3)
    Xd = torch.from_numpy(X).to(torch.complex64).cuda()
    Yd = torch.empty_like(Xd)
    c.apply_h(Xd, Yd)
    torch.cuda.synchronize()
    assert rel(Yd.cpu().numpy(), d.apply_h(X)) < 1e-5
    assert c.tune(8) == vb                   # cached
    c.close()


def test_tuner_json_cache_and_nonlocal_engine(g, tmp_path, monkeypatch):
    """The tuner's cache file is JSON: per key (device, FP32, p, k != 0, vector bucket) the
    chosen cell-apply variant and nonlocal engine with the measured times of every
    candidate; the context runs the chosen engine with parity kept."""
    import json
    path = tmp_path / "tune.json"
    monkeypatch.setenv("GBC_TUNE_CACHE", str(path))
    prob = syn.make_problem(ncell=(3, 3, 3), h=(1.0, 1.0, 1.0), p=4, k=(0.0, 0.1, 0.0), natoms=3,
                            rc=1.5, seed=12, channels=syn.SPD_CHANNELS)
    d = fe.Discretisation(prob)
    c = g.Context(0)
    c.set_problem(prob)
    c.set_precision(1)
    c.tune(40)                               # bucket nvec64: not tuned by the other tests
    data = json.loads(path.read_text())
    key = [k for k in data if k.endswith("/fp32/p4/k1/nvec64")]
    assert len(key) == 1, list(data)
    e = data[key[0]]
    assert e["variant"] == c.cell_variant()[0]
    assert e["nl_engine"] == c.nonlocal_engine() and e["nl_engine"] in (0, 1)
    assert len(e["ms"]) == 5 and min(e["ms"]) > 0 and len(e["nl_ms"]) == 2
    X = syn.random_block(d.mesh.nnodes, 40, 4)
    Xd = torch.from_numpy(X).to(torch.complex64).cuda()
    Yd = torch.empty_like(Xd)
    c.apply_h(Xd, Yd)
    c.sync_status()
    assert rel(Yd.cpu().numpy(), d.apply_h(X)) < 1e-5
    c.close()


VARIANT_CASES = [
    # ncell, p, k, nvec: every compiled order's largest tables at p = 6 and 7 (n_q = p + 2),
    # vector counts that leave a ragged last chunk of 2 and of 4 vectors
    ((2, 2, 2), 6, (0.1, -0.05, 0.2), 7),
    ((2, 2, 2), 6, (0.0, 0.0, 0.0), 5),
    ((3, 2, 2), 2, (0.2, 0.0, 0.0), 9),
    ((2, 1, 2), 7, (0.0, 0.1, 0.0), 6),
]


@pytest.mark.parametrize("var", range(5))
@pytest.mark.parametrize("case", VARIANT_CASES, ids=lambda c: f"p{c[1]}-k{int(any(c[2]))}-n{c[3]}")
def test_every_cell_variant_matches_oracle(g, var, case):
    """Each FP32 cell-apply variant (2 or 4 vectors per CTA), set explicitly, in both
    assembly modes: H X (accumulate) and a degree-3 filter (recurrence fused for the
    cell-interior rows) against the FP64 oracle."""
    ncell, p, k, nvec = case
    prob = syn.make_problem(ncell=ncell, h=(1.0, 1.0, 1.0), p=p, k=k, natoms=2, rc=1.2, seed=21)
    d = fe.Discretisation(prob)
    X = syn.random_block(d.mesh.nnodes, nvec, 8)
    c = g.Context(0)
    c.set_problem(prob)
    c.set_precision(1)
    c.set_cell_variant(var)
    v, vb, nt = c.cell_variant()
    assert v == var and (vb, nt) == ((4, 512) if var == 4 else (2, 256))
    Xd = torch.from_numpy(X).to(torch.complex64).cuda()
    Yd = torch.empty_like(Xd)
    c.apply_h(Xd, Yd)
    c.sync_status()
    assert rel(Yd.cpu().numpy(), d.apply_h(X)) < 1e-5
    bounds = (1.0, 80.0, -2.0)
    c.filter(Xd, 3, *bounds)
    c.sync_status()
    ref = oc.cheb_filter(d.apply_htilde, X, 3, *bounds)
    assert rel(Xd.cpu().numpy().astype(np.complex128), ref) < 2e-5
    c.close()
