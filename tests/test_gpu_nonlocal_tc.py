"""FP32 nonlocal step on the tcgen05 tensor cores (3xTF32) against the SIMT
engine and the FP64 oracle.

The cases exercise the projection over several 1024-node support chunks, the
expansion's atom slots (chunks of 128 owned nodes split when more than 16 atoms
touch them), K tiles that straddle slot boundaries (npj = 18 gives 36 reals a
slot), a single projector (N = 16), ragged and padded column tiles, and the
fallback to the SIMT engine when one node lies in more than 16 supports.
Blocks with ldx == nvec and at least 32 vectors take the TMA-fed projection
(tile::gather4 of X rows), the others the register-fed one.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import fe

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def g():
    import __graft_entry__ as ge
    ge.build()
    import paper_2410_02754_gb300 as pkg
    return pkg


def max_node_multiplicity(prob):
    """Largest number of atom supports sharing one free node (mesh geometry only)."""
    p = prob.p
    nx, ny, _ = prob.ncell
    n = [c * p if b else c * p - 1 for c, b in zip(prob.ncell, prob.periodic)]
    count = {}
    for a in prob.atoms:
        nodes = set()
        for e in a.supp_cell:
            cell = (e % nx, (e // nx) % ny, e // (nx * ny))
            axes = []
            for d in range(3):
                gidx = cell[d] * p + np.arange(p + 1)
                if prob.periodic[d]:
                    axes.append(gidx % n[d])
                else:
                    axes.append(gidx[(gidx > 0) & (gidx <= n[d])] - 1)
            I = (axes[2][:, None, None] * n[1] + axes[1][None, :, None]) * n[0] + axes[0][None, None, :]
            nodes.update(I.ravel().tolist())
        for I in nodes:
            count[I] = count.get(I, 0) + 1
    return max(count.values())


CASES = [
    # ncell, p, periodic, natoms, rc, channels, nvec, ldx
    ((4, 4, 4), 3, (1, 1, 1), 6, 2.0, "spd", 37, 40),       # 2 projection chunks per atom
    ((4, 4, 4), 3, (1, 1, 1), 6, 2.0, "spd", 48, 48),       # TMA-fed projection, ragged tiles
    ((6, 6, 6), 2, (1, 1, 1), 40, 0.8, "spd", 64, 64),      # many slot splits, mult 13
    ((3, 2, 3), 4, (1, 0, 1), 3, 1.2, "s", 5, 8),           # npj = 1, Dirichlet faces
    ((5, 5, 5), 2, (1, 1, 1), 40, 1.2, "spd", 9, 9),        # mult 30 > 16: SIMT fallback
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-p{c[1]}-a{c[3]}-{c[5]}-n{c[6]}")
def test_tensor_nonlocal_matches_simt_and_oracle(g, case):
    ncell, p, per, natoms, rc, ch, nvec, ldx = case
    channels = syn.SPD_CHANNELS if ch == "spd" else ((0.5, 0),)
    prob = syn.make_problem(ncell=ncell, h=(1.0, 1.0, 1.0), p=p, periodic=per,
                            k=(0.1, -0.05, 0.2), natoms=natoms, rc=rc, seed=7, channels=channels)
    d = fe.Discretisation(prob)
    X = syn.random_block(d.mesh.nnodes, nvec, 13)
    ref = d.apply_h(X)
    expect_tc = max_node_multiplicity(prob) <= 16
    out = {}
    for engine in (0, 1):
        ctx = g.Context(0)
        ctx.set_problem(prob)
        ctx.set_precision(1)
        ctx.set_nonlocal_engine(engine)
        assert ctx.nonlocal_engine() == (1 if engine == 1 and expect_tc else 0)
        Xd = torch.zeros((X.shape[0], 2, ldx), dtype=torch.complex64, device="cuda")
        Xd[:, :, :nvec] = torch.from_numpy(X).to(torch.complex64).cuda()
        Yd = torch.full_like(Xd, 3.0)
        ctx.apply_h(Xd, Yd, nvec=nvec)
        ctx.sync_status()
        out[engine] = Yd.cpu().numpy()
        ctx.close()
        err = rel(out[engine][:, :, :nvec].astype(np.complex128), ref)
        assert err < 1e-5, (engine, err)
    assert rel(out[1][:, :, :nvec], out[0][:, :, :nvec]) < 5e-6


def test_tensor_nonlocal_filter_and_engine_errors(g):
    """A degree-8 FP32 filter through the tensor engine agrees with the SIMT
    engine, gbc_sync_status reports no expired wait, and an unknown engine id is
    rejected."""
    prob = syn.make_problem(ncell=(4, 4, 4), h=(1.0, 1.0, 1.0), p=3, k=(0.0, 0.1, 0.0),
                            natoms=6, rc=2.0, seed=8, channels=syn.SPD_CHANNELS)
    X = syn.random_block(prob.nnodes, 16, 2)
    ctx = g.Context(0)
    ctx.set_problem(prob)
    lo, hi = ctx.lanczos_bounds(torch.from_numpy(syn.random_start(prob.nnodes, 1)).cuda(), 12)
    ctx.close()
    lmin, lT = lo - 0.5, lo + 4.0
    res = {}
    for engine in (0, 1):
        ctx = g.Context(0)
        ctx.set_problem(prob)
        ctx.set_precision(1)
        ctx.set_nonlocal_engine(engine)
        Xd = torch.from_numpy(X).to(torch.complex64).cuda()
        ctx.filter(Xd, 8, lT, hi, lmin)
        ctx.sync_status()
        res[engine] = Xd.cpu().numpy().astype(np.complex128)
        if engine == 1:
            assert ctx.nonlocal_engine() == 1
            with pytest.raises(g.GbcError):
                ctx.set_nonlocal_engine(2)
        ctx.close()
    assert rel(res[1], res[0]) < 1e-5


def test_tensor_nonlocal_long_chains_unbiased(g):
    """cube16_p6 atoms (19k-node supports: projection chains of 1024 nodes, 4-14
    expansion slots) with Delta scaled by 1e5 so that the nonlocal part dominates
    H X: (H X - H_loc X) from the FP32 tensor engine against the FP64 oracle's
    nonlocal apply.  The tensor core's accumulator truncates toward zero, which
    unmitigated scaled C = P^H X by about -5e-6 here; the check bounds both the
    relative error and its systematic part (the error's component along the
    exact result)."""
    import dataclasses
    prob = syn.config("cube16_p6", kindex=1)
    # at Delta x 1 the nonlocal part is ~2.5e-4 of the local one on random blocks
    prob = prob.with_(atoms=[dataclasses.replace(a, delta=a.delta * 1e5) for a in prob.atoms])
    d = fe.Discretisation(prob)
    X = syn.random_block(d.mesh.nnodes, 32, 21)   # 32 vectors: TMA-fed projection
    ref = d.apply_nonlocal(X)
    out = {}
    for name, p in (("full", prob), ("local", prob.with_(atoms=[]))):
        ctx = g.Context(0)
        ctx.set_problem(p)
        ctx.set_precision(1)
        if name == "full":
            assert ctx.nonlocal_engine() == 1
        Xd = torch.from_numpy(X).to(torch.complex64).cuda()
        Yd = torch.empty_like(Xd)
        ctx.apply_h(Xd, Yd)
        ctx.sync_status()
        out[name] = Yd.cpu().numpy().astype(np.complex128)
        ctx.close()
    nl = out["full"] - out["local"]
    err = nl - ref
    assert np.linalg.norm(out["local"]) < 0.1 * np.linalg.norm(ref)
    assert rel(nl, ref) < 3e-6, rel(nl, ref)
    scale = np.real(np.vdot(ref, err)) / np.real(np.vdot(ref, ref))
    assert abs(scale) < 1e-6, scale


def test_expired_device_wait_is_reported_and_context_recovers(g):
    """A bounded wait that runs out (an mbarrier nothing arrives at) is reported by
    gbc_sync_status as GBC_ETIMEOUT; the flag is then cleared and the tensor-core
    nonlocal step runs normally again on the same context."""
    from paper_2410_02754_gb300.gbchfsi import tc_wait_selftest
    prob = syn.make_problem(ncell=(4, 4, 4), h=(1.0, 1.0, 1.0), p=3, k=(0.1, 0.0, 0.0),
                            natoms=6, rc=2.0, seed=9, channels=syn.SPD_CHANNELS)
    X = syn.random_block(prob.nnodes, 32, 4)
    ref = fe.Discretisation(prob).apply_h(X)
    ctx = g.Context(0)
    ctx.set_problem(prob)
    ctx.set_precision(1)
    assert ctx.nonlocal_engine() == 1
    ctx.sync_status()
    tc_wait_selftest(1000)
    with pytest.raises(g.GbcError) as err:
        ctx.sync_status()
    assert err.value.status == 6   # GBC_ETIMEOUT
    ctx.sync_status()              # cleared
    Xd = torch.from_numpy(X).to(torch.complex64).cuda()
    Yd = torch.empty_like(Xd)
    ctx.apply_h(Xd, Yd)
    ctx.sync_status()
    assert rel(Yd.cpu().numpy().astype(np.complex128), ref) < 1e-5
    ctx.close()


FILTER_CASES = [
    # ncell, p, periodic, natoms, rc, channels, nvec  (ldx == nvec)
    ((4, 4, 4), 3, (1, 1, 1), 6, 2.0, "spd", 48),      # two column tiles, the second half full
    ((4, 4, 4), 3, (1, 1, 1), 6, 2.0, "spd", 37),      # last tile 20 real columns
    ((6, 6, 6), 2, (1, 1, 1), 40, 0.8, "spd", 64),     # many atoms per expansion chunk
    ((3, 2, 3), 4, (1, 0, 1), 3, 1.2, "s", 33),        # npj = 1, Dirichlet faces
]


@pytest.mark.parametrize("case", FILTER_CASES, ids=lambda c: f"{c[0]}-p{c[1]}-a{c[3]}-{c[5]}-n{c[6]}")
def test_packed_expansion_filter_matches_oracle(g, case):
    """The fused FP32 filter writes P C' into the accumulator with the expansion
    from packed operands (ldx == nvec, tensor engine): a degree-3 filter against
    the FP64 oracle's three-term recurrence and against the SIMT engine."""
    from oracle import chfsi as oc
    ncell, p, per, natoms, rc, ch, nvec = case
    channels = syn.SPD_CHANNELS if ch == "spd" else ((0.5, 0),)
    prob = syn.make_problem(ncell=ncell, h=(1.0, 1.0, 1.0), p=p, periodic=per,
                            k=(0.1, -0.05, 0.2), natoms=natoms, rc=rc, seed=9, channels=channels)
    d = fe.Discretisation(prob)
    X = syn.random_block(d.mesh.nnodes, nvec, 17)
    bounds = (1.0, 80.0, -2.0)
    ref = oc.cheb_filter(d.apply_htilde, X, 3, *bounds)
    out = {}
    for engine in (0, 1):
        ctx = g.Context(0)
        ctx.set_problem(prob)
        ctx.set_precision(1)
        ctx.set_nonlocal_engine(engine)
        assert ctx.nonlocal_engine() == engine
        Xd = torch.from_numpy(X).to(torch.complex64).cuda()
        ctx.filter(Xd, 3, *bounds)
        ctx.sync_status()
        out[engine] = Xd.cpu().numpy().astype(np.complex128)
        ctx.close()
        assert rel(out[engine], ref) < 2e-5, (engine, rel(out[engine], ref))
    assert rel(out[1], out[0]) < 1e-5
