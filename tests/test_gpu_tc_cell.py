"""The tensor-core cell apply -- the precision paths GBC_TF32 and GBC_BF16X3 of reading
R18, the cell products as tcgen05 GEMMs -- against the FP64 oracle, through the C ABI.

* H.X for orders p = 2..7, periodic and Dirichlet faces, k = 0 and k != 0, ragged vector
  counts (nvec < ldx): BF16x3 within 1e-5 relative (the FP32-path tolerance); single-pass
  TF32 (10 mantissa bits in every product) within 5e-3, its error reported;
* near convergence (reading R11): on the cube6_p4 mesh and block, six FP64 cycles then six
  with the low precision through the residual-split filter keep the lowest Ritz values
  within 1e-6 Ha of the converged FP64 chain.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import chfsi as oc
from oracle import fe

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TF32, BF16X3 = 2, 3


@pytest.fixture(scope="module")
def g():
    import __graft_entry__ as ge
    ge.build()
    import paper_2410_02754_gb300 as pkg
    return pkg


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [
    # ncell, p, periodic, k, natoms, nvec, ldx
    ((2, 2, 2), 2, (1, 1, 1), (0, 0, 0), 1, 3, 3),
    ((3, 2, 2), 3, (1, 1, 0), (0.1, -0.2, 0.3), 2, 5, 7),
    ((2, 3, 2), 4, (1, 1, 1), (0.2, 0.1, -0.1), 2, 9, 9),
    ((2, 2, 3), 5, (0, 1, 1), (0.0, 0.3, 0.0), 1, 4, 4),
    ((2, 2, 2), 6, (1, 1, 1), (0.05, 0.05, 0.05), 2, 6, 8),
    ((2, 2, 2), 7, (1, 0, 1), (0.1, 0.0, 0.2), 1, 2, 2),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"p{c[1]}-{c[0]}-per{c[2]}")
def test_tensor_core_apply_h(g, case, capsys):
    ncell, p, per, k, natoms, nvec, ldx = case
    prob = syn.make_problem(ncell=ncell, h=(1.1, 1.2, 1.3), p=p, periodic=per, k=k,
                            natoms=natoms, rc=1.2, seed=p, channels=((0.5, 0), (0.5, 1)))
    d = fe.Discretisation(prob)
    X = syn.random_block(d.mesh.nnodes, nvec, 11)
    ref = d.apply_h(X)
    errs = {}
    for prec, tol in ((BF16X3, 1e-5), (TF32, 5e-3)):
        ctx = g.Context(0)
        ctx.set_problem(prob)
        ctx.set_precision(prec)
        Xd = torch.zeros((d.mesh.nnodes, 2, ldx), dtype=torch.complex64, device="cuda")
        Xd[:, :, :nvec] = torch.from_numpy(X).to(torch.complex64).cuda()
        Yd = torch.full_like(Xd, 7.0)
        ctx.apply_h(Xd, Yd, nvec=nvec)
        ctx.sync_status()
        Y = Yd.cpu().numpy().astype(np.complex128)
        errs[prec] = rel(Y[:, :, :nvec], ref)
        assert errs[prec] < tol, (prec, errs[prec])
        ctx.close()
    with capsys.disabled():
        print(f"  p={p}: H.X relative error BF16x3 {errs[BF16X3]:.2e}, TF32 {errs[TF32]:.2e}")


NCYC, DEG, NLOW = 12, 20, 8     # cycles, filter degree, Ritz values compared


@pytest.fixture(scope="module")
def c0_fp64_chain(g):
    """cube6_p4 mesh and block, ChFSI in FP64 on the GPU (parity-tested against the oracle
    to 1e-12 on every step) at degree 20: the Ritz values after each of 12 cycles."""
    prob = syn.config("cube6_p4")
    c = syn.CONFIGS["cube6_p4"]
    d = fe.Discretisation(prob)
    M = d.mesh.nnodes
    X0 = syn.random_block(M, c["nvec"], 0)
    v0 = syn.random_start(M, 0)
    lmin, lmax = oc.lanczos_bounds(d.apply_htilde, d.md, v0, c["lanczos"])
    return prob, c, X0, lmin, lmax, run_chain(g, prob, c, X0, lmin, lmax, None, NCYC)


def run_chain(g, prob, c, X0, lmin, lmax, prec, cycles, low_from=0):
    """cycle 0 + ``cycles`` x (filter, CholGS, Rayleigh-Ritz); cycles >= low_from in
    ``prec`` with the residual-split filter (FP64 throughout when prec is None)."""
    ctx = g.Context(0)
    ctx.set_problem(prob)
    ctx.set_precision(0)
    Xd = torch.from_numpy(X0).cuda()
    ctx.cholgs(Xd)
    ritz = ctx.rayleigh_ritz(Xd)
    out = []
    for cyc in range(cycles):
        low = prec is not None and cyc >= low_from
        if low and Xd.dtype != torch.complex64:
            ctx.set_precision(prec)
            Xd = Xd.to(torch.complex64)
        args = (Xd, DEG, float(ritz[-1]), lmax, min(lmin, float(ritz[0])))
        if low:
            ctx.filter_residual(*args, ritz)
        else:
            ctx.filter(*args)
        ctx.cholgs(Xd)
        ritz = ctx.rayleigh_ritz(Xd)
        out.append(np.array(ritz))
    ctx.sync_status()
    ctx.close()
    return out


@pytest.mark.parametrize("prec", [BF16X3, TF32])
def test_tensor_core_ritz_values_near_convergence(g, c0_fp64_chain, prec, capsys):
    """Reading R11: the low-precision filter enters through the residual split, whose error
    is ~ eps_low ||R||^2, small once the block is near convergence.  On the cube6_p4 mesh
    and block (degree 20) the first six cycles run in FP64 and the last six with the
    tensor-core cell apply and the residual-split filter: the lowest 8 Ritz values stay
    within 1e-6 Ha of the FP64 chain's after the same twelve cycles (which have converged
    to 1e-8).  The same run with every cycle in the low precision is printed beside it."""
    prob, c, X0, lmin, lmax, ref = c0_fp64_chain
    assert np.abs(ref[-1] - ref[-2])[:NLOW].max() < 1e-8      # the reference has converged
    late = run_chain(g, prob, c, X0, lmin, lmax, prec, NCYC, low_from=NCYC // 2)
    full = run_chain(g, prob, c, X0, lmin, lmax, prec, NCYC, low_from=0)
    err_late = np.abs(late[-1] - ref[-1])[:NLOW].max()
    err_full = np.abs(full[-1] - ref[-1])[:NLOW].max()
    with capsys.disabled():
        print(f"  precision {prec}: lowest {NLOW} Ritz values after {NCYC} cycles: error "
              f"{err_late:.2e} Ha with the last {NCYC // 2} cycles in it, {err_full:.2e} Ha with "
              f"every cycle in it")
    assert err_late < 1e-6, err_late
