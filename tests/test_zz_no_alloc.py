"""gbc_apply_h_noalloc: H.X for callers that cannot let the library allocate
device memory (applications that own all device memory through their own
pool, or must not trigger cudaMalloc's device-wide synchronisation).

Its output must match gbc_apply_h's on two calls in a row (the fixed scratch
array keeps the previous call's contents, so the second call checks that the
kernels clear it), for FP64 and for FP32 with both nonlocal engines (the
SIMT kernels and the tcgen05 projector contractions, whose bounded waits must
not have expired).  Oversized requests and host pointers must be refused.
The file sorts last so that a run stopping at the first failure has run
every other GPU test first; each test also runs on its own."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import __graft_entry__ as ge
    ge.build()
    import paper_2410_02754_gb300 as pkg
    return pkg


def _dev(X, prec):
    dt = torch.complex128 if prec == 0 else torch.complex64
    return torch.from_numpy(X).to(dt).cuda()


@pytest.mark.parametrize("prec,engine,nvec,tol", [(0, 0, 6, 1e-12), (1, 0, 6, 1e-5),
                                                  (1, 1, 32, 1e-5)])
def test_noalloc_matches_apply_h_on_two_calls(g, prec, engine, nvec, tol):
    prob = syn.make_problem(ncell=(3, 2, 2), h=(1.1, 1.2, 1.3), p=4, k=(0.1, -0.2, 0.05),
                            natoms=3, rc=1.2, seed=8, channels=((0.5, 0), (0.5, 1)))
    ctx = g.Context(0)
    ctx.set_problem(prob)
    ctx.set_precision(prec)
    if prec == 1:
        ctx.set_nonlocal_engine(engine)
        assert ctx.nonlocal_engine() == engine
    X = _dev(syn.random_block(ctx.nnodes, nvec, 2), prec)
    Yref = torch.empty_like(X)
    ctx.apply_h(X, Yref)                   # existing entry point (builds the tables)
    ctx.sync_status()
    ref = Yref.cpu().numpy()
    for _ in range(2):
        Y = torch.full_like(X, 3.0)
        ctx.apply_h_noalloc(X, Y)
        ctx.sync_status()                  # raises if a tensor-core wait expired
        got = Y.cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol
    ctx.close()


def test_noalloc_refuses_oversized_scratch_and_host_memory(g):
    prob = syn.make_problem(ncell=(2, 2, 2), h=(1.0, 1.0, 1.0), p=2, natoms=3, rc=1.2, seed=9)
    ctx = g.Context(0)
    ctx.set_problem(prob)
    X = _dev(syn.random_block(ctx.nnodes, 1, 2), 0)
    Y = torch.empty_like(X)
    ctx.apply_h(X, Y)
    nvec = 60000                           # 2 * 18 rows * 60000 * 16 B > 32 MiB
    Xb = torch.zeros((ctx.nnodes, 2, nvec), dtype=torch.complex128, device="cuda")
    Yb = torch.zeros_like(Xb)
    with pytest.raises(g.GbcError) as ei:
        ctx.apply_h_noalloc(Xb, Yb)
    assert ei.value.status == 1 and "exceeds the fixed scratch" in str(ei.value)
    del Xb, Yb
    # a host array where device memory is required is refused before any launch
    Xh = np.zeros((ctx.nnodes, 2, 1), np.complex128)
    st = ctx.lib.gbc_apply_h_noalloc(ctx.h, Xh.ctypes.data, Y.data_ptr(), 1, 1, None)
    assert st == 1
    ctx.apply_h_noalloc(X, Y)              # the context stays usable
    torch.cuda.synchronize()
    ctx.close()
