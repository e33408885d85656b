"""The package's SCF driver over k-points sharded on two gloo ranks (CPU), three k-points
split 2 + 1, against the oracle's single-process loop over all of them.  The library
context is replaced by a stand-in that does each step with the oracle (same method names),
so the test covers the driver's sequencing, the common chemical potential, the
Brillouin-zone sum and identical mixing on every rank -- not the kernels.  The ranks sum
the densities in another order than the single process, and the filter amplifies rounding
differences across steps: agreement to 1e-7 (residuals) and 1e-8 (densities)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

KW = [0.25, 0.25, 0.5]
KS = [(0.3, 0.0, 0.0), (-0.2, 0.4, 0.1), (0.0, 0.0, 0.5)]
SPLIT = [(0, 2), (2, 3)]
ARGS = dict(nelec=3.0, kT=0.05, degree=16, lanczos_steps=12, alpha=0.5, nhist=4, iters=8)


def _problem(k):
    import synthetic as syn
    z = np.zeros((8, 4 ** 3))
    return syn.make_problem(ncell=(2, 2, 2), h=(1.0, 1.0, 1.0), p=2, k=k, natoms=2, rc=1.0,
                            seed=9, well_depth=3.0, bmax=0.0).with_(bx=z, by=z, bz=z)


class OracleCtx:
    """Stand-in for a library context: every step done by the oracle on CPU tensors."""

    def __init__(self, prob):
        from oracle import fe
        self.prob, self.fe = prob, fe
        self.d = fe.Discretisation(prob)
        self.md = self.d.md
        self.ncells, self.nq = prob.ncells, prob.nq

    def _ht(self, Z):
        return self.d.apply_h(Z) / self.md[:, None, None]

    def cholgs(self, X):
        from oracle import chfsi as oc
        X.copy_(torch.from_numpy(oc.cholgs(X.numpy(), self.md)))

    def rayleigh_ritz(self, X):
        from oracle import chfsi as oc
        w, Xn, _ = oc.rayleigh_ritz(self.d.apply_h, X.numpy())
        X.copy_(torch.from_numpy(Xn))
        return w

    def scf_fields(self, dens, vext):
        from oracle import scf
        x = dens.numpy()
        _, V, B = scf.lsda_exchange(x[:, 0], np.moveaxis(x[:, 1:], 1, 0))
        self.d = self.fe.Discretisation(self.prob.with_(veff=vext.numpy() + V, bx=B[0], by=B[1],
                                                        bz=B[2]))

    def lanczos_bounds(self, v0, steps):
        from oracle import chfsi as oc
        return oc.lanczos_bounds(self._ht, self.md, v0.numpy(), steps)

    def filter(self, X, degree, lT, lmax, lmin):
        from oracle import chfsi as oc
        X.copy_(torch.from_numpy(oc.cheb_filter(self._ht, X.numpy(), degree, lT, lmax, lmin)))

    def density_dev(self, X, occ, out, nvec=None, accumulate=False):
        from oracle import density as od
        r, m = od.densities(self.d, X.numpy(), occ.numpy())
        val = torch.from_numpy(np.concatenate([r[:, None], np.moveaxis(m, 0, 1)], 1))
        if accumulate:
            out += val
        else:
            out.copy_(val)

    def anderson_mix(self, xs, fs, alpha, xnext):
        from oracle import scf
        W = self.d.tab.W
        xn, b = scf.anderson(W, [x.numpy() for x in xs], [f.numpy() - x.numpy()
                                                         for x, f in zip(xs, fs)], alpha)
        xnext.copy_(torch.from_numpy(xn))
        r = fs[-1].numpy() - xs[-1].numpy()
        return b, float(np.sqrt(scf.inner(W, r, r)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _inputs():
    import synthetic as syn
    probs = [_problem(k) for k in KS]
    M = probs[0].nnodes
    return (probs, [syn.random_block(M, 12, 3 + i) for i in range(3)],
            [syn.random_start(M, 3 + i) for i in range(3)])


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2410_02754_gb300 import scf
        probs, X0s, v0s = _inputs()
        a, b = SPLIT[rank]
        ctxs = [OracleCtx(p) for p in probs[a:b]]
        Xs = [torch.from_numpy(X.copy()) for X in X0s[a:b]]
        v0 = [torch.from_numpy(v) for v in v0s[a:b]]
        vext = torch.from_numpy(np.ascontiguousarray(probs[0].veff))
        out = scf.scf_loop_k(ctxs, Xs, vext, v0, KW[a:b], **ARGS)
        q.put((rank, out["res"], out["dens"].numpy(), out["ritz"]))
    except Exception as exc:          # report instead of leaving the parent waiting
        q.put((rank, None, repr(exc), None))
    finally:
        dist.destroy_process_group()


def test_sharded_scf_matches_single_process_oracle():
    import __graft_entry__ as ge
    ge.build()
    from oracle import scf as osc
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, qu)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((qu.get(timeout=600) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    probs, X0s, v0s = _inputs()
    r_o, x_o, e_o = osc.scf_loop_k(probs, X0s, v0s, KW, **ARGS)
    for rank, r, x, e in res:
        assert r is not None, f"rank {rank}: {x}"
        a, b = SPLIT[rank]
        np.testing.assert_allclose(r, r_o, rtol=1e-7)
        np.testing.assert_allclose(x, x_o, rtol=0, atol=1e-8 * np.abs(x_o).max())
        np.testing.assert_allclose(e[:, :3], e_o[a:b, :3], rtol=0, atol=1e-9)
    assert np.array_equal(res[0][2], res[1][2])           # identical densities on both ranks
