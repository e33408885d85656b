"""k-point sharding of the occupations and densities on CPU with the gloo backend,
world size 2 and an uneven split of five k-points (3 + 2): the chemical potential and
the occupations of every rank equal the oracle's on the full set, and the all-reduced
density equals the single-process Brillouin-zone sum.  The density kernel is replaced
by a host fake with the same accumulate contract (out += sum_n occ_n * unit_k), so the
test covers the k-weight folding, the ordering and the collective, not the kernel."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

KT = 500.0 * 3.166811563e-6
NK, NS, NELEC = 5, 12, 7.3
SPLIT = [(0, 3), (3, 5)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem():
    rng = np.random.default_rng(11)
    eps = np.sort(rng.uniform(-0.6, 1.2, (NK, NS)), axis=1)
    w = rng.uniform(0.5, 1.5, NK)
    w /= w.sum()
    units = rng.normal(size=(NK, 3, 4, 8))          # fake per-k density "units" [E, 4, q]
    return eps, w, units


class FakeCtx:
    def __init__(self, unit):
        self.unit = torch.from_numpy(unit)

    def density_dev(self, X, occ, out, nvec=None, accumulate=False):
        assert accumulate and occ.dtype == torch.float64 and occ.numel() == nvec
        out += occ.sum() * self.unit


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2410_02754_gb300 import kpoints
        eps, w, units = _problem()
        a, b = SPLIT[rank]
        occ, mu = kpoints.sharded_occupations(eps[a:b], w[a:b], NELEC, KT)
        out = torch.empty(3, 4, 8, dtype=torch.float64)
        kpoints.sharded_density([FakeCtx(u) for u in units[a:b]], [None] * (b - a), occ, w[a:b],
                                out)
        q.put((rank, occ, mu, out.numpy()))
    except Exception as exc:          # report instead of leaving the parent waiting
        q.put((rank, None, repr(exc), None))
    finally:
        dist.destroy_process_group()


def test_sharded_occupations_and_density():
    import __graft_entry__ as ge
    ge.build()
    from oracle import density as od
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    eps, w, units = _problem()
    f_o, mu_o = od.fermi_occupations(eps, w, NELEC, KT)
    expect = np.einsum("k,kn,keq->eq", w, f_o, units.reshape(NK, 3, -1)).reshape(3, 4, 8)
    for rank, occ, mu, out in res:
        assert occ is not None, f"rank {rank}: {mu}"
        a, b = SPLIT[rank]
        assert abs(mu - mu_o) < 1e-12
        np.testing.assert_allclose(occ, f_o[a:b], rtol=0, atol=1e-12)
        np.testing.assert_allclose(out, expect, rtol=1e-13, atol=1e-13)
    assert res[0][2] == res[1][2]                    # bit-identical mu on both ranks


def test_single_process_is_the_plain_routine():
    import __graft_entry__ as ge
    ge.build()
    from paper_2410_02754_gb300 import fermi_occupations, kpoints
    eps, w, _ = _problem()
    occ, mu = kpoints.sharded_occupations(eps, w, NELEC, KT)
    occ2, mu2 = fermi_occupations(eps, w, NELEC, KT)
    assert mu == mu2 and np.array_equal(occ, occ2)
