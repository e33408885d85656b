"""SCF steps on the GPU (gbc_scf_fields, gbc_anderson_mix and the package's scf_loop)
against the FP64 oracle.

* fields: the H.X of the context after gbc_scf_fields equals the oracle's apply of H with
  V_eff = V_ext + V_xc and B_xc from the same densities (exchange stand-in), and the energy
  density matches;
* Anderson mixing: coefficients, mixed densities and the residual norm for 1..5 history
  pairs, and the singular case;
* the loop: residual history and the converged densities of a small two-atom problem
  (one ChFSI cycle per SCF step) equal the oracle loop's.
FP64 throughout; tolerances 1e-12 relative for the pointwise steps, 1e-6 on the residual
history (each step goes through a full eigensolver cycle) and 1e-7 on the converged
densities.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import fe
from oracle import scf as osc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import __graft_entry__ as ge
    ge.build()
    import paper_2410_02754_gb300 as pkg
    return pkg


def rand_dens(E, q, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.05, 1.5, (E, q))
    m = rng.normal(size=(3, E, q))
    m *= (rng.uniform(0.0, 0.9, (E, q)) * rho / np.sqrt((m * m).sum(0)))[None]
    m[:, 0, :3] = 0.0                                     # a few unpolarised points
    # [E, 4, q] in C order: the binding takes contiguous device arrays only
    return np.ascontiguousarray(np.concatenate([rho[:, None], np.moveaxis(m, 0, 1)], 1))


def test_scf_fields_match_oracle(g):
    prob = syn.make_problem(ncell=(2, 2, 3), h=(1.0, 1.1, 0.9), p=3, k=(0.1, 0.0, -0.2),
                            natoms=1, rc=1.0, seed=3, bmax=0.0)
    E, q = prob.ncells, prob.nq ** 3
    x = rand_dens(E, q, 4)
    e_o, V, B = osc.lsda_exchange(x[:, 0], np.moveaxis(x[:, 1:], 1, 0))
    d = fe.Discretisation(prob.with_(veff=prob.veff + V, bx=B[0], by=B[1], bz=B[2]))
    X = syn.random_block(d.mesh.nnodes, 3, 5)
    ref = d.apply_h(X)
    c = g.Context(0)
    c.set_problem(prob)
    dens = torch.from_numpy(x).cuda()
    vext = torch.from_numpy(np.ascontiguousarray(prob.veff)).cuda()
    exc = torch.empty((E, q), dtype=torch.float64, device="cuda")
    c.scf_fields(dens, vext, exc)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.empty_like(Xd)
    c.apply_h(Xd, Yd)
    torch.cuda.synchronize()
    out = Yd.cpu().numpy()
    assert np.linalg.norm(out - ref) < 1e-12 * np.linalg.norm(ref)
    np.testing.assert_allclose(exc.cpu().numpy(), e_o, rtol=1e-13, atol=1e-15)
    c.close()


@pytest.mark.parametrize("n", [1, 2, 5])
def test_anderson_mix_matches_oracle(g, n):
    prob = syn.make_problem(ncell=(2, 3, 2), h=(1.2, 0.9, 1.0), p=2, natoms=0, seed=6)
    d = fe.Discretisation(prob)
    E, q = prob.ncells, prob.nq ** 3
    xs = [rand_dens(E, q, 10 + j) for j in range(n)]
    fs = [rand_dens(E, q, 20 + j) for j in range(n)]
    x_o, b_o = osc.anderson(d.tab.W, xs, [f - x for x, f in zip(xs, fs)], 0.4)
    rn_o = np.sqrt(osc.inner(d.tab.W, fs[-1] - xs[-1], fs[-1] - xs[-1]))
    c = g.Context(0)
    c.set_problem(prob)
    xin = [torch.from_numpy(x).cuda() for x in xs]
    xout = [torch.from_numpy(f).cuda() for f in fs]
    nxt = torch.empty_like(xin[0])
    b, rn = c.anderson_mix(xin, xout, 0.4, nxt)
    np.testing.assert_allclose(b, b_o, rtol=1e-10, atol=1e-12)
    assert abs(rn - rn_o) < 1e-12 * rn_o
    np.testing.assert_allclose(nxt.cpu().numpy(), x_o, rtol=0, atol=1e-12 * np.abs(x_o).max())
    # the result may overwrite the oldest input
    b2, _ = c.anderson_mix(xin, xout, 0.4, xin[0])
    np.testing.assert_allclose(xin[0].cpu().numpy(), x_o, rtol=0, atol=1e-12 * np.abs(x_o).max())
    # repeated pairs make the residual Gram matrix singular
    if n == 1:
        with pytest.raises(g.GbcError):
            c.anderson_mix([xin[0], xin[0]], [xout[0], xout[0]], 0.4, nxt)
        with pytest.raises(g.GbcError):
            c.anderson_mix(xin, xout, 0.0, nxt)                 # alpha must be > 0
    c.close()


def test_scf_loop_matches_oracle(g):
    from paper_2410_02754_gb300 import scf
    z = np.zeros((8, 4 ** 3))
    prob = syn.make_problem(ncell=(2, 2, 2), h=(1.0, 1.0, 1.0), p=2, natoms=2, rc=1.0, seed=9,
                            well_depth=3.0, bmax=0.0).with_(bx=z, by=z, bz=z)
    M = prob.nnodes
    X0 = syn.random_block(M, 12, 3)
    v0 = syn.random_start(M, 3)
    args = dict(nelec=3.0, kT=0.05, degree=16, lanczos_steps=12, alpha=0.5, nhist=4, iters=30)
    r_o, x_o, e_o = osc.scf_loop(prob, X0, v0, eig="chfsi", **args)
    c = g.Context(0)
    c.set_problem(prob)
    X = torch.from_numpy(X0).cuda()
    out = scf.scf_loop(c, X, torch.from_numpy(np.ascontiguousarray(prob.veff)).cuda(),
                       torch.from_numpy(v0).cuda(), **args)
    np.testing.assert_allclose(out["res"][:8], r_o[:8], rtol=1e-6)
    assert out["res"][-1] < 1e-7 * out["res"][0]
    np.testing.assert_allclose(out["dens"].cpu().numpy(), x_o, rtol=0, atol=1e-7 * np.abs(x_o).max())
    np.testing.assert_allclose(out["ritz"][:3], e_o[:3], rtol=0, atol=1e-8)
    c.close()


def test_scf_loop_two_kpoints_matches_oracle(g):
    """Two k-points in one process: common chemical potential, Brillouin-zone-summed
    densities (accumulate mode), the same fields at both k-points."""
    from paper_2410_02754_gb300 import scf
    z = np.zeros((8, 4 ** 3))
    probs = [syn.make_problem(ncell=(2, 2, 2), h=(1.0, 1.0, 1.0), p=2, k=k, natoms=2, rc=1.0,
                              seed=9, well_depth=3.0, bmax=0.0).with_(bx=z, by=z, bz=z)
             for k in ((0.3, 0.0, 0.0), (-0.2, 0.4, 0.1))]
    M = probs[0].nnodes
    X0s = [syn.random_block(M, 12, 3 + i) for i in range(2)]
    v0s = [syn.random_start(M, 3 + i) for i in range(2)]
    args = dict(nelec=3.0, kT=0.05, degree=16, lanczos_steps=12, alpha=0.5, nhist=4, iters=20)
    r_o, x_o, e_o = osc.scf_loop_k(probs, X0s, v0s, [0.5, 0.5], **args)
    ctxs = []
    for p in probs:
        c = g.Context(0)
        c.set_problem(p)
        ctxs.append(c)
    out = scf.scf_loop_k(ctxs, [torch.from_numpy(X).cuda() for X in X0s],
                         torch.from_numpy(np.ascontiguousarray(probs[0].veff)).cuda(),
                         [torch.from_numpy(v).cuda() for v in v0s], [0.5, 0.5], **args)
    np.testing.assert_allclose(out["res"][:8], r_o[:8], rtol=1e-6)
    np.testing.assert_allclose(out["dens"].cpu().numpy(), x_o, rtol=0, atol=1e-7 * np.abs(x_o).max())
    np.testing.assert_allclose(out["ritz"][:, :3], e_o[:, :3], rtol=0, atol=1e-8)
    for c in ctxs:
        c.close()
