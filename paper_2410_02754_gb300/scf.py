"""Self-consistent-field loop around the eigensolver (Sec. III.B.1) over k-points.

Every numerical step runs in the library: the fields from the densities
(``gbc_scf_fields``: V_eff = V_ext + V_xc, B_xc, with the closed-form exchange
stand-in), one ChFSI cycle per SCF step on the block carried over
(``gbc_lanczos_bounds``, ``gbc_filter``, ``gbc_cholgs``, ``gbc_rayleigh_ritz``),
Fermi-Dirac occupations of the Ritz values (``gbc_fermi_occupations``), the
output densities (``gbc_density_dev``) and Anderson mixing
(``gbc_anderson_mix``).  Over k-points the occupations share one chemical
potential and the densities are Brillouin-zone sums, through ``kpoints``
(whose collectives join k-points sharded over ranks).  This module only
sequences the calls and holds the device buffers of the mixing history.
"""
from __future__ import annotations

import numpy as np


def scf_loop(ctx, X, vext, v0, nelec, kT, degree, lanczos_steps, alpha=0.5, nhist=4, iters=20,
             tol=0.0):
    """Run up to ``iters`` SCF steps on one context (one k-point of weight 1).

    ctx: a Context whose fields are V_ext with B = 0 on entry (the first block comes
    from CholGS + Rayleigh-Ritz of X under H[V_ext]); X: its block [M, 2, nvec] on the
    device, updated in place; vext: float64 CUDA tensor [E, nq^3]; v0: the Lanczos
    start vector (complex128 CUDA tensor [M, 2]).  Stops early once the residual norm
    || F(x) - x || (Eq. innerPdt) is <= tol.  Returns a dict with the residual norms,
    the final input densities [E, 4, nq^3] and the final Ritz values."""
    out = scf_loop_k([ctx], [X], vext, [v0], [1.0], nelec, kT, degree, lanczos_steps, alpha,
                     nhist, iters, tol)
    out["ritz"] = out["ritz"][0]
    return out


def scf_loop_k(ctxs, Xs, vext, v0s, kweights, nelec, kT, degree, lanczos_steps, alpha=0.5,
               nhist=4, iters=20, tol=0.0, group=None):
    """SCF steps over k-points: ctxs, Xs, v0s, kweights are this rank's k-points (at
    least one).  With torch.distributed initialised, the other ranks' k-points enter
    through the common chemical potential and the Brillouin-zone sum of the densities
    (``kpoints.sharded_occupations`` / ``sharded_density``); every rank then holds the
    same densities and takes the same mixing step.  The fields are the same at every
    k-point.  Returns a dict with the residual norms, the final input densities and the
    final Ritz values of this rank's k-points [nk_local, nvec]."""
    import torch
    from . import kpoints
    if not ctxs or not (len(ctxs) == len(Xs) == len(v0s) == len(kweights)):
        raise ValueError("one context, block, start vector and weight per local k-point")
    c0 = ctxs[0]
    E, q = c0.ncells, c0.nq ** 3

    def new():
        return torch.empty((E, 4, q), dtype=torch.float64, device=Xs[0].device)

    def densities(ritz):
        occ, _ = kpoints.sharded_occupations(np.array(ritz), kweights, nelec, kT, group)
        out = new()
        kpoints.sharded_density(ctxs, Xs, occ, kweights, out, group)
        return out

    ritz = []
    for c, X in zip(ctxs, Xs):
        c.cholgs(X)
        ritz.append(np.asarray(c.rayleigh_ritz(X)))
    x_in = densities(ritz)
    xs, fs, res = [], [], []
    for _ in range(iters):
        for k, (c, X) in enumerate(zip(ctxs, Xs)):
            c.scf_fields(x_in, vext)
            lo, hi = c.lanczos_bounds(v0s[k], lanczos_steps)
            c.filter(X, degree, float(ritz[k][-1]), hi, min(lo, float(ritz[k][0])))
            c.cholgs(X)
            ritz[k] = np.asarray(c.rayleigh_ritz(X))
        x_out = densities(ritz)
        xs, fs = (xs + [x_in])[-nhist:], (fs + [x_out])[-nhist:]
        x_next = new()
        _, rn = c0.anderson_mix(xs, fs, alpha, x_next)
        res.append(rn)
        x_in = x_next
        if rn <= tol:
            break
    return {"res": np.array(res), "dens": x_in, "ritz": np.array(ritz)}
