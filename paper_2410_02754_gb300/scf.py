"""Self-consistent-field loop around the eigensolver (Sec. III.B.1), one context.

Every numerical step runs in the library: the fields from the densities
(``gbc_scf_fields``: V_eff = V_ext + V_xc, B_xc, with the closed-form exchange
stand-in), one ChFSI cycle per SCF step on the block carried over
(``gbc_lanczos_bounds``, ``gbc_filter``, ``gbc_cholgs``, ``gbc_rayleigh_ritz``),
Fermi-Dirac occupations of the Ritz values (``gbc_fermi_occupations``), the
output densities (``gbc_density_dev``) and Anderson mixing
(``gbc_anderson_mix``).  This module only sequences the calls and holds the
device buffers of the mixing history.
"""
from __future__ import annotations

import numpy as np

from .gbchfsi import fermi_occupations


def scf_loop(ctx, X, vext, v0, nelec, kT, degree, lanczos_steps, alpha=0.5, nhist=4, iters=20,
             tol=0.0):
    """Run up to ``iters`` SCF steps.

    ctx: a Context whose fields are V_ext with B = 0 on entry (the first block comes
    from CholGS + Rayleigh-Ritz of X under H[V_ext]); X: its block [M, 2, nvec] on the
    device, updated in place; vext: float64 CUDA tensor [E, nq^3]; v0: the Lanczos
    start vector (complex128 CUDA tensor [M, 2]).  Stops early once the residual norm
    || F(x) - x || (Eq. innerPdt) is <= tol.  Returns a dict with the residual norms,
    the final input densities [E, 4, nq^3] and the final Ritz values."""
    import torch
    E, q = ctx.ncells, ctx.nq ** 3

    def new():
        return torch.empty((E, 4, q), dtype=torch.float64, device=X.device)

    def densities(ritz):
        f, _ = fermi_occupations(np.asarray(ritz)[None], None, nelec, kT)
        occ = torch.from_numpy(np.ascontiguousarray(f[0])).to(X.device)
        out = new()
        ctx.density_dev(X, occ, out)
        return out

    ctx.cholgs(X)
    ritz = ctx.rayleigh_ritz(X)
    x_in = densities(ritz)
    xs, fs, res = [], [], []
    for _ in range(iters):
        ctx.scf_fields(x_in, vext)
        lo, hi = ctx.lanczos_bounds(v0, lanczos_steps)
        ctx.filter(X, degree, float(ritz[-1]), hi, min(lo, float(ritz[0])))
        ctx.cholgs(X)
        ritz = ctx.rayleigh_ritz(X)
        x_out = densities(ritz)
        xs, fs = (xs + [x_in])[-nhist:], (fs + [x_out])[-nhist:]
        x_next = new()
        _, rn = ctx.anderson_mix(xs, fs, alpha, x_next)
        res.append(rn)
        x_in = x_next
        if rn <= tol:
            break
    return {"res": np.array(res), "dens": x_in, "ritz": np.asarray(ritz)}
