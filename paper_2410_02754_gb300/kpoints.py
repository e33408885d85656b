"""k-points sharded over ranks, one GPU per rank.

The eigenproblems of different k-points are independent (Sec. III.B): each rank
filters its own k-point blocks with no exchange.  Two steps after the filter
couple them, and these are the only collectives of the path:

* occupations -- the chemical potential mu fixes the electron count over all
  k-points (Sec. II), so every rank's Ritz values and Brillouin-zone weights are
  all-gathered (small host arrays) and every rank evaluates
  ``gbc_fermi_occupations`` on the full set.  The routine is deterministic, so
  all ranks obtain the same mu and occupations;
* densities -- rho and m are Brillouin-zone sums over k-points of the Eqs. rho /
  mag densities: each rank accumulates its own k-points into one device array
  with ``gbc_density_dev`` (the weight w_k folded into that k-point's
  occupations), then one all-reduce (SUM) over ranks.

Global k-point order: rank 0's k-points, then rank 1's, and so on.
"""
from __future__ import annotations

import numpy as np

from .gbchfsi import fermi_occupations


def _dist():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist
    return None


def gather_ritz(ritz_local, kweights_local, group=None):
    """All-gather the Ritz values ([nk_local][nstates]) and weights of every rank.

    Returns (eps [nk_total, nstates], w [nk_total], first global index of this rank)."""
    eps_l = np.atleast_2d(np.asarray(ritz_local, np.float64))
    w_l = np.asarray(kweights_local, np.float64).reshape(-1)
    if eps_l.shape[0] != w_l.shape[0]:
        raise ValueError("one weight per local k-point required")
    dist = _dist()
    if dist is None:
        return eps_l, w_l, 0
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, (eps_l, w_l), group=group)
    ns = {p[0].shape[1] for p in parts}
    if len(ns) != 1:
        raise ValueError("every k-point needs the same number of states")
    rank = dist.get_rank(group)
    first = sum(p[0].shape[0] for p in parts[:rank])
    return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]),
            first)


def sharded_occupations(ritz_local, kweights_local, nelec, kT, group=None):
    """Fermi-Dirac occupations of this rank's k-points with the chemical potential
    of all ranks' k-points: returns (occ [nk_local, nstates], mu)."""
    eps, w, first = gather_ritz(ritz_local, kweights_local, group)
    occ, mu = fermi_occupations(eps, w, nelec, kT)
    nk_l = np.atleast_2d(np.asarray(ritz_local)).shape[0]
    return occ[first:first + nk_l], mu


def sharded_density(contexts, blocks, occ_local, kweights_local, out, group=None):
    """out [E, 4, nq^3] (float64, on this rank's device) = sum over every rank's
    k-points of w_k (rho_k, m_k): this rank's k-points accumulated by the density
    kernel, then one all-reduce (SUM).  contexts / blocks: this rank's k-points
    (one context and one filtered block each); occ_local [nk_local, nvec].  The
    kernels and the all-reduce both run on torch's current stream, in that order."""
    import torch
    if not (len(contexts) == len(blocks) == len(occ_local) == len(kweights_local)):
        raise ValueError("one context, block, occupation row and weight per local k-point")
    out.zero_()
    for ctx, X, f, wk in zip(contexts, blocks, occ_local, kweights_local):
        fw = torch.from_numpy(np.ascontiguousarray(float(wk) * np.asarray(f, np.float64)))
        ctx.density_dev(X, fw.to(out.device), out, nvec=len(f), accumulate=True)
    dist = _dist()
    if dist is not None:
        dist.all_reduce(out, op=dist.ReduceOp.SUM, group=group)
    return out
