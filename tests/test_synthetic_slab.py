"""Synthetic generator pieces of the semi-periodic slab workload (no GPU, no full-size
generation): the 16x8x5 atom lattice inside the slab, the free-node count of the
periodic/periodic/Dirichlet mesh, and the locally summed wells equal to the full sum within
the cut (6 well widths: relative 1.5e-8) on a small mesh."""
import numpy as np

import synthetic as syn


def test_slab_lattice_and_node_count():
    c = syn.CONFIGS["slab40_p6"]
    n, sp, jit, origin = c["slab_lattice"]
    pos = syn._jittered_lattice(n, sp, jit, 0, origin)
    assert pos.shape == (640, 3)
    assert pos[:, 2].min() > 4.0 - jit and pos[:, 2].max() < 4.0 + 5 * 2.4 + jit   # inside the slab
    assert pos[:, 0].max() < 40.0 and pos[:, 1].max() < 40.0
    nodes = syn.n_free_nodes(c["ncell"], c["p"], c["periodic"])
    assert nodes == 240 * 240 * 119 == 6_854_400


def test_local_wells_match_the_full_sum():
    kw = dict(ncell=(6, 6, 5), h=(1.0, 1.0, 1.0), p=2, periodic=(1, 1, 0), natoms=5, seed=3,
              bmax=0.0)
    full = syn.make_problem(**kw)
    local = syn.make_problem(well_cutoff=4.8, **kw)
    np.testing.assert_allclose(local.veff, full.veff, rtol=0, atol=2e-8 * 2.0)
    assert not np.array_equal(local.veff, np.zeros_like(local.veff))
