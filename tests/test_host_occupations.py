"""gbc_fermi_occupations (host code in the library, no GPU needed) against the oracle's
Fermi-Dirac occupations: the chemical potential and every f_nk to rounding, equal and
uneven Brillouin-zone weights, a fractional and an integer electron count, and the
argument errors."""
import numpy as np
import pytest

from oracle import density as od

KT = 500.0 * 3.166811563e-6


@pytest.fixture(scope="module")
def g():
    import __graft_entry__ as ge
    ge.build()
    import paper_2410_02754_gb300 as pkg
    return pkg


@pytest.mark.parametrize("nk,ns,nelec,weights", [(1, 64, 32.0, None), (4, 48, 20.5, "mp"),
                                                 (3, 10, 0.3, "uneven")])
def test_fermi_matches_oracle(g, nk, ns, nelec, weights):
    rng = np.random.default_rng(nk * 100 + ns)
    eps = np.sort(rng.uniform(-0.8, 1.5, (nk, ns)), axis=1)
    if weights is None:
        w = np.full(nk, 1.0 / nk)
    elif weights == "mp":
        w = np.full(nk, 1.0 / nk)
    else:
        w = rng.uniform(0.1, 1.0, nk)
    f, mu = g.fermi_occupations(eps, None if weights is None else w, nelec, KT)
    fo, muo = od.fermi_occupations(eps, w, nelec, KT)
    assert abs(mu - muo) < 1e-12
    np.testing.assert_allclose(f, fo, rtol=0, atol=1e-12)
    assert abs((w[:, None] * f).sum() - nelec) < 1e-10


def test_fermi_argument_errors(g):
    eps = np.linspace(-1, 1, 8)[None, :]
    for args in [(eps, None, 0.0, KT), (eps, None, 8.0, KT), (eps, None, 3.0, 0.0),
                 (eps, [-1.0], 3.0, KT), (np.array([[0.0, np.nan]]), None, 1.0, KT)]:
        with pytest.raises(g.GbcError):
            g.fermi_occupations(*args)
