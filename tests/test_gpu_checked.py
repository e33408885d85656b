"""The checked build (-DGBCHFSI_CHECKED, libgbchfsi_checked.so): device index checks in
the FP32 / FP64 cell applies, the face-row recurrence and the nonlocal kernels, read back
by gbc_sync_status as GBC_ECHECK; and the default build, whose checks are compiled out."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def g():
    import __graft_entry__ as ge
    ge.build()
    import paper_2410_02754_gb300 as pkg
    return pkg


def test_default_build_has_no_checks(g):
    """The default library reports an unchecked build and refuses the self-test's
    out-of-range index on the host (no guard on the device to catch it)."""
    assert not g.build_info()["checked"]
    assert g.check_selftest(3) == 0
    assert g.check_selftest(100) == 7   # GBC_EUNSUPPORTED, nothing launched
    assert g.check_selftest(-1) == 7


def test_checked_build_parity_and_selftest(g):
    """Build the checked library, then in a child process that loads it: H.X and a
    degree-3 filter (FP64; FP32 with the SIMT and the tensor-core nonlocal engines)
    against the FP64 oracle with no check firing, and the self-test's out-of-range
    store reported once as GBC_ECHECK (site 7, index 100) and then cleared."""
    from paper_2410_02754_gb300 import _build
    _build.build(checked=True)
    env = dict(os.environ, GBCHFSI_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_checked_child.py")],
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "CHECKED-OK" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
