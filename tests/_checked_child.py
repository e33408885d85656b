"""Child process of test_gpu_checked.py, run with GBCHFSI_CHECKED=1 so the binding loads
the checked build: parity of the checked kernels against the FP64 oracle with no index
check firing, then the self-test's out-of-range store reported once as GBC_ECHECK."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import synthetic as syn  # noqa: E402
from oracle import chfsi as oc  # noqa: E402
from oracle import fe  # noqa: E402
import paper_2410_02754_gb300 as g  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def main():
    assert g.LIB_PATH.endswith("libgbchfsi_checked.so"), g.LIB_PATH
    assert g.build_info()["checked"]
    # periodic in x, Dirichlet in y and z (absent nodes on two face pairs), 18 SOC
    # projectors (tensor engine: packed and operand-staging expansion, projection)
    prob = syn.make_problem(ncell=(4, 3, 3), h=(1.0, 1.0, 1.0), p=4, periodic=(1, 0, 0),
                            k=(0.1, 0.0, 0.0), natoms=4, rc=1.6, seed=31,
                            channels=syn.SPD_CHANNELS)
    d = fe.Discretisation(prob)
    M = d.mesh.nnodes
    X = syn.random_block(M, 33, 5)
    bounds = (1.0, 80.0, -2.0)
    ref_h = d.apply_h(X)
    ref_f = oc.cheb_filter(d.apply_htilde, X, 3, *bounds)
    for prec, engine, tol in ((0, 0, 1e-11), (1, 0, 1e-5), (1, 1, 1e-5)):
        c = g.Context(0)
        c.set_problem(prob)
        c.set_precision(prec)
        if prec == 1:
            c.set_nonlocal_engine(engine)
        dt = torch.complex128 if prec == 0 else torch.complex64
        Xd = torch.from_numpy(X).to(dt).cuda()
        Yd = torch.empty_like(Xd)
        c.apply_h(Xd, Yd)
        c.sync_status()                          # raises on GBC_ECHECK
        e = rel(Yd.cpu().numpy().astype(np.complex128), ref_h)
        assert e < tol, ("apply_h", prec, engine, e)
        c.filter(Xd, 3, *bounds)                 # FP32: fused recurrence, face-row pass
        c.sync_status()
        e = rel(Xd.cpu().numpy().astype(np.complex128), ref_f)
        assert e < 2 * tol, ("filter", prec, engine, e)
        c.close()
    # the self-test: an in-range store passes, an out-of-range one is recorded and skipped
    c = g.Context(0)
    c.set_problem(prob)
    assert g.check_selftest(5) == 0
    c.sync_status()
    assert g.check_selftest(100) == 0
    try:
        c.sync_status()
    except g.GbcError as exc:
        assert exc.status == 8 and "index 100" in str(exc) and "site 7" in str(exc), str(exc)
    else:
        raise AssertionError("GBC_ECHECK not reported")
    c.sync_status()                              # the word was cleared
    c.close()
    print("CHECKED-OK")


if __name__ == "__main__":
    main()
