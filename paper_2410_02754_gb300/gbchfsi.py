"""ctypes binding of libgbchfsi (the C ABI in include/gbchfsi.h).

Argument marshalling only: every arithmetic step runs in the library's CUDA
kernels.  Device blocks are torch CUDA tensors used as plain memory:
complex128 for ``FP64``, complex64 for ``FP32``, shape [M, 2, ldx] (or a
contiguous view with that layout).  The library is loaded from this package
directory; importing this module on a machine without the built library or
without a CUDA device raises, there is no fallback.  With GBCHFSI_CHECKED=1 in
the environment the checked build (libgbchfsi_checked.so, device index checks)
is loaded instead.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbchfsi_checked.so" if os.environ.get("GBCHFSI_CHECKED") == "1"
                        else "libgbchfsi.so")

FP64, FP32 = 0, 1
TF32, BF16X3 = 2, 3          # FP32 blocks, cell products as tcgen05 GEMMs (single TF32 / BF16 x3)
STATUS = {0: "GBC_OK", 1: "GBC_EINVAL", 2: "GBC_ENOMEM", 3: "GBC_ECUDA", 4: "GBC_ESTATE",
          5: "GBC_ENOTPD", 6: "GBC_ETIMEOUT", 7: "GBC_EUNSUPPORTED", 8: "GBC_ECHECK"}

# every entry point declared in include/gbchfsi.h
EXPORTS = ["gbc_create", "gbc_destroy", "gbc_last_error", "gbc_version", "gbc_set_mesh",
           "gbc_set_kpoint", "gbc_set_fields", "gbc_set_projectors", "gbc_set_precision",
           "gbc_get_nnodes", "gbc_get_mass", "gbc_apply_h", "gbc_lanczos_bounds", "gbc_filter",
           "gbc_filter_residual",
           "gbc_cholgs", "gbc_rayleigh_ritz", "gbc_set_timing", "gbc_get_timing",
           "gbc_apply_h_noalloc", "gbc_batch_create", "gbc_batch_destroy",
           "gbc_batch_last_error", "gbc_batch_filter", "gbc_batch_launches", "gbc_tune",
           "gbc_get_tile", "gbc_filter_vjp", "gbc_energy_grad", "gbc_set_delta",
           "gbc_tc_gemm_nt", "gbc_tc_wait_selftest", "gbc_set_nonlocal_engine", "gbc_get_nonlocal_engine",
           "gbc_sync_status", "gbc_density", "gbc_density_dev", "gbc_fermi_occupations",
           "gbc_prolongate", "gbc_scf_fields", "gbc_anderson_mix", "gbc_get_ndof",
           "gbc_filter_backward", "gbc_alu_peak", "gbc_set_cell_variant",
           "gbc_get_cell_variant", "gbc_build_info", "gbc_check_selftest",
           "gbc_set_deterministic", "gbc_get_deterministic"]
FAMILIES = {"hx_local": 0, "nonlocal": 1, "cheb": 2, "gram": 3, "rotate": 4, "dense": 5}


class GbcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load (once) and type the shared library.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{os.path.basename(path)} not built at {path}; run __graft_entry__.build()"
                          " (the checked build: paper_2410_02754_gb300._build.build(checked=True))")
    lib = ct.CDLL(path)
    P, I, D, V = ct.c_void_p, ct.c_int, ct.c_double, ct.c_void_p
    IP, DP = ct.POINTER(ct.c_int), ct.POINTER(ct.c_double)
    sig = {
        "gbc_create": ([ct.POINTER(P), I], I),
        "gbc_destroy": ([P], None),
        "gbc_last_error": ([P], ct.c_char_p),
        "gbc_version": ([], ct.c_char_p),
        "gbc_set_mesh": ([P, IP, DP, I, I, IP], I),
        "gbc_set_kpoint": ([P, DP], I),
        "gbc_set_fields": ([P, DP, DP, DP, DP], I),
        "gbc_set_projectors": ([P, I, IP, IP, IP, IP, DP, DP], I),
        "gbc_set_precision": ([P, I], I),
        "gbc_get_nnodes": ([P, ct.POINTER(ct.c_longlong)], I),
        "gbc_get_mass": ([P, DP], I),
        "gbc_apply_h": ([P, V, V, I, I, V], I),
        "gbc_lanczos_bounds": ([P, V, I, DP, DP, V], I),
        "gbc_filter": ([P, V, I, I, I, D, D, D, V], I),
        "gbc_cholgs": ([P, V, I, I, V], I),
        "gbc_filter_residual": ([P, V, I, I, I, D, D, D, DP, V], I),
        "gbc_rayleigh_ritz": ([P, V, I, I, DP, V], I),
        "gbc_set_timing": ([P, I], I),
        "gbc_apply_h_noalloc": ([P, V, V, I, I, V], I),
        "gbc_batch_create": ([ct.POINTER(P), I, ct.POINTER(P)], I),
        "gbc_batch_destroy": ([P], None),
        "gbc_batch_last_error": ([P], ct.c_char_p),
        "gbc_batch_filter": ([P, ct.POINTER(P), IP, IP, IP, DP, V], I),
        "gbc_batch_launches": ([P, IP], I),
        "gbc_tune": ([P, I, V], I),
        "gbc_get_tile": ([P, IP], I),
        "gbc_filter_vjp": ([P, V, V, V, DP, DP, DP, I, I, I, D, D, D, I, V], I),
        "gbc_energy_grad": ([P, V, DP, V, DP, DP, DP, DP, I, I, V], I),
        "gbc_set_delta": ([P, DP], I),
        "gbc_density": ([P, V, DP, DP, DP, I, I, V], I),
        "gbc_density_dev": ([P, V, V, V, I, I, I, V], I),
        "gbc_fermi_occupations": ([DP, DP, I, I, D, D, DP, DP], I),
        "gbc_prolongate": ([P, P, V, I, V, I, I, V], I),
        "gbc_get_ndof": ([P, ct.POINTER(ct.c_longlong)], I),
        "gbc_filter_backward": ([P, V, V, V, DP, DP, DP, I, I, I, D, D, D, I, V], I),
        "gbc_scf_fields": ([P, V, V, V, V], I),
        "gbc_anderson_mix": ([P, ct.POINTER(V), ct.POINTER(V), I, D, V, DP, DP, V], I),
        "gbc_tc_gemm_nt": ([V, V, V, I, I, I, V], I),
        "gbc_tc_wait_selftest": ([I, V], I),
        "gbc_build_info": ([IP], I),
        "gbc_set_deterministic": ([P, I], I),
        "gbc_get_deterministic": ([P, IP], I),
        "gbc_check_selftest": ([ct.c_longlong, V], I),
        "gbc_set_nonlocal_engine": ([P, I], I),
        "gbc_get_nonlocal_engine": ([P, IP], I),
        "gbc_sync_status": ([P, V], I),
        "gbc_get_timing": ([P, I, DP, ct.POINTER(ct.c_longlong)], I),
        "gbc_alu_peak": ([I, DP, DP, V], I),
        "gbc_set_cell_variant": ([P, I], I),
        "gbc_get_cell_variant": ([P, IP, IP, IP], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _iarr(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ct.POINTER(ct.c_int))


def _darr(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ct.POINTER(ct.c_double))


def fermi_occupations(eps, kweights, nelec, kT):
    """Fermi-Dirac occupations of Ritz values eps [nk, nstates] (Ha) with Brillouin-zone
    weights (None: equal) and mu fixed by the electron count; returns (occ, mu)."""
    lib = load_library()
    e, ep = _darr(np.atleast_2d(np.asarray(eps, np.float64)))
    nk, ns = e.shape
    w, wp = (None, None) if kweights is None else _darr(np.asarray(kweights, np.float64))
    occ = np.zeros_like(e)
    mu = ct.c_double()
    st = lib.gbc_fermi_occupations(ep, wp, int(nk), int(ns), float(nelec), float(kT),
                                   occ.ctypes.data_as(ct.POINTER(ct.c_double)), ct.byref(mu))
    if st != 0:
        raise GbcError(st, "gbc_fermi_occupations: invalid arguments" if st == 1 else
                       "gbc_fermi_occupations: no bracket for the chemical potential")
    return occ, mu.value


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ct.c_void_p(getattr(stream, "cuda_stream", stream))


class Context:
    """One problem (mesh, k-point, fields, projectors) on one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load_library()
        h = ct.c_void_p()
        st = self.lib.gbc_create(ct.byref(h), device)
        if st != 0:
            raise GbcError(st, f"gbc_create(device={device}) failed")
        self.h = h
        self.device = device
        self.prec = FP64
        self.nnodes = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.gbc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        if st != 0:
            raise GbcError(st, self.lib.gbc_last_error(self.h).decode())

    # ---- problem definition ---------------------------------------------------
    def set_mesh(self, ncell, h, p, nq, periodic):
        nc, ncp = _iarr(ncell)
        hh, hp = _darr(h)
        pe, pp = _iarr([1 if b else 0 for b in periodic])
        self._chk(self.lib.gbc_set_mesh(self.h, ncp, hp, int(p), int(nq), pp))
        n = ct.c_longlong()
        self._chk(self.lib.gbc_get_nnodes(self.h, ct.byref(n)))
        self.nnodes = n.value
        self.ncells = int(np.prod(ncell))
        self.nq = int(nq)
        self.ndelta = 0

    def set_kpoint(self, k):
        kk, kp = _darr(k)
        self._chk(self.lib.gbc_set_kpoint(self.h, kp))

    def set_fields(self, veff, bx, by, bz):
        arrs = [_darr(x) for x in (veff, bx, by, bz)]
        self._chk(self.lib.gbc_set_fields(self.h, *[p for _, p in arrs]))

    def set_projectors(self, natoms, npj, nsupp, supp_cell, supp_img, pvals, delta):
        if natoms == 0:
            self._chk(self.lib.gbc_set_projectors(self.h, 0, None, None, None, None, None, None))
            self.ndelta = 0
            return
        self.ndelta = int(sum(4 * int(n) * int(n) for n in npj))
        a1, p1 = _iarr(npj)
        a2, p2 = _iarr(nsupp)
        a3, p3 = _iarr(supp_cell)
        a4, p4 = _iarr(supp_img)
        a5, p5 = _darr(pvals)
        d = np.ascontiguousarray(delta, dtype=np.complex128)
        a6, p6 = _darr(d.view(np.float64))
        self._chk(self.lib.gbc_set_projectors(self.h, int(natoms), p1, p2, p3, p4, p5, p6))

    def set_problem(self, prob):
        """Load a problem object with attributes ncell, h, p, nq, periodic, k,
        veff, bx, by, bz and flat_projectors() (the synthetic generator's)."""
        self.set_mesh(prob.ncell, prob.h, prob.p, prob.nq, prob.periodic)
        self.set_kpoint(prob.k)
        self.set_fields(prob.veff, prob.bx, prob.by, prob.bz)
        fp = prob.flat_projectors()
        self.set_projectors(fp["natoms"], fp["npj"], fp["nsupp"], fp["supp_cell"], fp["supp_img"],
                            fp["pvals"], fp["delta"])

    def set_precision(self, prec):
        self._chk(self.lib.gbc_set_precision(self.h, int(prec)))
        self.prec = prec

    def set_deterministic(self, on=True):
        """Fixed-order sums instead of atomics in the FP64 kernels (gbc_set_deterministic)."""
        self._chk(self.lib.gbc_set_deterministic(self.h, 1 if on else 0))

    def deterministic(self):
        v = ct.c_int()
        self._chk(self.lib.gbc_get_deterministic(self.h, ct.byref(v)))
        return bool(v.value)

    def set_nonlocal_engine(self, engine):
        """0 = SIMT cores, 1 = tcgen05 tensor cores (FP32 projector contractions)."""
        self._chk(self.lib.gbc_set_nonlocal_engine(self.h, int(engine)))

    def nonlocal_engine(self):
        """Engine the FP32 nonlocal step runs for the current projectors."""
        e = ct.c_int()
        self._chk(self.lib.gbc_get_nonlocal_engine(self.h, ct.byref(e)))
        return e.value

    def sync_status(self, stream=None):
        """Synchronise and raise if a device-side bounded wait expired."""
        self._chk(self.lib.gbc_sync_status(self.h, _stream_ptr(stream)))

    def mass(self):
        md = np.empty(self.nnodes, np.float64)
        self._chk(self.lib.gbc_get_mass(self.h, md.ctypes.data_as(ct.POINTER(ct.c_double))))
        return md

    # ---- block calls ------------------------------------------------------------
    def _block(self, X):
        import torch
        want = torch.complex128 if self.prec == FP64 else torch.complex64
        if not X.is_cuda:
            raise ValueError("block must be a CUDA tensor")
        if X.dtype != want:
            raise ValueError(f"block dtype {X.dtype} does not match the precision ({want})")
        if X.dim() != 3 or X.shape[0] != self.nnodes or X.shape[1] != 2:
            raise ValueError(f"block must have shape [M={self.nnodes}, 2, ldx]")
        if X.stride(2) != 1 or X.stride(1) != X.shape[2] or X.stride(0) != 2 * X.shape[2]:
            raise ValueError("block must be contiguous [M][2][ldx]")
        return ct.c_void_p(X.data_ptr()), X.shape[2]

    def apply_h(self, X, Y, nvec=None, stream=None):
        px, ldx = self._block(X)
        py, ldy = self._block(Y)
        if ldx != ldy:
            raise ValueError("X and Y need the same ldx")
        nvec = ldx if nvec is None else nvec
        self._chk(self.lib.gbc_apply_h(self.h, px, py, int(nvec), int(ldx), _stream_ptr(stream)))

    def apply_h_noalloc(self, X, Y, nvec=None, stream=None):
        """H.X without any device allocation by the library (fixed 32 MiB
        scratch); the tables must have been built by an earlier call."""
        px, ldx = self._block(X)
        py, ldy = self._block(Y)
        if ldx != ldy:
            raise ValueError("X and Y need the same ldx")
        nvec = ldx if nvec is None else nvec
        self._chk(self.lib.gbc_apply_h_noalloc(self.h, px, py, int(nvec), int(ldx),
                                               _stream_ptr(stream)))

    def filter(self, X, degree, lT, lmax, lmin, nvec=None, stream=None):
        px, ldx = self._block(X)
        nvec = ldx if nvec is None else nvec
        self._chk(self.lib.gbc_filter(self.h, px, int(nvec), int(ldx), int(degree), float(lT),
                                      float(lmax), float(lmin), _stream_ptr(stream)))

    def filter_residual(self, X, degree, lT, lmax, lmin, ritz, nvec=None, stream=None):
        """Residual-split filter of a block of Ritz pairs (X, ritz)."""
        px, ldx = self._block(X)
        nvec = ldx if nvec is None else nvec
        r, rp = _darr(np.asarray(ritz, np.float64)[:nvec])
        self._chk(self.lib.gbc_filter_residual(self.h, px, int(nvec), int(ldx), int(degree),
                                               float(lT), float(lmax), float(lmin), rp,
                                               _stream_ptr(stream)))

    def cholgs(self, X, nvec=None, stream=None):
        px, ldx = self._block(X)
        nvec = ldx if nvec is None else nvec
        self._chk(self.lib.gbc_cholgs(self.h, px, int(nvec), int(ldx), _stream_ptr(stream)))

    def rayleigh_ritz(self, X, nvec=None, stream=None):
        px, ldx = self._block(X)
        nvec = ldx if nvec is None else nvec
        out = np.empty(nvec, np.float64)
        self._chk(self.lib.gbc_rayleigh_ritz(self.h, px, int(nvec), int(ldx),
                                             out.ctypes.data_as(ct.POINTER(ct.c_double)),
                                             _stream_ptr(stream)))
        return out

    def lanczos_bounds(self, v0, steps, stream=None):
        import torch
        if not (v0.is_cuda and v0.dtype == torch.complex128 and v0.is_contiguous()
                and tuple(v0.shape) == (self.nnodes, 2)):
            raise ValueError("v0 must be a contiguous complex128 CUDA tensor [M, 2]")
        lo, hi = ct.c_double(), ct.c_double()
        self._chk(self.lib.gbc_lanczos_bounds(self.h, ct.c_void_p(v0.data_ptr()), int(steps),
                                              ct.byref(lo), ct.byref(hi), _stream_ptr(stream)))
        return lo.value, hi.value

    # ---- tracing --------------------------------------------------------------------
    def set_timing(self, enable=True):
        self._chk(self.lib.gbc_set_timing(self.h, 1 if enable else 0))

    def timing(self):
        """{family: (total_ms, launches)} since the last set_timing."""
        out = {}
        for name, fam in FAMILIES.items():
            t, n = ct.c_double(), ct.c_longlong()
            self._chk(self.lib.gbc_get_timing(self.h, fam, ct.byref(t), ct.byref(n)))
            out[name] = (t.value, n.value)
        return out

    # ---- backward ----------------------------------------------------------------
    def _grad_outputs(self):
        nq3 = self.nq ** 3
        gV = np.zeros(self.ncells * nq3)
        gB = np.zeros(3 * self.ncells * nq3)
        gD = np.zeros(2 * self.ndelta)
        return gV, gB, gD

    def _split(self, gV, gB, gD):
        n = self.ncells * self.nq ** 3
        return (gV.reshape(self.ncells, -1), gB[:n].reshape(self.ncells, -1),
                gB[n:2 * n].reshape(self.ncells, -1), gB[2 * n:].reshape(self.ncells, -1),
                gD.view(np.complex128))

    def filter_vjp(self, X0, GY, GX, degree, lT, lmax, lmin, ckpt_every=5, nvec=None, stream=None):
        """Backward of filter: fills GX; returns (gV, gBx, gBy, gBz, gDelta)."""
        px, ldx = self._block(X0)
        pg, _ = self._block(GY)
        po, _ = self._block(GX)
        nvec = ldx if nvec is None else nvec
        gV, gB, gD = self._grad_outputs()
        dp = lambda a: a.ctypes.data_as(ct.POINTER(ct.c_double))
        self._chk(self.lib.gbc_filter_vjp(self.h, px, pg, po, dp(gV), dp(gB), dp(gD), int(nvec),
                                          int(ldx), int(degree), float(lT), float(lmax),
                                          float(lmin), int(ckpt_every), _stream_ptr(stream)))
        return self._split(gV, gB, gD)

    def energy_grad(self, Y, w, GY, nvec=None, stream=None):
        """L = sum_i w_i y_i^H H y_i; fills GY = 2 H Y diag(w); returns
        (L, gV, gBx, gBy, gBz, gDelta) at fixed Y."""
        py, ldx = self._block(Y)
        pg, _ = self._block(GY)
        nvec = ldx if nvec is None else nvec
        ww, wp = _darr(np.asarray(w, np.float64)[:nvec])
        gV, gB, gD = self._grad_outputs()
        loss = ct.c_double()
        dp = lambda a: a.ctypes.data_as(ct.POINTER(ct.c_double))
        self._chk(self.lib.gbc_energy_grad(self.h, py, wp, pg, ct.byref(loss), dp(gV), dp(gB),
                                           dp(gD), int(nvec), int(ldx), _stream_ptr(stream)))
        return (loss.value,) + self._split(gV, gB, gD)

    def density(self, X, occ, nvec=None, stream=None):
        """rho and m at the Gauss points (Eqs. rho, mag) of the block X with
        occupations occ: returns numpy (rho [E, nq^3], m [3, E, nq^3])."""
        px, ldx = self._block(X)
        nvec = ldx if nvec is None else nvec
        _, op = _darr(np.asarray(occ, np.float64)[:nvec])
        n = self.ncells * self.nq ** 3
        rho, mag = np.zeros(n), np.zeros(3 * n)
        dp = lambda a: a.ctypes.data_as(ct.POINTER(ct.c_double))
        self._chk(self.lib.gbc_density(self.h, px, op, dp(rho), dp(mag), int(nvec), int(ldx),
                                       _stream_ptr(stream)))
        return rho.reshape(self.ncells, -1), mag.reshape(3, self.ncells, -1)

    def density_dev(self, X, occ, out, nvec=None, accumulate=False, stream=None):
        """Device form: occ (float64 CUDA tensor [nvec]) and out (float64 CUDA tensor
        [E, 4, nq^3]: rho, m_x, m_y, m_z; overwritten, or added to with accumulate).
        Asynchronous."""
        import torch
        px, ldx = self._block(X)
        nvec = ldx if nvec is None else nvec
        n = self.ncells * 4 * self.nq ** 3
        for t, size in ((occ, nvec), (out, n)):
            if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() < size:
                raise ValueError("occ / out must be contiguous float64 CUDA tensors of the stated size")
        self._chk(self.lib.gbc_density_dev(self.h, px, ct.c_void_p(occ.data_ptr()),
                                           ct.c_void_p(out.data_ptr()), int(nvec), int(ldx),
                                           int(bool(accumulate)), _stream_ptr(stream)))

    def prolongate_from(self, coarse, Xc, Xf, nvec=None, stream=None):
        """Two-grid transfer into this (fine, order p or p_c + 1) context's block Xf from
        the block Xc of ``coarse`` (order p_c, same mesh): exact nodal interpolation."""
        pc, ldxc = coarse._block(Xc)
        pf, ldxf = self._block(Xf)
        nvec = min(ldxc, ldxf) if nvec is None else nvec
        self._chk(self.lib.gbc_prolongate(coarse.h, self.h, pc, int(ldxc), pf, int(ldxf),
                                          int(nvec), _stream_ptr(stream)))

    def _dens(self, t, comps):
        import torch
        n = self.ncells * comps * self.nq ** 3
        if t is None:
            return None
        if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != n:
            raise ValueError(f"expected a contiguous float64 CUDA tensor of {n} values")
        return ct.c_void_p(t.data_ptr())

    def scf_fields(self, dens, vext, exc=None, stream=None):
        """V_eff = vext + V_xc and B_xc from dens [E, 4, nq^3] into this context's fields
        (closed-form exchange-only local spin density stand-in).  Synchronous."""
        self._chk(self.lib.gbc_scf_fields(self.h, self._dens(dens, 4), self._dens(vext, 1),
                                          self._dens(exc, 1), _stream_ptr(stream)))

    def anderson_mix(self, xin, xout, alpha, xnext, stream=None):
        """Anderson mixing of the histories (lists of [E, 4, nq^3] tensors, oldest first)
        into xnext; returns (coefficients, residual norm of the last pair)."""
        n = len(xin)
        if n != len(xout) or not 1 <= n <= 8:
            raise ValueError("need 1..8 input/output pairs")
        pin = (ct.c_void_p * n)(*[self._dens(x, 4) for x in xin])
        pout = (ct.c_void_p * n)(*[self._dens(x, 4) for x in xout])
        coef = np.zeros(n)
        rn = ct.c_double()
        self._chk(self.lib.gbc_anderson_mix(self.h, pin, pout, n, float(alpha),
                                            self._dens(xnext, 4),
                                            coef.ctypes.data_as(ct.POINTER(ct.c_double)),
                                            ct.byref(rn), _stream_ptr(stream)))
        return coef, rn.value

    def set_delta(self, delta):
        d = np.ascontiguousarray(delta, dtype=np.complex128)
        a, p = _darr(d.view(np.float64))
        self._chk(self.lib.gbc_set_delta(self.h, p))

    # ---- tile autotuner -------------------------------------------------------------
    def tune(self, nvec, stream=None):
        """Pick the FP32 cell-apply variant by timing; returns vectors per CTA."""
        self._chk(self.lib.gbc_tune(self.h, int(nvec), _stream_ptr(stream)))
        return self.tile()

    def tile(self):
        v = ct.c_int()
        self._chk(self.lib.gbc_get_tile(self.h, ct.byref(v)))
        return v.value

    def set_cell_variant(self, variant):
        """Override the tuner's FP32 cell-apply variant (0 .. GBC_CELL_VARIANTS - 1)."""
        self._chk(self.lib.gbc_set_cell_variant(self.h, int(variant)))

    def cell_variant(self):
        """(variant, vectors per CTA, threads per CTA) of the FP32 cell apply."""
        v, vb, nt = ct.c_int(), ct.c_int(), ct.c_int()
        self._chk(self.lib.gbc_get_cell_variant(self.h, ct.byref(v), ct.byref(vb), ct.byref(nt)))
        return v.value, vb.value, nt.value


class Batch:
    """Several contexts filtered together (one persistent cell-apply launch per
    group of systems sharing FE order, cell edges and k-point; CUDA-graph replay)."""

    def __init__(self, contexts):
        self.lib = load_library()
        self.ctxs = list(contexts)
        arr = (ct.c_void_p * len(self.ctxs))(*[c.h for c in self.ctxs])
        h = ct.c_void_p()
        st = self.lib.gbc_batch_create(ct.byref(h), len(self.ctxs), arr)
        if st != 0:
            raise GbcError(st, "gbc_batch_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.gbc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def filter(self, blocks, degrees, bounds, stream):
        """blocks: tensors [M_i, 2, ldx_i]; degrees: ints; bounds: (lT, lmax, lmin) per
        system; stream: a torch.cuda.Stream that is not the legacy default stream."""
        n = len(self.ctxs)
        ptrs, nv, ld = [], [], []
        for c, X in zip(self.ctxs, blocks):
            p, ldx = c._block(X)
            ptrs.append(p.value)
            nv.append(ldx)
            ld.append(ldx)
        Xa = (ct.c_void_p * n)(*ptrs)
        a1, p1 = _iarr(nv)
        a2, p2 = _iarr(ld)
        a3, p3 = _iarr(degrees)
        a4, p4 = _darr(np.asarray(bounds, np.float64).reshape(-1))
        st = self.lib.gbc_batch_filter(self.h, Xa, p1, p2, p3, p4, _stream_ptr(stream))
        if st != 0:
            raise GbcError(st, self.lib.gbc_batch_last_error(self.h).decode())

    def launches(self):
        v = ct.c_int()
        self.lib.gbc_batch_launches(self.h, ct.byref(v))
        return v.value


def tc_gemm_nt(A, B, stream=None):
    """D = A @ B.T on the tcgen05 tensor cores (3xTF32); A [M, K], B [N, K] float32 CUDA."""
    import torch
    lib = load_library()
    A = A.contiguous()
    B = B.contiguous()
    M, K = A.shape
    N = B.shape[0]
    D = torch.empty((M, N), dtype=torch.float32, device=A.device)
    st = lib.gbc_tc_gemm_nt(ct.c_void_p(A.data_ptr()), ct.c_void_p(B.data_ptr()),
                            ct.c_void_p(D.data_ptr()), M, N, K, _stream_ptr(stream))
    if st != 0:
        raise GbcError(st, "gbc_tc_gemm_nt failed")
    return D



PEAKS = {"ffma": 0, "ffma2": 1, "dfma": 2, "tf32": 3, "bf16": 4}


def alu_peak(which, stream=None):
    """Measured arithmetic rate of the current device: (FLOP/s, seconds of the timed
    launch) for which in PEAKS (FP32 FMA, paired FP32 FMA, FP64 FMA, tcgen05 TF32 and
    BF16 MMA)."""
    rate, sec = ct.c_double(), ct.c_double()
    st = load_library().gbc_alu_peak(int(PEAKS[which]), ct.byref(rate), ct.byref(sec),
                                     _stream_ptr(stream))
    if st != 0:
        raise GbcError(st, f"gbc_alu_peak({which}) failed")
    return rate.value, sec.value


def build_info():
    """{'checked': True} for the checked build (device index checks), else False."""
    v = ct.c_int()
    st = load_library().gbc_build_info(ct.byref(v))
    if st != 0:
        raise GbcError(st, "gbc_build_info failed")
    return {"checked": bool(v.value)}


def check_selftest(index, stream=None):
    """One guarded store at ``index`` into a 64-entry device array (gbc_check_selftest);
    returns the status code (0, or 7 = GBC_EUNSUPPORTED outside [0, 64) in the default
    build)."""
    return load_library().gbc_check_selftest(int(index), _stream_ptr(stream))


def tc_wait_selftest(max_iter=1000, stream=None):
    """Make one bounded device wait expire on purpose (see gbc_tc_wait_selftest)."""
    st = load_library().gbc_tc_wait_selftest(int(max_iter), _stream_ptr(stream))
    if st != 0:
        raise GbcError(st, "gbc_tc_wait_selftest failed")
