#!/usr/bin/env python
"""ChFSI filter throughput on one GB300 (spinor-DOF x vectors x degree / s).

Workload (default, N = 1): the 16^3-cell, p = 6 (n_q = 8) periodic mesh with
884,736 FE nodes, 64 atoms with 18 SOC projectors each, a block of 256
two-component spinors, Chebyshev degree 20, on each of the 4 k-points of a
2x2x1 Monkhorst-Pack grid.  One timed step = the degree-20 filter of all four
k-point blocks (each degree = one H.X with its fused recurrence update), inputs
resident in HBM; value = 884736 * 256 * 20 * 4 / step time.  The mixed path
(complex64 filter, FP64 Gram/Rayleigh-Ritz) is timed; the FP64 filter and the
Ritz-value difference between the two paths are reported beside it.

``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the only place, with the ``cpu_baseline`` leg,
where this script runs the oracle).

Under torchrun (N > 1) every rank runs its own copy of the workload on its own
GPU (weak scaling, no collective in the data path); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ChFSI filter spinor-DOF·vectors·degree/s, mixed vs FP64 at 1e-6 Ha, 1 GB300"
UNIT = "spinor-DOF*vectors*degree/s"
WORKLOAD = ("16x16x16 periodic cells, p=6, nq=8 (884,736 nodes), 64 atoms x 18 SOC projectors, "
            "256 spinor vectors, Chebyshev degree 20, 4 k-points (2x2x1 MP)")


# ----------------------------------------------------------------------------
# distributed plumbing (shared with the gloo tests)
# ----------------------------------------------------------------------------
def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def dist_init(backend):
    import torch.distributed as dist
    rank, world, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return rank, world


def dist_barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def dist_max(x: float, device="cpu") -> float:
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        t = torch.tensor([x], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return x


def dist_sum(x: float, device="cpu") -> float:
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        t = torch.tensor([x], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())
    return x


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        # raw samples (the summary goes into the JSON line); GBC_CLOCKS_DIR keeps them
        d = os.environ.get("GBC_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"gbc_clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[4:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(r[0] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[2][1:]) if v.lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------
def _eo_flops(no: int, ni: int) -> int:
    """FP32 flops of one even-odd 1-D contraction of a complex pencil
    (ni inputs -> no outputs): e/o formation, E/O multiply-adds (2 flop),
    the middle column when ni is odd, and the output combination."""
    hi, ho = ni // 2, (no + 1) // 2
    f = 4 * hi                                   # e, o (re, im)
    for i in range(ho):
        f += 2 * (4 * hi + (2 if ni % 2 else 0))
        f += 2 + (2 if no - 1 - i != i else 0)
    return f


def flops_per_cell_vector(p: int, nq: int, kpt: bool) -> int:
    """Algorithmic flops (FMA = 2) of the cell apply as implemented, for one cell
    and one two-component vector: the kinetic/k part as 7 one-dimensional
    contractions (complex G = Gr + i Gi when k != 0), 3 + 3 interpolation /
    testing contractions n <-> nq, the pointwise 2x2 spin operator at the nq^3
    Gauss points, all 1-D contractions in even-odd form."""
    n, q = p + 1, nq
    b = _eo_flops(n, n)
    g = b + (_eo_flops(n, n) + 2 * n if kpt else 0)
    per_ps = n * n * 2                            # pencils x spins of an n^3 stage
    kin = per_ps * ((b + g) + (g + 2 * b + 2 * n) + (g + b + 2 * n))
    interp = 2 * (n * n + q * n + q * q) * _eo_flops(q, n)
    test = 2 * (q * q + q * n + n * n) * _eo_flops(n, q) + per_ps * 2 * n
    pointwise = q ** 3 * 32
    return kin + interp + test + pointwise


def hbm_peak():
    """Measured copy bandwidth of this machine's GPUs (GB/s) and where it came from."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "of fallback (6.8 TB/s)"


def CELL_TRAFFIC(nvec, variant):
    """DRAM bytes of one fused-recurrence cell-apply launch at ``nvec`` vectors on the
    cube16_p6 mesh, scaled from the ncu capture of the same variant at 32 vectors
    (profiles/), or None."""
    per32 = CELL_TRAFFIC_32.get(variant)
    if per32 is None:
        return None, f"no ncu capture of variant {variant} of this kernel version"
    return (0.034e9 + (per32 - 0.034e9) * nvec / 32,
            f"ncu capture of variant {variant} at 32 vectors (recurrence mode) scaled by "
            f"vectors: {per32 / 1.654e9:.2f}x the algorithmic bytes (X gather, interior Y / "
            "X_{k-1} reads and X_{k+1} writes, face-row Y read-modify-write)")


# DRAM bytes (read + write) of one recurrence-mode cell-apply launch on the cube16_p6 mesh at
# 32 vectors, per cell-apply variant, from the ncu capture in
# profiles/hx_cell_fused_cube16_p6_nvec32.md; 34 MB of it are the fields (fixed), the rest
# grows with the vector count
CELL_TRAFFIC_32 = {2: 1.781e9, 4: 1.786e9}


def tc_cell_leg(g, prob, k, X, nvec, peaks, simt_ms):
    """Time the TF32 and BF16x3 cell apply (tcgen05 GEMMs) on one H.X of X."""
    import torch
    np3, nq3 = (prob.p + 1) ** 3, prob.nq ** 3
    pad = lambda n: -(-n // 64) * 64
    QP, NPP = pad(nq3), pad(np3)
    rows = prob.ncells * 4 * nvec
    dense = 2.0 * rows * (QP * NPP + NPP * (QP + 2 * NPP))     # the two GEMMs as computed
    res = {"simt_fp32_ms": round(simt_ms, 3),
           "flops_dense_per_launch": dense,
           "how": "one H.X of the k-point-0 block (3 launches after one warm-up, CUDA events "
                  "of the cell-apply family); rows = cells x spins x vectors x re/im; GEMM 1 "
                  "interpolation (K = n_p^3), GEMM 2 testing + kinetic (K = n_q^3 + 2 n_p^3)"}
    Yref = torch.empty_like(X)
    c = g.Context(torch.cuda.current_device())
    c.set_problem(prob.with_(k=k))
    c.set_precision(g.FP32)
    c.apply_h(X, Yref)
    for name, prec, passes, pk in (("tf32", 2, 1, "tf32"), ("bf16x3", 3, 3, "bf16")):
        c.set_precision(prec)
        Y = torch.empty_like(X)
        c.apply_h(X, Y)
        c.sync_status()
        c.set_timing(True)
        for _ in range(3):
            c.apply_h(X, Y)
        t = c.timing()
        c.set_timing(False)
        c.sync_status()
        ms = t["hx_local"][0] / t["hx_local"][1]
        err = float(((Y - Yref).abs().pow(2).sum() / Yref.abs().pow(2).sum()).sqrt())
        peak = peaks.get(pk)
        ach = dense * passes / (ms / 1e3) / 1e12
        res[name] = {"ms": round(ms, 3), "tensor_tflops": round(ach, 1),
                     "frac_tensor": round(ach / peak, 4) if isinstance(peak, float) else None,
                     "peak_tflops": peak, "rel_diff_vs_fp32": err,
                     "over_simt": round(ms / simt_ms, 3)}
        del Y
    c.close()
    best = min(("simt_fp32", simt_ms), ("tf32", res["tf32"]["ms"]), ("bf16x3", res["bf16x3"]["ms"]),
               key=lambda x: x[1])
    res["fastest"] = best[0]
    return res


def build_contexts(g, prob, ks, prec, nl_engine=1):
    import torch
    ctxs = []
    for k in ks:
        c = g.Context(torch.cuda.current_device())
        c.set_problem(prob.with_(k=k))
        c.set_precision(prec)
        c.set_nonlocal_engine(nl_engine)
        ctxs.append(c)
    return ctxs


def run_gpu(args):
    import numpy as np
    import torch

    import __graft_entry__ as ge
    import synthetic as syn
    import paper_2410_02754_gb300 as g

    rank, world = dist_init("nccl" if int(os.environ.get("WORLD_SIZE", "1")) > 1 else "gloo")
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    ge.build()
    cfg = syn.CONFIGS[args.config]
    nvec = args.nvec or cfg["nvec"]
    degree = args.degree or cfg["degree"]
    prob = syn.config(args.config, seed=0)
    ks = syn.mp_kpoints(*cfg["kgrid"], prob.box)
    if args.kpoints:
        ks = ks[:args.kpoints]
    M = prob.nnodes
    units_per_step = M * nvec * degree * len(ks)

    # ---- arithmetic peaks of this GPU (the roofline denominators), measured by the
    # library's probes before anything else runs
    peaks = {}
    for w in ("ffma", "ffma2", "dfma", "tf32", "bf16"):
        try:
            peaks[w] = round(g.alu_peak(w)[0] / 1e12, 2)
        except Exception as exc:   # pragma: no cover - reported, not fatal
            peaks[w] = f"{type(exc).__name__}: {exc}"

    # ---- contexts, blocks, bounds (outside the timed region)
    ctx32 = build_contexts(g, prob, ks, g.FP32, args.nl_engine)
    for c in ctx32:
        c.tune(nvec)             # FP32 cell-apply variant (cached per p, k, block size)
        if args.cell_variant >= 0:
            c.set_cell_variant(args.cell_variant)
    X0 = syn.random_block(M, nvec, 0)
    v0 = torch.from_numpy(syn.random_start(M, 0)).cuda()
    bounds = []
    X32 = []
    ritz_k = []
    for c in ctx32:
        lo, hi = c.lanczos_bounds(v0, cfg["lanczos"])
        X = torch.from_numpy(X0).to(torch.complex64).cuda()
        c.cholgs(X)
        ritz = c.rayleigh_ritz(X)
        bounds.append((float(ritz[-1]), hi, min(lo, float(ritz[0]))))
        X32.append(X)
        ritz_k.append(ritz)
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()

    def step():
        for c, X, (lT, lmax, lmin) in zip(ctx32, X32, bounds):
            c.filter(X, degree, lT, lmax, lmin)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for c in ctx32:
        c.set_timing(True)
    dist_barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    dist_barrier()
    for c in ctx32:
        c.sync_status()      # raises if a tensor-core wait expired inside the timed region
    ms_total = ev0.elapsed_time(ev1)
    ms_total = dist_max(ms_total, device="cuda" if world > 1 else "cpu")
    ms_step = ms_total / args.steps
    value = dist_sum(units_per_step, device="cuda" if world > 1 else "cpu") / (ms_step / 1e3)

    # ---- per-kernel-family device time (CUDA events around every launch)
    fams = {}
    for c in ctx32:
        for name, (t, n) in c.timing().items():
            a = fams.setdefault(name, [0.0, 0])
            a[0] += t
            a[1] += n
        c.set_timing(False)
    # kernels per family launch: local 1, nonlocal 3 (project, couple, expand), epilogue 1
    # nonlocal family: projection, coupling and expansion, plus the packing of C' when the
    # tensor engine expands from packed operands (2 n_pj <= 40, ldx = nvec)
    packed = (ctx32[0].nonlocal_engine() == 1 and prob.atoms
              and 2 * max(a.npj for a in prob.atoms) <= 40)
    launches = fams["hx_local"][1] + (4 if packed else 3) * fams["nonlocal"][1] + fams["cheb"][1]
    launches += (degree % 2) * len(ks) * args.steps      # final block copy for odd degree
    tot = sum(v[0] for v in fams.values()) or 1.0
    kernels = {k: {"ms_total": round(v[0], 3), "launches": v[1],
                   "avg_ms": round(v[0] / v[1], 4) if v[1] else None,
                   "share": round(v[0] / tot, 4)} for k, v in fams.items() if v[1]}
    loc = fams["hx_local"]
    avg_local_ms = loc[0] / loc[1]
    kpt = any(abs(x) > 0 for k in ks for x in k)
    flops_launch = flops_per_cell_vector(prob.p, prob.nq, kpt) * prob.ncells * nvec
    clocks = clk.summary()
    fp32 = [v for k, v in peaks.items() if k in ("ffma", "ffma2") and isinstance(v, float)]
    if fp32:
        peak_alu = max(fp32)
        peak_note = ("of measured: FP32 FMA probe (gbc_alu_peak ffma / ffma2, best of three "
                     "launches) on this GPU in this run")
    else:
        peak_alu = 152 * 128 * 2 * 2.07e9 / 1e12
        peak_note = "derived (probe failed): 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"
    var, vb, nt = ctx32[0].cell_variant()
    traffic, traffic_note = None, "no ncu capture of this kernel version"
    if args.config == "cube16_p6":
        traffic, traffic_note = CELL_TRAFFIC(nvec, var)
    roofline = {"bound": "alu",
                "kernel": f"hx_cell_kernel<7,8,k!=0,VB={vb},NT={nt}> variant {var} (even-odd sum "
                          "factorisation, recurrence fused for cell-interior nodes)",
                "achieved": round(flops_launch / (avg_local_ms / 1e3) / 1e12, 3),
                "peak": round(peak_alu, 2), "unit": "TFLOP/s",
                "frac": round(flops_launch / (avg_local_ms / 1e3) / 1e12 / peak_alu, 4),
                "traffic": traffic,
                "traffic_note": traffic_note,
                "peak_note": peak_note,
                "flops_per_launch": flops_launch}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "config": args.config, "nodes": M, "nvec": nvec,
                      "degree": degree, "kpoints": len(ks), "precision": "FP32 filter (complex64)",
                      "l2": "inputs larger than L2 (3.6 GB per k-point block, 126 MB L2)",
                      "parallelism": f"replicas x{world}",
                      "nonlocal_engine": ["simt", "tensor"][ctx32[0].nonlocal_engine()]},
           "roofline": roofline, "clocks": clocks, "gpu_launches": launches,
           "kernels": kernels, "peaks_measured_tflops": peaks}

    # ---- end to end through the C ABI with host buffers (copies inside the timed region):
    # each k-point block is uploaded on a copy stream, filtered on the compute stream once
    # its upload is done, and read back on a second copy stream once its filter is done, so
    # the copies of one block overlap the filters of its neighbours
    def e2e_pipelined():
        host = [torch.empty(X.shape, dtype=X.dtype, pin_memory=True) for X in X32]
        for h, X in zip(host, X32):
            h.copy_(X)
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        nk = len(X32)
        ev_in = [torch.cuda.Event() for _ in range(nk)]
        ev_f = [torch.cuda.Event() for _ in range(nk)]
        ev_out = [torch.cuda.Event() for _ in range(nk)]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nrep = max(1, min(args.steps, 2))
        e0.record(stream)
        s_in.wait_stream(stream)
        s_out.wait_stream(stream)
        for r in range(nrep):
            with torch.cuda.stream(s_in):
                for i in range(nk):
                    if r > 0:                 # the block's previous read-back must be done
                        s_in.wait_event(ev_out[i])
                    X32[i].copy_(host[i], non_blocking=True)
                    ev_in[i].record(s_in)
            for i, (c, (lT, lmax, lmin)) in enumerate(zip(ctx32, bounds)):
                stream.wait_event(ev_in[i])
                c.filter(X32[i], degree, lT, lmax, lmin, stream=stream)
                ev_f[i].record(stream)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_f[i])
                    host[i].copy_(X32[i], non_blocking=True)
                    ev_out[i].record(s_out)
        stream.wait_stream(s_out)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = dist_max(e0.elapsed_time(e1), device="cuda" if world > 1 else "cpu") / nrep
        nbytes = sum(X.numel() * X.element_size() for X in X32)
        return {"value": dist_sum(units_per_step, "cuda" if world > 1 else "cpu") / (ms_e2e / 1e3),
                "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                "ms_per_step": ms_e2e,
                "how": "pinned host blocks; per k-point: upload on a copy stream, filter on the "
                       "compute stream, read-back on a second copy stream, ordered by events "
                       "(copies overlap the neighbouring filters)"}

    def e2e_sequential():
        host = [torch.empty(X.shape, dtype=X.dtype, pin_memory=True) for X in X32]
        for h, X in zip(host, X32):
            h.copy_(X)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nrep = max(1, min(args.steps, 2))
        e0.record(stream)
        for _ in range(nrep):
            for c, X, h, (lT, lmax, lmin) in zip(ctx32, X32, host, bounds):
                X.copy_(h, non_blocking=True)
                c.filter(X, degree, lT, lmax, lmin)
                h.copy_(X, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = dist_max(e0.elapsed_time(e1), device="cuda" if world > 1 else "cpu") / nrep
        nbytes = sum(X.numel() * X.element_size() for X in X32)
        return {"value": dist_sum(units_per_step, "cuda" if world > 1 else "cpu") / (ms_e2e / 1e3),
                "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                "ms_per_step": ms_e2e,
                "how": "pinned host blocks; per k-point: upload, filter, read-back in order on "
                       "one stream"}

    if not args.no_e2e:
        try:
            out["e2e"] = e2e_pipelined()
        except Exception as exc:   # keep an end-to-end number: the one-stream form
            torch.cuda.synchronize()
            out["e2e"] = e2e_sequential()
            out["e2e"]["pipelined_error"] = f"{type(exc).__name__}: {exc}"

    # ---- the cell apply on the tensor cores (precision paths TF32 and BF16x3): one H.X of
    # the k-point-0 block per precision, the cell-apply family's CUDA-event time against the
    # FP32 SIMT kernel's, dense products counted as computed (tensor work x3 for BF16x3)
    if not args.no_tc and rank == 0:
        try:
            out["tc_cell"] = tc_cell_leg(g, prob, ks[0], X32[0], nvec, peaks, avg_local_ms)
        except Exception as exc:   # an auxiliary leg must not cost the headline line
            out["tc_cell"] = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- batch16 (config 2): sixteen uneven systems, one batched filter call per step
    if not args.no_batch16 and rank == 0:
        try:
            r = batch16_measure(g, syn, args, steps=3, warmup=2)
            r.pop("systems")
            out["batch16"] = r
        except Exception as exc:   # an auxiliary leg must not cost the headline line
            out["batch16"] = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- densities rho, m at the Gauss points from the filtered block (Eqs. rho, mag):
    # one gbc_density_dev launch on device-resident inputs, Fermi-Dirac occupations of the
    # block's Ritz values (N_e = nvec / 2 electrons, 500 K), timed with CUDA events
    if not args.no_density and rank == 0:
        try:
            c, X = ctx32[0], X32[0]
            nq3 = prob.nq ** 3
            kt_500k = 500.0 * 3.166811563e-6             # Ha
            f_h, mu = g.fermi_occupations(ritz_k[0][None, :], None, nvec / 2, kt_500k)
            occ = torch.from_numpy(np.ascontiguousarray(f_h[0])).cuda()
            dens = torch.empty((prob.ncells, 4, nq3), dtype=torch.float64, device="cuda")
            for _ in range(3):
                c.density_dev(X, occ, dens)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            nrep = 5
            e0.record(stream)
            for _ in range(nrep):
                c.density_dev(X, occ, dens)
            e1.record(stream)
            torch.cuda.synchronize()
            c.sync_status()
            ms_d = e0.elapsed_time(e1) / nrep
            npp, nq = prob.p + 1, prob.nq
            # sum-factorised interpolation to the Gauss points (2 spins x re/im, 3 stages) plus
            # the 22 FP32 operations of the four spin products per point
            fl_cv = 2 * 4 * npp * nq * (npp * npp + npp * nq + nq * nq) + 22 * nq3
            fl = fl_cv * prob.ncells * nvec
            by = M * 2 * nvec * X.element_size() + dens.numel() * 8
            out["density"] = {
                "ms": round(ms_d, 4), "kernel": "quad_grad_kernel<float,7,8,2> point-wise",
                "flops_per_launch": fl, "achieved_tflops": round(fl / (ms_d / 1e3) / 1e12, 2),
                "frac_alu": round(fl / (ms_d / 1e3) / 1e12 / peak_alu, 4),
                "algorithmic_bytes": by, "achieved_gbs": round(by / (ms_d / 1e3) / 1e9, 1),
                "occupations": f"Fermi-Dirac, N_e = {nvec / 2:g}, 500 K, mu = {mu:.6f} Ha "
                               "(gbc_fermi_occupations on the k-point-0 Ritz values)",
                "how": f"cube16_p6 k-point 0 filtered block ({nvec} vectors, FP32), {nrep} launches after 3 "
                       "warm-up, CUDA events; bytes = X read once + rho/m written (FP64)"}
        except Exception as exc:   # an auxiliary leg must not cost the headline line
            out["density"] = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- two-grid transfer (Eq. FEWfnsCMesh): the order-5 block of the same mesh carried to
    # order 6 (the bench mesh), 256 vectors FP32, device-resident, CUDA events
    if not args.no_twogrid and rank == 0 and prob.p > 2:
        try:
            pc = prob.p - 1
            cc = g.Context(torch.cuda.current_device())
            cc.set_mesh(prob.ncell, prob.h, pc, pc + 2, prob.periodic)
            cc.set_precision(g.FP32)
            xc = torch.randn((cc.nnodes, 2, nvec), dtype=torch.complex64, device="cuda")
            xf = torch.empty_like(X32[0])
            c = ctx32[0]
            for _ in range(3):
                c.prolongate_from(cc, xc, xf)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            nrep = 5
            e0.record(stream)
            for _ in range(nrep):
                c.prolongate_from(cc, xc, xf)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_t = e0.elapsed_time(e1) / nrep
            by = (xc.numel() + xf.numel()) * xf.element_size()
            peak, peak_src = hbm_peak()
            gbs = by / (ms_t / 1e3) / 1e9
            out["twogrid"] = {
                "ms": round(ms_t, 4), "kernel": f"k_prolongate<float,{pc + 1},{prob.p + 1},8>",
                "algorithmic_bytes": by, "achieved_gbs": round(gbs, 1),
                "frac_hbm": round(gbs / peak, 4), "peak_gbs": peak, "peak_note": peak_src,
                "how": f"order {pc} -> {prob.p} on the bench mesh, {nvec} vectors FP32, {nrep} "
                       "launches after 3 warm-up; bytes = coarse block read once + fine block "
                       "written once"}
            cc.close()
            del xc, xf
        except Exception as exc:   # an auxiliary leg must not cost the headline line
            out["twogrid"] = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- SCF steps (Sec. III.B.1) over the 4 k-points: fields from the densities, one ChFSI
    # cycle per k-point, one Fermi level, Brillouin-zone-summed densities, Anderson mixing;
    # wall time per step with CUDA events
    if args.scf_steps > 0 and rank == 0:
        try:
            from paper_2410_02754_gb300 import scf as gscf
            vext = torch.from_numpy(np.ascontiguousarray(prob.veff)).cuda()
            nk = len(ctx32)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            res = gscf.scf_loop_k(ctx32, X32, vext, [v0] * nk, [1.0 / nk] * nk, nelec=nvec / 2,
                                  kT=500.0 * 3.166811563e-6, degree=degree,
                                  lanczos_steps=cfg["lanczos"], alpha=0.5, nhist=4,
                                  iters=args.scf_steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_scf = e0.elapsed_time(e1)
            out["scf"] = {
                "ms_per_step": round(ms_scf / args.scf_steps, 1), "steps": args.scf_steps,
                "kpoints": nk, "residual_norms": [float(r) for r in res["res"]],
                "how": f"{nk} k-points (weight 1/{nk}), FP32 blocks of {nvec} vectors, degree "
                       f"{degree}, N_e = {nvec / 2:g}, 500 K, Anderson alpha 0.5 over 4 pairs; "
                       "the time includes the initial CholGS + Rayleigh-Ritz of every k-point"}
        except Exception as exc:   # an auxiliary leg must not cost the headline line
            out["scf"] = {"error": f"{type(exc).__name__}: {exc}"}
        finally:                   # the accuracy leg below uses these contexts' original H
            for c in ctx32:
                try:
                    c.set_fields(prob.veff, prob.bx, prob.by, prob.bz)
                except Exception as exc:
                    out.setdefault("scf", {})["restore_error"] = f"{type(exc).__name__}: {exc}"

    # ---- FP64 filter and accuracy of the mixed path at the same inputs (k-point 0):
    # three chains from the same seeded block -- FP64, mixed direct, mixed residual-split --
    # each cycle 0 (CholGS + RR) then ``--cycles`` x (filter, CholGS, RR); CholGS/RR
    # run in FP64 in every chain.
    if not args.no_fp64 and rank == 0:
        c64 = build_contexts(g, prob, ks[:1], g.FP64)[0]
        c32 = ctx32[0]
        lo, hi = c64.lanczos_bounds(v0, cfg["lanczos"])
        chains = {"fp64": (c64, torch.from_numpy(X0).cuda()),
                  "mixed_direct": (c32, torch.from_numpy(X0).to(torch.complex64).cuda()),
                  "mixed_split": (c32, torch.from_numpy(X0).to(torch.complex64).cuda())}
        ritz = {}
        for name, (c, X) in chains.items():
            c.cholgs(X)
            ritz[name] = c.rayleigh_ritz(X)
        half = nvec // 2
        per_cycle = {"mixed_direct": [], "mixed_split": []}
        fp64_moves = []   # how far the FP64 chain's own Ritz values still move per cycle
        ms = {"fp64": [], "mixed_direct": [], "mixed_split": []}
        ms_cycle = {"fp64": [], "mixed_direct": [], "mixed_split": []}
        for cyc in range(args.cycles):
            prev64 = np.asarray(ritz["fp64"]).copy()
            for name, (c, X) in chains.items():
                r = ritz[name]
                lT, lmn = float(r[-1]), min(lo, float(r[0]))
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if name == "mixed_split":
                    c.filter_residual(X, degree, lT, hi, lmn, r)
                else:
                    c.filter(X, degree, lT, hi, lmn)
                e1.record(stream)
                c.cholgs(X)
                ritz[name] = c.rayleigh_ritz(X)   # synchronises (Ritz values to the host)
                e2 = torch.cuda.Event(enable_timing=True)
                e2.record(stream)
                torch.cuda.synchronize()
                ms[name].append(e0.elapsed_time(e1))
                ms_cycle[name].append(e0.elapsed_time(e2))
            for name in per_cycle:
                per_cycle[name].append(float(np.abs(ritz[name] - ritz["fp64"])[:half].max()))
            fp64_moves.append(float(np.abs(np.asarray(ritz["fp64"]) - prev64)[:half].max()))
        ms64 = min(ms["fp64"])
        out["fp64"] = {"value": M * nvec * degree / (ms64 / 1e3), "unit": UNIT,
                       "ms_per_filter": ms64,
                       "mixed_over_fp64": value / (M * nvec * degree / (ms64 / 1e3))}
        out["accuracy"] = {
            "ritz_maxdiff_vs_fp64_ha_lower_half_per_cycle": per_cycle,
            "fp64_chain_change_ha_lower_half_per_cycle": fp64_moves,
            "reading": "the target applies to converged Ritz values; while the FP64 chain's own "
                       "values still move by more than 1e-6 Ha per cycle, the two chains are "
                       "compared before convergence",
            "final_ha": {k: v[-1] for k, v in per_cycle.items()} if args.cycles else None,
            "target_ha": 1e-6,
            "how": f"k-point 0, cycle 0 + {args.cycles} x (filter degree {degree}, CholGS, RR); "
                   "CholGS/RR in FP64 in every chain; lower half of the block",
            "ms_per_filter": {k: round(min(v), 2) for k, v in ms.items() if v},
            "ms_per_cycle": {k: round(min(v), 2) for k, v in ms_cycle.items() if v},
            "cycle_note": "filter + CholGS + Rayleigh-Ritz (the latter two in FP64 in every chain)",
            "lowest_ritz_ha": [float(x) for x in ritz["fp64"][:4]]}
        c64.close()

    # ---- slab40_p6 (the semi-periodic slab, 6.85M nodes, 640 atoms): one 32-vector block
    # at degree 30 in FP32 and in FP64 from the same seeded block, and the Ritz-value
    # difference after one filter + CholGS + RR (the full 256-vector block: --config slab40_p6)
    if not args.no_slab and rank == 0:
        try:
            torch.cuda.empty_cache()
            r = slab_measure(g, syn, torch.cuda.current_device(), 32, syn.CONFIGS["slab40_p6"]["degree"],
                             3, 1)
            out["slab"] = {
                "value": r["units"] / (r["ms32"] / 1e3), "unit": UNIT, "ms_per_filter": r["ms32"],
                "fp64": {"value": r["units"] / (r["ms64"] / 1e3), "ms_per_filter": r["ms64"],
                         "mixed_over_fp64": r["ms64"] / r["ms32"]},
                "ritz_maxdiff_vs_fp64_ha_lower_half": r["ritz_maxdiff_vs_fp64_ha_lower_half"],
                "target_ha": 1e-6, "nonlocal_engine": r["engine"], "clocks": r["clocks"],
                "how": f"40x40x20 cells, p = 6 ({r['nodes']:,} nodes), periodic x/y, Dirichlet z, "
                       "640 atoms x 18 SOC projectors, one 32-vector block, degree "
                       f"{syn.CONFIGS['slab40_p6']['degree']}, Gamma; FP32 = median of 3 filters "
                       "after 1 warm-up, FP64 = one filter; cycle 0 (CholGS + RR) before, "
                       "CholGS + RR after, lower half of the block"}
        except Exception as exc:   # an auxiliary leg must not cost the headline line
            out["slab"] = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- CPU baseline: the oracle as it stands, bounded sample (rank 0, N = 1)
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_sample(args, prob, ks[0], budget_s=args.cpu_budget)

    for c in ctx32:
        c.close()
    if rank == 0:
        print(json.dumps(out), flush=True)


def batch16_measure(g, syn, args, clock_index=None, steps=None, warmup=None):
    """batch16: sixteen uneven systems (8^3..14^3 cells, p in {4, 5, 6}, 64..320 vectors,
    8..40 atoms, degree 12..24) filtered by one batched call per step: per degree one
    persistent cell-apply launch per group of systems sharing order, cell edges and
    k-point, their nonlocal steps and one face-row recurrence launch, the whole degree
    loop replayed as a CUDA graph; beside it the same work as one gbc_filter call per
    system."""
    import torch
    descs = syn.batch16_systems(0)
    ctxs, blocks, bounds, degrees, units = [], [], [], [], 0
    for d in descs:
        prob = syn.batch16_problem(d)
        c = g.Context(torch.cuda.current_device())
        c.set_problem(prob)
        c.set_precision(g.FP32)
        c.set_nonlocal_engine(args.nl_engine)
        c.tune(d["nvec"])
        M = prob.nnodes
        v0 = torch.from_numpy(syn.random_start(M, d["seed"])).cuda()
        lo, hi = c.lanczos_bounds(v0, 10)
        X = torch.from_numpy(syn.random_block(M, d["nvec"], d["seed"])).to(torch.complex64).cuda()
        c.cholgs(X)
        r = c.rayleigh_ritz(X)
        ctxs.append(c)
        blocks.append(X)
        bounds.append((float(r[-1]), hi, min(lo, float(r[0]))))
        degrees.append(d["degree"])
        units += M * d["nvec"] * d["degree"]
    steps = steps or args.steps
    warmup = warmup if warmup is not None else args.warmup
    batch = g.Batch(ctxs)
    stream = torch.cuda.Stream()
    clocks = None
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            batch.filter(blocks, degrees, bounds, stream)
        stream.synchronize()
        dist_barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(clock_index) if clock_index is not None else None
        if sampler:
            sampler.__enter__()
        e0.record(stream)
        for _ in range(steps):
            batch.filter(blocks, degrees, bounds, stream)
        e1.record(stream)
        stream.synchronize()
        if sampler:
            sampler.__exit__()
            clocks = sampler.summary()
        ms = e0.elapsed_time(e1) / steps
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for c, X, dg, b in zip(ctxs, blocks, degrees, bounds):
            c.filter(X, dg, *b, stream=stream)
        s1.record(stream)
        stream.synchronize()
        ms_seq = s0.elapsed_time(s1)
    for c in ctxs:
        c.sync_status()
    res = {"units_per_step": units, "ms_per_step": ms, "value": units / (ms / 1e3), "unit": UNIT,
           "systems": descs, "batched_graph_kernels_per_step": batch.launches(),
           "tiles": [c.tile() for c in ctxs], "unbatched_ms_per_step": ms_seq,
           "batching_speedup": ms_seq / ms, "clocks": clocks,
           "how": f"{steps} batched filter calls after {warmup} warm-up, CUDA events on the "
                  "batch stream; unbatched = one gbc_filter per system on the same stream"}
    batch.close()
    for c in ctxs:
        c.close()
    return res


def run_batch(args):
    """The batch16 workload as the bench line (--config batch16)."""
    import __graft_entry__ as ge
    import synthetic as syn
    import paper_2410_02754_gb300 as g
    import torch

    rank, world = dist_init("nccl" if int(os.environ.get("WORLD_SIZE", "1")) > 1 else "gloo")
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    ge.build()
    r = batch16_measure(g, syn, args, clock_index=local)
    ms = dist_max(r["ms_per_step"], "cuda" if world > 1 else "cpu")
    value = dist_sum(r["units_per_step"], "cuda" if world > 1 else "cpu") / (ms / 1e3)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "16 uneven periodic systems, 8^3..14^3 cells, p in {4,5,6}, "
                                  "64..320 vectors, 8..40 atoms x 18 projectors, degree 12..24",
                      "config": "batch16", "systems": r["systems"],
                      "l2": "inputs larger than L2"},
           "batched_graph_kernels_per_step": r["batched_graph_kernels_per_step"],
           "tiles": r["tiles"], "unbatched_ms_per_step": r["unbatched_ms_per_step"],
           "batching_speedup": r["batching_speedup"], "clocks": r["clocks"]}
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_backward(args):
    """cube16_p6_grad: the cube16_p6 mesh and atoms at the Gamma point, 128 vectors, degree 20: one
    step = FP32 forward filter + energy gradient (G_Y = 2 H Y W) + the backward of the
    filter (gbc_filter_vjp, checkpoints every 5 degrees) giving dL/dX, dL/dV_eff,
    dL/dB_xc at the quadrature points and dL/dDelta."""
    import numpy as np
    import torch

    import __graft_entry__ as ge
    import synthetic as syn
    import paper_2410_02754_gb300 as g

    rank, world = dist_init("nccl" if int(os.environ.get("WORLD_SIZE", "1")) > 1 else "gloo")
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    ge.build()
    cfg = syn.CONFIGS["cube16_p6_grad"]
    nvec = args.nvec or cfg["nvec"]
    degree = args.degree or cfg["degree"]
    prob = syn.config("cube16_p6_grad", seed=0)
    M = prob.nnodes
    c = g.Context(torch.cuda.current_device())
    c.set_problem(prob)
    c.set_precision(g.FP32)
    c.set_nonlocal_engine(args.nl_engine)
    lo, hi = c.lanczos_bounds(torch.from_numpy(syn.random_start(M, 0)).cuda(), cfg["lanczos"])
    X0 = torch.from_numpy(syn.random_block(M, nvec, 0)).to(torch.complex64).cuda()
    c.cholgs(X0)
    ritz = c.rayleigh_ritz(X0)
    lT, lmin = float(ritz[-1]), min(lo, float(ritz[0]))
    w = np.random.default_rng(5).uniform(0.0, 1.0, nvec)
    X = torch.empty_like(X0)
    GY = torch.empty_like(X0)
    GX = torch.empty_like(X0)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        X.copy_(X0)
        c.filter(X, degree, lT, hi, lmin)
        if ev:
            ev[0].record(stream)
        c.energy_grad(X, w, GY)
        c.filter_vjp(X0, GY, GX, degree, lT, hi, lmin, ckpt_every=5)
        if ev:
            ev[1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dist_barrier()
    t_fwd, t_bwd = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            step((e1, e2))
            torch.cuda.synchronize()
            t_fwd.append(e0.elapsed_time(e1))
            t_bwd.append(e1.elapsed_time(e2))
    ms_fwd, ms_bwd = float(np.mean(t_fwd)), float(np.mean(t_bwd))
    ms = dist_max(ms_fwd + ms_bwd, "cuda" if world > 1 else "cpu")
    units = M * nvec * degree
    out = {"metric": "ChFSI filter forward + backward spinor-DOF\u00b7vectors\u00b7degree/s, 1 GB300",
           "value": dist_sum(units, "cuda" if world > 1 else "cpu") / (ms / 1e3), "unit": UNIT,
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": f"16x16x16 periodic cells, p=6, nq=8 ({M:,} nodes), 64 atoms x 18 "
                                  f"SOC projectors, {nvec} vectors, degree {degree}, Gamma point; "
                                  "L = sum_i w_i y_i^H H y_i",
                      "config": "cube16_p6_grad", "checkpoint_every": 5},
           "ms_forward_filter": ms_fwd, "ms_backward": ms_bwd,
           "backward_over_forward": ms_bwd / ms_fwd,
           "backward_note": "energy gradient + filter VJP, gradients copied to the host",
           "clocks": clk.summary()}
    c.close()
    if rank == 0:
        print(json.dumps(out), flush=True)


def slab_measure(g, syn, local, nvec, degree, steps, warmup):
    """The slab40_p6 mesh and atoms (40x40x20 cells, p = 6, 6,854,400 nodes, 640 atoms): one
    block of ``nvec`` vectors filtered to ``degree`` in FP32 and in FP64 from the same seeded
    block: cycle 0 (CholGS + Rayleigh-Ritz), the timed filters (FP32: median of ``steps``
    after ``warmup``; FP64: one), then CholGS + Rayleigh-Ritz and the Ritz-value difference
    of the lower half.  The block is drawn on the device from a seeded generator (uniform
    [-1, 1) parts), once per precision from the same seed."""
    import numpy as np
    import torch

    cfg = syn.CONFIGS["slab40_p6"]
    prob = syn.config("slab40_p6", seed=0)
    M = prob.nnodes
    v0 = torch.from_numpy(syn.random_start(M, 0)).cuda()
    stream = torch.cuda.current_stream()
    def block(dtype):
        gen = torch.Generator(device="cuda")
        gen.manual_seed(1234)
        re = torch.rand((M, 2, nvec), generator=gen, dtype=torch.float64, device="cuda") * 2 - 1
        im = torch.rand((M, 2, nvec), generator=gen, dtype=torch.float64, device="cuda") * 2 - 1
        X = torch.complex(re, im).to(dtype)
        del re, im
        # the FP64 temporaries (up to 112 GB) go back to the driver: the library allocates
        # its work blocks with cudaMalloc, outside torch's caching allocator
        torch.cuda.empty_cache()
        return X

    def run(prec, dtype, nrep):
        c = g.Context(local)
        c.set_problem(prob)
        c.set_precision(prec)
        if prec == g.FP32:
            c.tune(nvec)
        lo, hi = c.lanczos_bounds(v0, cfg["lanczos"])
        X = block(dtype)
        c.cholgs(X)
        ritz = c.rayleigh_ritz(X)
        lT, lmin = float(ritz[-1]), min(lo, float(ritz[0]))
        # each timed filter starts from the cycle-0 block (restored outside the timed region);
        # with nrep = 1 the block is filtered in place (no second copy of a 56 GB FP64 block)
        Xw = X.clone() if nrep > 1 else X
        for _ in range(warmup if nrep > 1 else 0):
            Xw.copy_(X)
            c.filter(Xw, degree, lT, hi, lmin)
        times = []
        with ClockSampler(local) as clk:
            for _ in range(nrep):
                if Xw is not X:
                    Xw.copy_(X)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                c.filter(Xw, degree, lT, hi, lmin)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
        ms = float(np.median(times))
        del X
        c.cholgs(Xw)
        r = c.rayleigh_ritz(Xw)
        c.sync_status()
        engine = ["simt", "tensor"][c.nonlocal_engine()] if prec == g.FP32 else "simt"
        c.close()
        del Xw
        torch.cuda.empty_cache()
        return ms, np.asarray(r), clk.summary(), engine

    ms32, r32, clocks, engine = run(g.FP32, torch.complex64, steps)
    ms64, r64, _, _ = run(g.FP64, torch.complex128, 1)
    units = M * nvec * degree
    half = nvec // 2
    return {"units": units, "nodes": M, "ms32": ms32, "ms64": ms64, "engine": engine,
            "clocks": clocks,
            "ritz_maxdiff_vs_fp64_ha_lower_half": float(np.abs(r32 - r64)[:half].max())}


def run_slab(args):
    """slab40_p6: the 40x40x20-cell semi-periodic slab (6,854,400 nodes, 640 atoms), measured
    as the per-block filter throughput of one 256-vector block at degree 30 (the 20,000 states
    are 79 such blocks, which do not fit the GPU together), FP32 against FP64 on the same
    block (slab_measure)."""
    import torch

    import __graft_entry__ as ge
    import synthetic as syn
    import paper_2410_02754_gb300 as g

    rank, world = dist_init("nccl" if int(os.environ.get("WORLD_SIZE", "1")) > 1 else "gloo")
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    ge.build()
    cfg = syn.CONFIGS["slab40_p6"]
    nvec = args.nvec or cfg["nvec"]
    degree = args.degree or cfg["degree"]
    r = slab_measure(g, syn, local, nvec, degree, args.steps, args.warmup)
    M, units, ms32, ms64, engine, clocks = (r["nodes"], r["units"], r["ms32"], r["ms64"],
                                            r["engine"], r["clocks"])
    out = {"metric": METRIC + " (slab, per 256-vector block)", "value": units / (ms32 / 1e3),
           "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"40x40x20 cells, p=6, nq=8 ({M:,} nodes), periodic x/y, "
                                  f"Dirichlet z, 640 atoms x 18 SOC projectors, one block of "
                                  f"{nvec} of the 20,000 states, degree {degree}, Gamma",
                      "config": "slab40_p6", "nonlocal_engine": engine,
                      "l2": "inputs larger than L2 (28 GB FP32 block)"},
           "fp64": {"value": units / (ms64 / 1e3), "ms_per_filter": ms64,
                    "mixed_over_fp64": ms64 / ms32},
           "accuracy": {"ritz_maxdiff_vs_fp64_ha_lower_half": r["ritz_maxdiff_vs_fp64_ha_lower_half"],
                        "target_ha": 1e-6,
                        "how": "cycle 0, one filter, CholGS, Rayleigh-Ritz, from the same seeded "
                               "block in each precision; FP32 time = median of the timed "
                               "filters, FP64 = one filter"},
           "clocks": clocks}
    if rank == 0:
        print(json.dumps(out), flush=True)


def cpu_sample(args, prob, k, budget_s=20.0, nv=2):
    """One recurrence step (H.X by element-by-element quadrature + the sigma-scaled
    update) of the FP64 oracle on an nv-vector sample of the workload."""
    import numpy as np

    import synthetic as syn
    from oracle import fe

    d = fe.Discretisation(prob.with_(k=k))
    M = d.mesh.nnodes
    X = syn.random_block(M, nv, 1)
    Xp = syn.random_block(M, nv, 2)
    t0 = time.perf_counter()
    reps = 0
    while True:
        Y = d.apply_htilde(X)
        _ = 0.1 * (Y - 3.0 * X) - 0.5 * Xp
        reps += 1
        if time.perf_counter() - t0 > budget_s or reps >= 50:
            break
    dt = (time.perf_counter() - t0) / reps
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": M * nv / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} x one recurrence step (FP64 O1b H.X + update), {nv} vectors, "
                      f"full mesh ({M} nodes), k-point 0; numpy/BLAS threads over all cores",
            "seconds": round(dt * reps, 2)}


def run_reference(args):
    """The FP64 CPU oracle as it stands, on this arm's config/metric, rank 0 only."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import synthetic as syn
    if args.config not in syn.CONFIGS:
        print(json.dumps({"impl": "reference", "unavailable":
                          f"the oracle arm times single-problem workloads; {args.config} is not one"}),
              flush=True)
        return
    cfg = syn.CONFIGS[args.config]
    prob = syn.config(args.config, seed=0)
    ks = syn.mp_kpoints(*cfg["kgrid"], prob.box)
    budget = max(2.0, min(30.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_sample(args, prob, ks[0], budget_s=budget / 4)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_sample(args, prob, ks[0], budget_s=budget))
    wall = time.perf_counter() - t0
    v = sum(x["value"] for x in vals) / len(vals)
    cb = dict(vals[-1])
    cb["value"] = v
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "config": args.config},
           "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                                       "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbchfsi", choices=["gbchfsi", "reference"])
    ap.add_argument("--config", default="cube16_p6")
    ap.add_argument("--kpoints", type=int, default=0, help="use only the first K k-points")
    ap.add_argument("--nvec", type=int, default=0, help="override the block size (profiling runs)")
    ap.add_argument("--degree", type=int, default=0, help="override the degree (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-density", action="store_true")
    ap.add_argument("--no-twogrid", action="store_true")
    ap.add_argument("--no-tc", action="store_true", help="skip the tensor-core cell-apply leg")
    ap.add_argument("--no-batch16", action="store_true", help="skip the batch16 leg")
    ap.add_argument("--no-slab", action="store_true", help="skip the slab40_p6 leg")
    ap.add_argument("--scf-steps", type=int, default=2, help="SCF steps of the scf leg (0: off)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--cycles", type=int, default=3, help="ChFSI cycles of the accuracy leg")
    ap.add_argument("--nl-engine", type=int, default=1, choices=[0, 1],
                    help="FP32 projector contractions: 0 SIMT cores, 1 tcgen05 tensor cores")
    ap.add_argument("--cell-variant", type=int, default=-1,
                    help="FP32 cell-apply variant of the main leg (profiling runs; -1: the tuner's)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "batch16":
        run_batch(args)
    elif args.config == "slab40_p6":
        run_slab(args)
    elif args.config == "cube16_p6_grad":
        run_backward(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
