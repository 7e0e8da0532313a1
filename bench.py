#!/usr/bin/env python3
"""Benchmark: Wilson-Dirac site-updates/s inside a mixed-precision CG solve to 1e-10.

Workload (one GPU): 32^4 periodic lattice (1,048,576 sites), m_q = 0.05, links
exp(0.3 i H) with H random traceless Hermitian (near the free field, the ill-conditioned
case), one Gaussian right-hand side.  One step = one full solve of D^dag D x = eta from
x = 0 with Algorithm 1: link packing to the inner format, FP64 residual, inner CG in
FP32 arithmetic (scaled-FP16 or FP32 storage, 12-real links, EO layout), FP64 reliable
updates, until the FP64 true residual is <= 1e-10 ||eta||.

value = Wilson-Dirac site-updates per second over the whole solve: every application of
D or D^dag to a full lattice counts V site-updates (inner and FP64 applies alike).
The line also carries the CG time-to-1e-10 of the mixed solver and of the plain FP64 CG
on the same inputs, the roofline of the dominant kernel, the CPU oracle's rate on a
bounded sample, and an end-to-end number with host buffers.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): every rank solves its own system (weak scaling, no collective on
the data path); value = all ranks' site-updates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (32, 32, 32, 32)
MASS = 0.05
EPS = 0.3
TOL = 1e-10
SEED_U, SEED_ETA = 3, 4
FLOPS_PER_SITE = 1464            # the paper's nominal count per stencil (Introduction)
# both arms (the library and the CPU oracle) report this metric; the workload says what a step is
METRIC = "Dslash site-updates/s"
WORKLOAD = "mixed-precision CG to 1e-10 on 32^4, m_q=0.05, links exp(0.3iH)"

# algorithmic bytes per site of the inner-loop kernels (each field read or written once)
#   K1: p in, 4 links, t out.  K2: t in, 4 links, p, psi, r in, psi, r out.  K3: r, p in, p out.
SPINOR_B = {"mixed_f16": 52, "mixed_f32": 96, "f64": 192, "f64x": 192, "mixed_i32": 100}
LINK4_B = {"mixed_f16": 96, "mixed_f32": 192, "f64": 576, "f64x": 576, "mixed_i32": 192}
# the inner solution psi is kept in FP32 when the other inner vectors are scaled FP16
PSI_B = {"mixed_f16": 96}


def kernel_bytes(mode):
    s, l = SPINOR_B[mode], LINK4_B[mode]
    x = PSI_B.get(mode, s)
    # K2 reads t, p, r and psi (in the psi precision) and the links, writes psi and r
    return {"K1": 2 * s + l, "K2": 4 * s + 2 * x + l, "K3": 3 * s}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the files the inner-loop kernels (K1, K2, K3 of the single-lattice solver) are built from
KERNEL_SOURCES = ("lq_internal.cuh", "dd.cuh", "dslash_kernels.cuh", "dslash_dispatch.cuh", "solver_impl.cuh",
                  "solver_f16.cu", "solver_f32.cu", "solver_f64.cu")


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1904_08616_gb300", "csrc")
    for fn in KERNEL_SOURCES:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_role):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current kernel sources (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            d = json.load(f)
        if d.get("source_hash") != source_hash():
            return None
        return d["kernels"][kernel_role]["dram_bytes_per_launch_full_size"]
    except Exception:
        return None


class ClockSampler:
    def __init__(self, gpu_index):
        self.proc = None
        # the raw samples go to $LQ_BENCH_OUT (default: bench_out/ beside this file)
        out = os.environ.get("LQ_BENCH_OUT") or os.path.join(ROOT, "bench_out")
        self.path = os.path.join(out, f"clocks_rank{gpu_index}.csv")
        self.gpu = gpu_index

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
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
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
            sm = [float(r[1]) for r in rows]
            mx = max(float(r[2]) for r in rows)
            reasons = set()
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for r in rows:
                for i, n in enumerate(names):
                    if r[5 + i].strip().lower() == "active":
                        reasons.add(n)
            return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                    "samples": len(sm)}
        except Exception as e:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "error": str(e)[:80]}


def make_inputs():
    import synth
    U = synth.gauge_field(DIMS, seed=SEED_U, kind="near_identity", eps=EPS)
    eta = synth.gaussian_spinor(DIMS, seed=SEED_ETA)
    return U, eta


def oracle_rate(U, eta, nsites, reps=1, threads=1):
    """The CPU oracle (plain C) applying D^dag D's two stencils on nsites sampled sites of the
    same 32^4 fields, its loop over sites split over `threads` host cores; returns
    (site-updates/s, seconds, threads used)."""
    import numpy as np
    import oracle
    V = U.shape[0]
    sites = np.random.default_rng(0).integers(0, V, nsites)
    used = oracle.set_threads(threads)
    try:
        t0 = time.perf_counter()
        for _ in range(reps):
            oracle.dslash_sites(DIMS, MASS, U, eta, sites, dagger=False)
            oracle.dslash_sites(DIMS, MASS, U, eta, sites, dagger=True)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(1)
    return 2 * nsites * reps / dt, dt, used


def oracle_cg_times(all_rate, threads, f64_iters=None):
    """The oracle's textbook FP64 CG to 1e-10, timed on the host: the 4^4 Haar system
    (m_q = 0.1, one thread) and the 16^4 exp(0.5iH) system (m_q = 0.1, all cores), both run to
    the end; the 32^4 and 64^3x128 figures are projected as (two applies of D per iteration
    at the measured all-core site-update rate) x iterations, and labelled as such."""
    import oracle
    import synth
    out = {}
    for name, dims, kind, eps, m, seeds, thr in (("4^4 haar m_q=0.1", (4, 4, 4, 4), "haar", 0.0, 0.1, (1, 2), 1),
                                                 ("16^4 exp(0.5iH) m_q=0.1", (16, 16, 16, 16), "near_identity",
                                                  0.5, 0.1, (7, 8), threads)):
        U = synth.gauge_field(dims, seed=seeds[0], kind=kind, eps=eps)
        eta = synth.gaussian_spinor(dims, seed=seeds[1])
        used = oracle.set_threads(thr)
        try:
            t0 = time.perf_counter()
            _, it, rel = oracle.cg(dims, m, U, eta, tol=TOL)
            dt = time.perf_counter() - t0
        finally:
            oracle.set_threads(1)
        out[name] = {"s": dt, "iters": it, "true_rel_resid": rel, "cores": used, "kind": "measured"}
    per_iter_32 = 2 * 32 ** 4 / all_rate
    out["32^4 exp(0.3iH) m_q=0.05 (the bench system)"] = {
        "s_per_iter": per_iter_32, "cores": threads, "kind": "projected: 2 applies per iteration at the measured "
        "all-core rate x iterations of the FP64 CG on the same system",
        "iters": f64_iters, "s": per_iter_32 * f64_iters if f64_iters else None}
    out["64^3x128 haar m_q=0.02"] = {"s_per_iter": 2 * 64 ** 3 * 128 / all_rate, "cores": threads,
                                     "kind": "projected: 2 applies per iteration at the measured all-core rate"}
    return out


def run_reference(args, rank):
    if rank != 0:
        return
    import oracle
    U, eta = make_inputs()
    threads = oracle.max_threads()
    nsites = 1 << 19
    for _ in range(args.warmup):
        oracle_rate(U, eta, nsites, threads=threads)
    t0 = time.perf_counter()
    used = 1
    for _ in range(args.steps):
        _, _, used = oracle_rate(U, eta, nsites, threads=threads)
    dt = time.perf_counter() - t0
    value = 2 * nsites * args.steps / dt
    sample = (f"D and D^dag of Eq. 1 on {nsites} sampled sites of the 32^4 fields per step (FP64 C oracle, "
              f"site loop over {used} host cores)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "site-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": list(DIMS), "m_q": MASS},
        "cpu_baseline": {"value": value, "unit": "site-updates/s", "cores": used, "kind": "oracle", "sample": sample,
                         "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def whole_job_rate(ms, updates, device):
    """(slowest rank's ms, units all ranks processed per second over that time); one rank
    without an initialised process group returns its own figures."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        tm = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        tu = torch.tensor([float(updates)], dtype=torch.float64, device=device)
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        dist.all_reduce(tu, op=dist.ReduceOp.SUM)
        ms_max = float(tm.item())
        return ms_max, float(tu.item()) / (ms_max * 1e-3)
    return float(ms), float(updates) / (float(ms) * 1e-3)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist
    import paper_1904_08616_gb300 as lq
    import synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    lq.load()
    V = int(np.prod(DIMS))
    U, eta = make_inputs()
    # complex128 (V,4,3,3) / (V,4,3) arrays are byte-for-byte the FP64 LEX ABI fields
    Ub = synth.as_reals(U).view(np.uint8).reshape(-1)
    eb = synth.as_reals(eta).view(np.uint8).reshape(-1)
    U_h = torch.from_numpy(Ub.view(np.uint8)).pin_memory()
    eta_h = torch.from_numpy(eb.view(np.uint8)).pin_memory()
    x_h = torch.empty(eb.size, dtype=torch.uint8).pin_memory()
    U_d = U_h.to(dev)
    eta_d = eta_h.to(dev)
    x_d = torch.zeros_like(eta_d)
    mode = args.mode
    # one workspace large enough for every mode this run solves with
    ws = torch.empty(max(lq.cg_workspace_bytes(DIMS, m) for m in ("f64", "f64x", "mixed_f32", "mixed_f16", "mixed_i32")),
                     dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def solve(m, profile=False, native_f64=False):
        x_d.zero_()
        _, info, st = lq.cg_solve(DIMS, MASS, U_d, eta_d, x=x_d, mode=m, tol=TOL, workspace=ws,
                                  stream=stream, profile=profile, native_f64=native_f64)
        if st != 0:
            raise RuntimeError(f"solve did not converge: {info}")
        return info

    def fp64_residual():
        """||eta - D^dag D x|| / ||eta|| of the current x, through the library's native FP64
        operator kernels (LEX, 18-real links), independent of the solver's own residual."""
        t = lq.dslash_apply(DIMS, MASS, U_d, x_d, prec="f64", link_fmt=18, layout="lex", stream=stream)
        q = lq.dslash_adjoint(DIMS, MASS, U_d, t, prec="f64", link_fmt=18, layout="lex", stream=stream)
        e = eta_d.view(torch.float64)
        r = e - q.view(torch.float64)
        return float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(e))

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        solve(mode)
    torch.cuda.synchronize()
    infos = []
    with ClockSampler(local_rank) as clk:
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            infos.append(solve(mode))
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        resid64 = fp64_residual()
        # the same K steps again with CUDA events around every solver kernel, for the
        # per-kernel split and the roofline (the events cost about 3% of a step, so they stay
        # out of the timed steps above)
        pinfos = [solve(mode, profile=True) for _ in range(args.steps)]
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clocks = clk.summary()
    info = infos[-1]
    upd = 2 * V * (info["iters"] + info["high_applies"])
    ms_max, value = whole_job_rate(ms, upd, dev)
    launches = sum(i["launches"] for i in infos)

    # end to end through the public API with pinned host buffers: every step copies its
    # inputs (U, eta) in and its result x out.  Serial: copy in, solve, copy out, on one
    # stream.  Pipelined (the reported value): two sets of device buffers; step i + 1's inputs
    # are copied on a second stream while step i solves, and each result is read back on that
    # stream after its solve; the timed region spans every step's copies and solve.
    def e2e_serial():
        torch.cuda.synchronize()
        barrier()
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        for _ in range(args.steps):
            U_d.copy_(U_h, non_blocking=True)
            eta_d.copy_(eta_h, non_blocking=True)
            solve(mode)
            x_h.copy_(x_d, non_blocking=True)
        h1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return h0.elapsed_time(h1) / args.steps

    def e2e_pipelined():
        cstream = torch.cuda.Stream(dev)
        bufs = [(U_d, eta_d, x_d), (torch.empty_like(U_d), torch.empty_like(eta_d), torch.empty_like(x_d))]
        landed = [torch.cuda.Event(), torch.cuda.Event()]   # inputs of buffer set k copied in
        read = [torch.cuda.Event(), torch.cuda.Event()]     # result of buffer set k copied out

        def copy_in(k):
            Uk, ek, _ = bufs[k]
            with torch.cuda.stream(cstream):
                Uk.copy_(U_h, non_blocking=True)
                ek.copy_(eta_h, non_blocking=True)
                landed[k].record(cstream)

        torch.cuda.synchronize()
        barrier()
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        cstream.wait_event(h0)
        copy_in(0)
        for i in range(args.steps):
            k = i % 2
            if i + 1 < args.steps:
                copy_in(1 - k)
            Uk, ek, xk = bufs[k]
            stream.wait_event(landed[k])
            stream.wait_event(read[k])
            xk.zero_()
            _, info_k, st_k = lq.cg_solve(DIMS, MASS, Uk, ek, x=xk, mode=mode, tol=TOL, workspace=ws, stream=stream)
            if st_k != 0:
                raise RuntimeError(f"solve did not converge: {info_k}")
            cstream.wait_stream(stream)
            with torch.cuda.stream(cstream):
                x_h.copy_(xk, non_blocking=True)
                read[k].record(cstream)
        stream.wait_stream(cstream)
        h1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return h0.elapsed_time(h1) / args.steps

    e2e_serial_ms = e2e_serial()
    e2e_ms = e2e_pipelined()
    _, e2e_value = whole_job_rate(e2e_ms, upd, dev)
    _, e2e_serial_value = whole_job_rate(e2e_serial_ms, upd, dev)

    # plain FP64 CG (native FP64 and FP32-pair arithmetic), the other mixed variants, and the
    # mixed solvers with a native FP64 outer loop (residual, reductions and solution in FP64,
    # as the configuration states it) on the same system: the median of three timed runs
    # after one warm run, each followed by the FP64 recomputation of its residual
    compare = {}
    if not args.no_compare:
        variants = [(m, False) for m in ("f64", "f64x", "mixed_f32", "mixed_f16", "mixed_i32") if m != mode]
        variants += [(m, True) for m in ("mixed_f16", "mixed_f32")]
        for m, nat in variants:
            solve(m, native_f64=nat)
            torch.cuda.synchronize()
            ts = []
            for _ in range(3):
                c0 = torch.cuda.Event(enable_timing=True)
                c1 = torch.cuda.Event(enable_timing=True)
                c0.record(stream)
                ci = solve(m, native_f64=nat)
                c1.record(stream)
                torch.cuda.synchronize()
                ts.append(c0.elapsed_time(c1))
            compare[m + ("+native_f64_outer" if nat else "")] = {
                "ms": statistics.median(ts), "iters": ci["iters"], "cycles": ci["cycles"],
                "true_rel_resid": ci["true_rel_resid"], "true_rel_resid_fp64_recomputed": fp64_residual()}

    if rank != 0:
        return
    peak, peak_kind = measured_peaks()
    kb = kernel_bytes(mode)
    kms = [sum(p["kernel_ms"][i] for p in pinfos) / len(pinfos) for i in range(4)]
    kcalls = [sum(p["kernel_calls"][i] for p in pinfos) / len(pinfos) for i in range(4)]
    kern = {}
    for role, idx in (("K1", 0), ("K2", 1), ("K3", 2)):
        if kcalls[idx] > 0:
            avg = kms[idx] / kcalls[idx] * 1e-3
            gbs = kb[role] * V / avg / 1e9
            kern[role] = {"avg_us": avg * 1e6, "bytes_per_site": kb[role], "gbs": gbs, "frac": gbs / peak,
                          "share_of_step": kms[idx] / ms}
    if kcalls[3] > 0:
        kern["HIGH_F64"] = {"avg_us": kms[3] / kcalls[3] * 1e3, "share_of_step": kms[3] / ms}
    dom = max(("K1", "K2", "K3"), key=lambda r: kern.get(r, {}).get("share_of_step", 0))
    bytes_per_launch = kb[dom] * V
    avg_s = kern[dom]["avg_us"] * 1e-6
    achieved = bytes_per_launch / avg_s / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": ncu_traffic(dom), "kernel": dom, "peak_kind": peak_kind,
            "algorithmic_bytes_per_launch": bytes_per_launch}
    cpu = None
    if world == 1 and not args.no_cpu:
        import oracle
        nth = oracle.max_threads()
        rate1, secs1, _ = oracle_rate(U, eta, 1 << 19, reps=1, threads=1)
        rate, secs, used = oracle_rate(U, eta, 1 << 21, reps=1, threads=nth)
        cpu = {"value": rate, "unit": "site-updates/s", "cores": used, "kind": "oracle",
               "sample": (f"D and D^dag of Eq. 1 on 2^21 sampled sites of the 32^4 fields ({secs:.1f} s, FP64 C "
                          f"oracle, site loop over {used} host cores)"),
               "nproc": os.cpu_count(),
               "single_thread": {"value": rate1, "unit": "site-updates/s", "cores": 1,
                                 "sample": f"2^19 sampled sites, {secs1:.1f} s"},
               "cg_time_to_1e-10": oracle_cg_times(rate, used, compare.get("f64", {}).get("iters"))}
    line = {
        "metric": METRIC,
        "value": value, "unit": "site-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"mixed_f16": "f32 accumulation, f16 spin projection (f16s storage) inner / f32-pair (fp64-class) outer",
                                       "mixed_f32": "f32 inner / f32-pair (fp64-class) outer",
                                       "f64": "f64", "f64x": "f32-pair (fp64-class)",
                                       "mixed_i32": "f32 (i32 fixed-point storage) inner / f32-pair outer"}[mode],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": list(DIMS), "m_q": MASS, "links": "exp(0.3iH), 12-real inner",
                   "inner": mode, "tol": TOL, "rhs_per_gpu": 1,
                   "step": "one whole solve from x = 0; every D or D^dag applied to the lattice counts V site-updates",
                   "l2": "no flush: each inner kernel streams > 200 MB, above the 126 MB L2"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "site-updates/s", "h2d_bytes_per_step": Ub.size + eb.size,
                "d2h_bytes_per_step": eb.size, "ms_per_step": e2e_ms,
                "pipeline": "two device buffer sets: step i+1's inputs copied on a second stream while step i "
                            "solves, each result copied back after its solve",
                "serial": {"value": e2e_serial_value, "ms_per_step": e2e_serial_ms,
                           "pipeline": "copy in, solve, copy out on one stream"}},
        "gpu_launches": launches,
        "clocks": clocks,
        "gflops_1464": value * FLOPS_PER_SITE / 1e9,
        "cg": {"time_to_1e-10_ms": ms_max, "iters": info["iters"], "cycles": info["cycles"],
               "high_applies": info["high_applies"], "true_rel_resid": info["true_rel_resid"],
               "true_rel_resid_fp64_recomputed": resid64,
               "compare": compare,
               "mixed_vs_fp64_speedup": (compare["f64"]["ms"] / ms_max) if "f64" in compare else None,
               "mixed_vs_fp64x_speedup": (compare["f64x"]["ms"] / ms_max) if "f64x" in compare else None,
               "native_f64_outer_vs_fp64_speedup": (compare["f64"]["ms"] / compare[mode + "+native_f64_outer"]["ms"])
               if "f64" in compare and mode + "+native_f64_outer" in compare else None},
        "kernels": kern,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------
# measurement legs for the other workloads (not the default line): uneven lattices in one
# solve, 12 right-hand sides batched, and the large volume; each prints one JSON line
# ------------------------------------------------------------------------------------
def _timed(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts), out


def _updates(dims, infos):
    V = int(__import__("numpy").prod(dims))
    return sum(2 * V * (i["iters"] + i["high_applies"]) for i in infos)


def run_workload(args):
    import numpy as np
    import torch
    import paper_1904_08616_gb300 as lq
    import synth
    lq.load()
    dev = torch.device("cuda", 0)

    def field(a):
        return torch.from_numpy(a.view(np.uint8).reshape(-1)).to(dev)

    def spinors(dims, seeds):
        sb = lq.field_bytes(dims, "spinor", "f64")
        out = torch.empty(len(seeds) * sb, dtype=torch.uint8, device=dev)
        for r, sd in enumerate(seeds):
            out[r * sb:(r + 1) * sb].copy_(torch.from_numpy(synth.gaussian_spinor(dims, seed=sd).view(np.uint8).reshape(-1)))
        return out

    line = {"workload": args.workload, "unit": "site-updates/s", "data": "synthetic", "steps": args.steps,
            "warmup": args.warmup, "mode": args.mode}
    if args.workload == "lattices":
        specs = [((8, 8, 8, 8), 4), ((12, 12, 12, 12), 4), ((16, 16, 16, 32), 4)]
        probs = []
        for i, (dims, nr) in enumerate(specs):
            probs.append({"dims": dims, "m_q": 0.1, "nrhs": nr, "U": field(synth.gauge_field(dims, seed=960 + 100 * i)),
                          "eta": spinors(dims, [961 + 100 * i + r for r in range(nr)])})

        def one(own=False):
            kw = {"block": args.lattice_block} if args.lattice_block else {"autotune": True}
            _, infos, st = lq.cg_solve_lattices(probs, mode=args.mode, tol=TOL, graph=args.inner_loop == "device",
                                                 own_cycles=own, **kw)
            assert st == 0
            return infos

        def seq():
            allinf = []
            for p in probs:
                _, infos, st = lq.cg_solve_multi(p["dims"], 0.1, p["nrhs"], p["U"], p["eta"], mode=args.mode, tol=TOL)
                assert st == 0
                allinf.append(infos)
            return allinf

        ms, infos = _timed(one, args.steps, args.warmup)
        ms_own = _timed(lambda: one(True), args.steps, args.warmup)[0]
        ms_seq = None if args.no_compare else _timed(seq, args.steps, args.warmup)[0]
        upd = sum(_updates(p["dims"], inf) for p, inf in zip(probs, infos))
        line.update({"config": {"lattices": [list(d) + [n] for d, n in specs], "m_q": 0.1, "links": "haar",
                                "tol": TOL},
                     "value": upd / (ms * 1e-3), "ms_per_solve": ms, "ms_sequential_multi": ms_seq,
                     "ms_per_solve_own_cycles": ms_own,
                     "speedup_vs_sequential": (ms_seq / ms) if ms_seq else None,
                     "block": infos[0][0]["block"], "iters": [max(i["iters"] for i in li) for li in infos],
                     "inner_loop": args.inner_loop})
    elif args.workload == "batched":
        dims, nr = (24, 24, 24, 48), 12
        U_d = field(synth.gauge_field(dims, seed=5))
        eta_d = spinors(dims, [500 + r for r in range(nr)])
        sb = lq.field_bytes(dims, "spinor", "f64")

        def multi(rb=None, tuned=False):
            _, infos, st = lq.cg_solve_multi(dims, 0.1, nr, U_d, eta_d, mode=args.mode, tol=TOL, rhs_block=rb,
                                             autotune=tuned)
            assert st == 0
            return infos

        def single():
            out = []
            for r in range(nr):
                _, info, st = lq.cg_solve(dims, 0.1, U_d, eta_d[r * sb:(r + 1) * sb], mode=args.mode, tol=TOL)
                assert st == 0
                out.append(info)
            return out

        ms, infos = _timed(multi, args.steps, args.warmup)
        by_rb = {rb: _timed(lambda rb=rb: multi(rb), args.steps, args.warmup)[0] for rb in (1, 2, 4)}
        # right-hand sides per thread chosen by the library's tuner (the first, untimed warm-up
        # call times the candidates; the timed calls take the cached choice)
        ms_tuned, infos_tuned = _timed(lambda: multi(tuned=True), args.steps, args.warmup)
        ms_single, _ = _timed(single, args.steps, args.warmup)
        # the same batch in plain FP64 CG (one timed solve: about two seconds at this size)
        f64 = None
        if not args.no_compare:
            def multi_f64():
                _, inf, st = lq.cg_solve_multi(dims, 0.1, nr, U_d, eta_d, mode="f64", tol=TOL)
                assert st == 0
                return inf
            ms_f64, infos_f64 = _timed(multi_f64, 1, 0)
            f64 = {"ms_per_solve": ms_f64, "iters": max(i["iters"] for i in infos_f64),
                   "mixed_speedup": ms_f64 / ms}
        line.update({"config": {"lattice": list(dims), "nrhs": nr, "m_q": 0.1, "links": "haar", "tol": TOL},
                     "value": _updates(dims, infos) / (ms * 1e-3), "ms_per_solve": ms,
                     "ms_per_solve_by_rhs_per_thread": by_rb,
                     "autotuned": {"rhs_per_thread": sorted({i["rhs_block"] for i in infos_tuned}),
                                   "ms_per_solve": ms_tuned},
                     "ms_one_by_one": ms_single, "speedup_vs_one_by_one": ms_single / ms,
                     "fp64_cg_same_batch": f64,
                     "iters": max(i["iters"] for i in infos)})
    elif args.workload == "cycles":
        # the whole solve's cycles in one graph launch (the default) against host-driven
        # cycles (graph=False), on small to large lattices: median device time per solve
        res = {}
        for dims in ((8, 8, 8, 8), (16, 16, 16, 16), DIMS):
            U_d = field(synth.gauge_field(dims, seed=SEED_U, kind="near_identity", eps=EPS))
            eta_d = field(synth.gaussian_spinor(dims, seed=SEED_ETA))
            for mode in ("mixed_f16", "mixed_f32", "f64x"):
                row = {}
                for loop in ("device", "host"):
                    def run(loop=loop, mode=mode, dims=dims):
                        _, info, st = lq.cg_solve(dims, MASS, U_d, eta_d, mode=mode, tol=TOL, graph=loop == "device")
                        assert st == 0
                        return info
                    ms, info = _timed(run, args.steps, args.warmup)
                    row[loop + "_ms"] = ms
                row.update({"iters": info["iters"], "cycles": info["cycles"],
                            "host_over_device": row["host_ms"] / row["device_ms"]})
                res["x".join(map(str, dims)) + "/" + mode] = row
        line.update({"config": {"lattices": ["8x8x8x8", "16x16x16x16", "x".join(map(str, DIMS))], "m_q": MASS,
                                "links": "exp(0.3iH)", "tol": TOL},
                     "value": None, "unit": "ms", "solves": res})
    elif args.workload == "dslash":
        # the operator alone on the 32^4 fields, every stored format: site-updates/s, GB/s
        # against the measured copy peak and the 8 TB/s nominal, GFLOP/s at 1464 flops/site
        U, psi = make_inputs()
        U_d, p_d = field(U), field(psi)
        peak, peak_kind = measured_peaks()
        V = int(np.prod(DIMS))
        spinor_b = {"f64": 192, "f64x": 192, "f32": 96, "f16s": 52, "i32s": 100}
        link_b = {"f64": 8, "f64x": 8, "f32": 4, "f16s": 2, "i32s": 4}
        rows = {}
        variants = (("f64", 18, "lex"), ("f64", 18, "eo"), ("f64", 10, "eo"), ("f64x", 18, "eo"),
                    ("f32", 18, "eo"), ("f32", 12, "eo"), ("f32", 10, "eo"), ("f16s", 12, "eo"),
                    ("f16s", 18, "eo"), ("f16s", 10, "eo"), ("i32s", 12, "eo"), ("i32s", 10, "eo"))
        if args.variants:
            keep = set(args.variants.split(","))
            variants = tuple(v for v in variants if f"{v[0]}/{v[1]}/{v[2]}" in keep)
        for prec, fmt, layout in variants:
            Ub = lq.convert_gauge(DIMS, U_d, "f64", "lex", dst_prec=prec, dst_fmt=fmt, dst_layout=layout)
            pb = lq.convert_spinor(DIMS, p_d, "f64", "lex", dst_prec=prec, dst_layout=layout)
            out = torch.empty_like(pb)
            for _ in range(max(args.warmup, 3)):
                lq.dslash_apply(DIMS, MASS, Ub, pb, out=out, prec=prec, link_fmt=fmt, layout=layout)
            torch.cuda.synchronize()
            reps = args.reps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                lq.dslash_apply(DIMS, MASS, Ub, pb, out=out, prec=prec, link_fmt=fmt, layout=layout)
            e1.record()
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) / reps * 1e3
            bytes_site = 2 * spinor_b[prec] + 4 * fmt * link_b[prec]
            rate = V / (us * 1e-6)
            gbs = bytes_site * rate / 1e9
            row = {"us": us, "site_updates_per_s": rate, "bytes_per_site": bytes_site, "gbs": gbs,
                   "frac_measured_hbm": gbs / peak, "frac_nominal_8tbs": gbs / 8000.0,
                   "gflops_1464": rate * FLOPS_PER_SITE / 1e9}
            if prec == "f64":
                row["frac_fp64_pipe_nominal_1.25tf"] = rate * FLOPS_PER_SITE / 1.25e12
            rows[f"{prec}/{fmt}/{layout}"] = row
        line.update({"config": {"lattice": list(DIMS), "m_q": MASS, "links": "exp(0.3iH)",
                                "l2": "every variant streams more than the 126 MB L2 (smallest: 210 MB, f16s/12)",
                                "peak_kind": peak_kind, "peak_gbs": peak},
                     "value": rows["f16s/12/eo"]["site_updates_per_s"] if "f16s/12/eo" in rows else None,
                     "variants": rows})
    elif args.workload == "schur":
        # D x = b on the 32^4 workload: the even-odd Schur solve against solving D^dag D x = D^dag b
        U, b = make_inputs()
        U_d, b_d = field(U), field(b)
        eta_d = lq.dslash_adjoint(DIMS, MASS, U_d, b_d)
        res = {}
        for name, fn in (("schur", lambda: lq.cg_solve_schur(DIMS, MASS, U_d, b_d, mode=args.mode, tol=TOL)),
                         ("normal_equations", lambda: lq.cg_solve(DIMS, MASS, U_d, eta_d, mode=args.mode, tol=TOL))):
            def run(fn=fn):
                out = fn()
                assert out[2] == 0
                return out[1][0] if isinstance(out[1], list) else out[1]
            ms, info = _timed(run, args.steps, args.warmup)
            res[name] = {"ms": ms, "iters": info["iters"], "cycles": info["cycles"],
                         "true_rel_resid": info["true_rel_resid"]}
        line.update({"config": {"lattice": list(DIMS), "m_q": MASS, "links": "exp(0.3iH)", "tol": TOL,
                                "system": "D x = b"},
                     "value": None, "unit": "ms", "solvers": res,
                     "schur_speedup": res["normal_equations"]["ms"] / res["schur"]["ms"]})
    elif args.workload == "grad":
        # the link-gradient kernel against its roofline on 32^4 (fields larger than the L2), and
        # the gradient of L = Re <chi, (D^dag D)^-1 eta> with respect to U and eta on 16^4 (links
        # exp(0.5iH), m_q = 0.1): forward solve, adjoint solve, two applies of D, two link gradients
        from paper_1904_08616_gb300.autograd import dirac_solve
        peak, peak_kind = measured_peaks()
        g_d, psi_d = spinors(DIMS, [81]), spinors(DIMS, [82])
        out = torch.empty(lq.field_bytes(DIMS, "gauge", "f64"), dtype=torch.uint8, device=dev)
        ms_k, _ = _timed(lambda: lq.link_grad(DIMS, g_d, psi_d, out=out), max(args.steps, 10), args.warmup)
        V = int(np.prod(DIMS))
        gbs = 960 * V / (ms_k * 1e-3) / 1e9
        dims16, m16 = (16, 16, 16, 16), 0.1
        V16 = int(np.prod(dims16))
        U16 = torch.from_numpy(synth.gauge_field(dims16, seed=83, kind="near_identity", eps=0.5)).to(dev)
        eta16 = torch.from_numpy(synth.gaussian_spinor(dims16, seed=84)).to(dev)
        chi16 = torch.from_numpy(synth.gaussian_spinor(dims16, seed=85)).to(dev)
        res = {}
        for m in ("f64", "f64x", "mixed_f32"):
            def grad_once(m=m):
                Ur = U16.clone().requires_grad_(True)
                er = eta16.clone().requires_grad_(True)
                x = dirac_solve(dims16, m16, Ur, er, mode=m, tol=1e-10)
                loss = torch.sum((chi16.conj() * x).real)
                loss.backward()
                return Ur.grad
            ms_g, gU = _timed(grad_once, args.steps, args.warmup)
            res[m] = {"ms_per_gradient": ms_g, "grad_U_norm": float(torch.linalg.vector_norm(gU))}
        line.update({"config": {"link_grad_lattice": list(DIMS), "gradient_lattice": list(dims16), "m_q": m16,
                                "links": "exp(0.5iH)", "tol": 1e-10, "V16": V16},
                     "value": gbs, "unit": "GB/s",
                     "link_grad": {"us": ms_k * 1e3, "bytes_per_site": 960, "gbs": gbs, "frac": gbs / peak,
                                   "peak": peak, "peak_kind": peak_kind},
                     "gradient": res})
    elif args.workload == "large":
        dims, nr = (64, 64, 64, 128), 4
        U_d = field(synth.gauge_field(dims, seed=70, kind="haar"))
        eta_d = spinors(dims, [72 + r for r in range(nr)])
        res = {}
        for m in (args.mode, "f64"):
            torch.cuda.empty_cache()

            def run(m=m):
                _, infos, st = lq.cg_solve_multi(dims, 0.02, nr, U_d, eta_d, mode=m, tol=TOL)
                assert st == 0
                return infos

            ms, infos = _timed(run, args.steps if m == args.mode else 1, args.warmup if m == args.mode else 0)
            res[m] = {"ms": ms, "iters": max(i["iters"] for i in infos), "cycles": infos[0]["cycles"],
                      "true_rel_resid": max(i["true_rel_resid"] for i in infos),
                      "site_updates_per_s": _updates(dims, infos) / (ms * 1e-3)}
        line.update({"config": {"lattice": list(dims), "nrhs": nr, "m_q": 0.02, "links": "haar", "tol": TOL},
                     "value": res[args.mode]["site_updates_per_s"], "ms_per_solve": res[args.mode]["ms"],
                     "solvers": res, "mixed_vs_fp64_speedup": res["f64"]["ms"] / res[args.mode]["ms"]})
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="mixed_f16", choices=["mixed_f16", "mixed_f32", "f64", "f64x", "mixed_i32"])
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64 / other-mode comparison solves")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--workload", default="cg32",
                    choices=["cg32", "lattices", "batched", "large", "schur", "dslash", "grad", "cycles"],
                    help="cg32: the 32^4 mixed-precision solve (the bench line); the others print a "
                         "measurement line for the uneven-lattice, 12-RHS, 64^3x128, Schur, operator-only, "
                         "gradient and device- against host-driven cycle workloads")
    ap.add_argument("--variants", default="",
                    help="dslash workload: comma-separated prec/link-reals/layout rows to run (default: all)")
    ap.add_argument("--reps", type=int, default=20, help="dslash workload: timed applies per variant")
    ap.add_argument("--lattice-block", type=int, default=0, choices=[0, 64, 128, 256],
                    help="lattices workload: inner block size (0: tuned)")
    ap.add_argument("--inner-loop", default="device", choices=["device", "host"],
                    help="lattices workload: the whole batch as one CUDA graph launch (device) or host-driven "
                         "cycles with the kernels launched one by one (every kernel visible to a profiler)")
    args = ap.parse_args()
    if args.workload != "cg32":
        run_workload(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
