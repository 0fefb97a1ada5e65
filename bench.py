#!/usr/bin/env python
"""Benchmark of the temporally preconditioned Wilson solve on GB300.

A step is one complete solve of the 24^3 x 128, xi = 3.5 anisotropic Wilson
workload for its 12 spin-colour point sources (one batched wf_solve call): source
preparation with S_L, CGNR on the temporal + 3-D Schur operator M-hat with FP32
applies and FP64 reliable updates, reconstruction with S_R, FP64 true residual
||eta - M psi|| / ||eta|| <= 1e-10 for every source.

value = algorithmic HBM bytes of all M-hat applies in the timed steps / device
time of the steps (GB/s). The roofline entry reports the dominant kernel's
algorithmic bytes per launch over its CUDA-event duration against the measured
HBM copy bandwidth. cpu_baseline (and --impl reference) time the FP64 NumPy
oracle's M-hat apply on the host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

import argparse
import hashlib
import json
import os
import resource
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "precond Wilson apply HBM GB/s & %roofline; time-to-solve 1e-10, 24^3x128 ξ=3.5"
WORKLOAD = "wilson_24c128_xi3.5"

# Algorithmic bytes per odd site of one M-hat apply, by kernel, in the axial frame the
# library works in by default (U_t = 1 on the line, so no U_t is read; the per-line P and
# Lambda add 144 B per 128 sites and are left out). FP32 storage: complex 8 B, half spinor
# 48 B, spinor 96 B, spatial link 48 B (two rows, the third rebuilt from SU(3)); FP64 storage:
# complex 16 B, spatial link 144 B (nine entries).
#   K-a  y = C_R^o x               : x upper half in, y upper half out                  (spinor 96)
#   K-b  z = C_R^e C_L^e D_s^eo y   : neighbour spinor (read once), z out; 6 spatial links (192; links)
#   K-c  out = x - C_L^o D_s^oe z   : neighbour z, x, out; 6 spatial links                (288; links)
# With several right-hand sides the nrhs warps of a line run together and read its links
# once (through L2), so a launch moves  odd_sites * (nrhs * spinor bytes + link bytes).
KERNEL_SPINOR_BYTES_F32 = {"schur_a_tdag": 96, "schur_b_hop_tsolve": 192, "schur_c_hop_tinv_axpy": 288}
KERNEL_LINKS = {"schur_a_tdag": 0, "schur_b_hop_tsolve": 6, "schur_c_hop_tinv_axpy": 6}
# The 4-D even-odd comparator per odd 4-D site (axial frame: temporal hops read no link):
#   dslash_eo: other-parity spinor (read once) + out; dslash_oe_axpy: + x. 6 spatial links each.
EO4D_SPINOR_BYTES_F32 = {"eo4d_dslash_eo": 192, "eo4d_dslash_oe_axpy": 288}
LINK_BYTES = {"_f32": 48, "_f64": 144}
APPLY_BYTES_F32 = sum(KERNEL_SPINOR_BYTES_F32.values()) + 12 * LINK_BYTES["_f32"]  # 1152 B per odd site


def launch_bytes(name, odd_sites, nrhs):
    """Algorithmic bytes of one launch of a Schur kernel over nrhs sources, or None."""
    for base, spinor in KERNEL_SPINOR_BYTES_F32.items():
        for suffix, scale in (("_f32", 1), ("_f64", 2)):
            if name == base + suffix:
                return odd_sites * (nrhs * scale * spinor + KERNEL_LINKS[base] * LINK_BYTES[suffix])
    return None


def eo4d_launch_bytes(name, odd_sites, nrhs):
    for base, spinor in EO4D_SPINOR_BYTES_F32.items():
        for suffix, scale in (("_f32", 1), ("_f64", 2)):
            if name == base + suffix:
                return odd_sites * (nrhs * scale * spinor + 6 * LINK_BYTES[suffix])
    return None


def apply_bytes(odd_sites, nrhs, scale=1):
    """Algorithmic bytes of one M-hat apply over nrhs sources (scale 2: FP64)."""
    suffix = "_f32" if scale == 1 else "_f64"
    return sum(launch_bytes(k + suffix, odd_sites, nrhs) for k in KERNEL_SPINOR_BYTES_F32)


def paper_flops_per_apply(L, T):
    """(3432 N_t - 576)(V_s / 2) FLOPs per M-hat apply (App. B, Wilson temporal + Schur)."""
    return (3432 * T - 576) * (L ** 3 // 2)


# the sources that compile, launch or lay out the data of the Schur operator's kernels: a change
# to any of them voids the DRAM traffic recorded in profiles/traffic.json
HOP_KERNEL_SOURCES = ("wf_abi.cu", "wf_async.cuh", "wf_common.cuh", "wf_df64.cuh", "wf_handle.h", "wf_internal.h",
                      "wf_kernels.cu", "wf_layout.cu", "wf_line.cuh", "wf_pipe.cu", "wf_wide.cu", "wf_wide.cuh",
                      "wf_wide_body.inc", "wf_line_kernels.cuh")


def source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_0910_0992_gb300", "csrc")
    for f in HOP_KERNEL_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_for(kernel, nrhs, config, path=None):
    """DRAM bytes per launch of `kernel` from a committed ncu record, or None.

    A record counts only for the workload, source count and hop-kernel configuration (the
    autotuner's kernel family and traversal) it was captured in, and only while the kernel
    sources are those of the capture (source hash)."""
    path = path or os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            t = json.load(fh)
    except Exception:
        return None
    if t.get("source_hash") != source_hash():
        return None
    entries = t.get("kernels", {}).get(kernel) or []
    if isinstance(entries, dict):  # one captured configuration, or a list of them
        entries = [entries]
    for e in entries:
        if e.get("workload") == WORKLOAD and e.get("nrhs") == nrhs and e.get("config") == config:
            return e.get("dram_bytes_per_launch")
    return None


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle (CPU)
def _oracle_worker(L, T, prm, seed, barrier, out):
    """One FP64 oracle M-hat apply of its own Gaussian source (a process of oracle_sample)."""
    import synthetic as S
    from oracle import wilson as W

    p = W.Params(L, T, prm["kappa_s"], kappa_t=prm["kappa_t"], bc=prm["bc"])
    U = S.random_gauge(L, T, prm["eps"], prm["seed"])
    par3 = W.parity3(L, T)
    x = W.restrict(S.gaussian_source(L, T, seed), par3 == 1)
    barrier.wait()  # every process applies at the same time
    t0 = time.time()
    W.M_hat(U, x, p, par3)
    out.put((t0, time.time()))


def oracle_sample(target_s, prm, procs=None):
    """Time the FP64 oracle's M-hat apply on the host's cores: one process per core (spawned, so
    nothing of a CUDA context is inherited), each applying M-hat to its own source on a lattice of
    the workload's couplings sized for ~target_s, all started together.

    Returns (GB/s in the FP64 model bytes: all processes' bytes over the span from the first start
    to the last end, description, processes, seconds).
    """
    import multiprocessing as mp

    procs = procs or os.cpu_count() or 1
    per_site_s = 1.4e-5  # one oracle apply per site on one GB300 host core (sizing only)
    L = int(round((target_s / (per_site_s * prm["T"])) ** (1.0 / 3.0)))
    L = max(4, min(prm["L"], L - (L % 2)))
    T = prm["T"]
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(procs), ctx.Queue()
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"  # one core per process
    try:
        ps = [ctx.Process(target=_oracle_worker, args=(L, T, prm, prm["seed"] + 7 + i, barrier, out))
              for i in range(procs)]
        for q in ps:
            q.start()
        spans = [out.get() for _ in ps]
        for q in ps:
            q.join()
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    dt = max(e for _, e in spans) - min(b for b, _ in spans)
    odd_sites = L ** 3 * T // 2
    gbs = procs * apply_bytes(odd_sites, 1, 2) / dt / 1e9
    desc = (f"{procs} concurrent FP64 oracle M-hat applies (one process per host core, one Gaussian source "
            f"each) on a {L}^3x{T} lattice with the workload's couplings; the full 24^3x128 x 12-source step "
            f"is {24 ** 3 / L ** 3 * 12 / procs:.1f}x that much work")
    return gbs, desc, procs, dt


def run_reference(args, prm):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    per_step = max(5.0, 150.0 / max(1, args.steps + args.warmup))
    vals, desc, threads, secs = [], "", 1, []
    for i in range(args.warmup + args.steps):
        gbs, desc, threads, dt = oracle_sample(per_step, prm)
        if i >= args.warmup:
            vals.append(gbs)
            secs.append(dt)
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": desc},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": threads, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- GPU arm
def run_ours(args, prm, U, eta):
    import numpy as np
    import torch

    import paper_0910_0992_gb300 as wf

    from paper_0910_0992_gb300.replicas import Replicas

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    reps = Replicas("nccl", device=torch.device("cuda", local))
    world, rank = reps.world, reps.rank

    def barrier():
        reps.barrier()
        torch.cuda.synchronize()

    prec = {"fp32": wf.WF_FP32, "fp64": wf.WF_FP64, "fp16mix": wf.WF_FP16MIX}[args.precision]
    stream = torch.cuda.Stream()
    w = wf.Wilson(prm["L"], prm["T"], prm["kappa_s"], kappa_t=prm["kappa_t"], bc=prm["bc"])
    w.set_stream(stream.cuda_stream)
    w.load_gauge(U)
    nsrc = eta.shape[0]
    rhs = torch.from_numpy(eta).cuda()
    x = torch.empty_like(rhs)

    def solve(r, xx):
        st, it, res = wf.wf_solve(w.h, r, xx, nsrc, args.tol, wf.WF_TEMPORAL_SCHUR, prec, 0)
        if st != wf.WF_OK or max(res) > args.tol:
            raise RuntimeError(f"solve failed: status {st}, residuals {res}")
        return it, res

    for _ in range(args.warmup):
        solve(rhs, x)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    n0 = wf.wf_launch_count(w.h)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    iters = None
    for _ in range(args.steps):
        iters, res = solve(rhs, x)
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = wf.wf_launch_count(w.h) - n0
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms = reps.max(ms, device="cuda")
    # per-kernel breakdown from one more solve with per-launch CUDA events (outside the timed
    # region: event pairs around every launch, and no CUDA graph replay, while profiling)
    wf.wf_profile(w.h, 1)
    solve(rhs, x)
    torch.cuda.synchronize()
    prof = wf.wf_profile_get(w.h)
    wf.wf_profile(w.h, 0)

    odd_sites = prm["L"] ** 3 * prm["T"] // 2
    launched_f32 = prof.get("schur_c_hop_tinv_axpy_f32", (0, 0))[0]
    applies_f64 = prof.get("schur_c_hop_tinv_axpy_f64", (0, 0))[0]
    # applies that did work: two per CG iteration plus the initial A^dag r of every CG run (one per
    # defect-correction pass, counted by the passes' S_L hops; with reliable updates one run plus a
    # completion per update, an FP64 apply each); the rest are block overshoot, whose kernels
    # return at once because every source had stopped
    passes = prof.get("prep_hop_f32", (0, 0))[0]
    extra = passes if passes else 1 + applies_f64
    applies_f32 = min(launched_f32, 2 * max(iters) + extra) if prec == wf.WF_FP32 else launched_f32
    # every M-hat launch sequence works on all nsrc sources at once; per solve
    solve_bytes = applies_f32 * apply_bytes(odd_sites, nsrc) + applies_f64 * apply_bytes(odd_sites, nsrc, 2)
    value = reps.whole_job_rate(args.steps * solve_bytes, ms * 1e-3) / 1e9
    flops = args.steps * (applies_f32 + applies_f64) * paper_flops_per_apply(prm["L"], prm["T"]) * nsrc

    # roofline: the dominant kernel by time
    cand = {k: v for k, v in prof.items() if launch_bytes(k, 1, 1) is not None and v[0] > 0}
    dom = max(cand, key=lambda k: cand[k][1])
    n_l, ms_l = cand[dom]
    bytes_launch = launch_bytes(dom, odd_sites, nsrc)
    achieved = bytes_launch / (ms_l / n_l * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    hop = _hop_config(wf, w, nsrc)
    traffic = traffic_for(dom, nsrc, hop_config_key(hop))
    schur_ms = sum(cand[k][1] for k in cand)
    total_prof_ms = sum(v[1] for v in prof.values())

    # end to end through the C-ABI with host (pinned) buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        h_rhs = torch.from_numpy(eta).pin_memory()
        h_x = torch.empty_like(h_rhs).pin_memory()
        solve(h_rhs, h_x)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            solve(h_rhs, h_x)
        torch.cuda.synchronize()
        e2e_s = reps.max(time.perf_counter() - t0, device="cuda")
        e2e = {"value": reps.whole_job_rate(args.steps * solve_bytes, e2e_s) / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": int(h_rhs.numel() * 16), "d2h_bytes_per_step": int(h_x.numel() * 16),
               "ms_per_step": 1e3 * e2e_s / args.steps}

    # same-GPU comparison (outside the timed region): the standard 4-D even-odd solve of the
    # same sources, batched and single-source, against the temporal + 3-D Schur solve
    compare = None
    if not args.no_compare:
        def timed(method, r, xx, nr, nrep):
            st, it, res = wf.wf_solve(w.h, r, xx, nr, args.tol, method, prec, 0)  # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(nrep):
                st, it, res = wf.wf_solve(w.h, r, xx, nr, args.tol, method, prec, 0)
            e1.record(stream)
            torch.cuda.synchronize()
            if st != wf.WF_OK or max(res) > args.tol:
                raise RuntimeError(f"comparison solve failed: method {method}, status {st}, residuals {res}")
            return e0.elapsed_time(e1) / nrep / 1e3, it

        r1, x1 = rhs[:1].contiguous(), x[:1].contiguous()
        t_eo, it_eo = timed(wf.WF_EO4D, rhs, x, nsrc, 2)
        t_ts1, it_ts1 = timed(wf.WF_TEMPORAL_SCHUR, r1, x1, 1, 3)
        t_eo1, it_eo1 = timed(wf.WF_EO4D, r1, x1, 1, 3)
        t_ts = ms / args.steps / 1e3
        compare = {
            "baseline_method": "standard 4-D even-odd (Schur) CGNR, same GPU, same precision scheme",
            "batched": {"nrhs": nsrc, "temporal_schur_s": t_ts, "eo4d_s": t_eo, "speedup": t_eo / t_ts,
                        "temporal_schur_iterations": iters, "eo4d_iterations": it_eo},
            "single": {"nrhs": 1, "temporal_schur_s": t_ts1, "eo4d_s": t_eo1, "speedup": t_eo1 / t_ts1,
                       "temporal_schur_iterations": it_ts1[0], "eo4d_iterations": it_eo1[0]},
        }

    # per-kernel rooflines of the operator applies (outside the timed region): the benchmarked
    # batch and one source (the single-RHS form), for M-hat and for the 4-D even-odd comparator
    applies = None
    if not args.no_compare:
        applies = {f"{op}_{n}src": apply_roofline(wf, torch, w, n, op, odd_sites, peak)
                   for op in ("schur", "eo4d") for n in (nsrc, 1)}
        if compare is not None:
            compare["kernels_batched"] = applies[f"eo4d_{nsrc}src"]
            compare["kernels_single"] = applies["eo4d_1src"]

    # the same solve with FP16-stored spinors (outside the timed region)
    fp16 = None
    if not args.no_compare and prec == wf.WF_FP32:
        t16, it16, res16 = _timed_solve(wf, torch, w, stream, rhs, x, wf.WF_TEMPORAL_SCHUR, wf.WF_FP16MIX,
                                        args.tol, reps=2)
        fp16 = {"precision": ("FP16-stored spinors, FP32 arithmetic, FP32 residual recomputations, inside "
                              "the defect-correction passes" if os.environ.get("WF_DC", "1") != "0" else
                              "FP16-stored spinors, FP32 arithmetic, FP32 and FP64 reliable updates"),
                "time_to_solve_s": t16, "iterations": it16, "max_true_residual": max(res16)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        gbs, desc, threads, dt = oracle_sample(10.0, prm)
        cpu = {"value": gbs, "unit": "GB/s", "cores": threads, "kind": "oracle", "sample": desc,
               "seconds": dt}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == wf.WF_FP32 else "f64", "data": "synthetic",
            "config": {
                "workload": f"{WORKLOAD}: 24^3x128, xi=3.5, kappa_s={prm['kappa_s']:.6f}, "
                            f"kappa_t={prm['kappa_t']:.6f}, antiperiodic, eps=0.2 random SU(3) links, "
                            f"12 point sources solved in one batched call",
                "method": "temporal + 3-D Schur preconditioned CGNR (S_L prep, S_R reconstruction)",
                "precision": (("FP32 defect correction: per pass S_L, CGNR on M-hat and S_R in FP32; FP64 "
                               "solution accumulation and true residual of M"
                               if os.environ.get("WF_DC", "1") != "0" else
                               "FP32 M-hat applies, FP64 reliable updates, S_L, S_R and true residual")
                              if prec == wf.WF_FP32 else "FP64 throughout"),
                "tol": args.tol, "parallelism": f"replicas x{world} (sources per GPU fixed)",
                "l2": "inputs larger than L2 (4.1 GB of sources, 2.5 GB of gauge copies)",
            },
            "time_to_solve_s": ms / args.steps / 1e3,
            "iterations": iters,
            "m_hat_applies_per_step": {"f32": applies_f32, "f64": applies_f64, "f32_launched": launched_f32},
            "gflops_paper_model": reps.whole_job_rate(flops, ms * 1e-3) / 1e9,
            "schur_kernel_share": schur_ms / total_prof_ms if total_prof_ms else None,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "algorithmic_bytes_per_launch": bytes_launch,
                         "avg_launch_ms": ms_l / n_l,
                         "apply_frac": applies[f"schur_{nsrc}src"]["apply_frac"] if applies else None,
                         "single_source_apply_frac": applies["schur_1src"]["apply_frac"] if applies else None},
            "operator_applies": applies,
            "fp16mix_same_sources": fp16,
            "kernels_one_solve": {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
            "hop_kernels_autotuned": hop,
            "clocks": clk,
            "gpu_launches": launches,
            "e2e": e2e,
            "vs_eo4d_same_gpu": compare,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    w.close()
    reps.close()
    return 0


def run_apply(args, prm, U, eta):
    """--mode apply: only M-hat applies (FP32, --nrhs sources) for kernel profiling; prints per-kernel times."""
    import torch

    import paper_0910_0992_gb300 as wf
    import synthetic as S

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w = wf.Wilson(prm["L"], prm["T"], prm["kappa_s"], kappa_t=prm["kappa_t"], bc=prm["bc"])
    w.load_gauge(U)
    half = prm["L"] ** 3 * prm["T"] // 2 * 12
    nr = args.nrhs
    x = torch.from_numpy(S.gaussian_source(prm["L"], prm["T"], 77).reshape(-1)[:half].copy()).cuda().repeat(nr)
    out = torch.empty_like(x)
    apply = wf.wf_apply_eo4d_f32 if args.op == "eo4d" else wf.wf_apply_schur_f32
    for _ in range(args.warmup):
        apply(w.h, x, out, 0, nr)
    wf.wf_profile(w.h, 1)
    for _ in range(args.steps):
        apply(w.h, x, out, 0, nr)
    prof = wf.wf_profile_get(w.h)
    odd_sites = prm["L"] ** 3 * prm["T"] // 2
    rows = {}
    for k, (n, ms) in prof.items():
        b = launch_bytes(k, odd_sites, nr) or eo4d_launch_bytes(k, odd_sites, nr)
        rows[k] = {"launches": n, "avg_ms": ms / n, "gbs": (b / (ms / n * 1e-3) / 1e9) if b else None}
    print(json.dumps({"mode": "apply", "workload": f"{prm['L']}^3x{prm['T']}", "nrhs": nr, "kernels": rows}))
    w.close()
    return 0


def hop_config_key(hop):
    """The hop-kernel configuration as a traffic-record key: "variant=<v>;tile_rows=<r>", and for
    the bulk-fed kernels ";sources=<g>;stages=<s>"."""
    if not hop:
        return None
    key = f"variant={hop['variant']};tile_rows={hop['tile_rows']}"
    if "stages" in hop:
        key += f";sources={hop['sources_per_unit']};stages={hop['stages']}"
    return key


HOP_VARIANTS = {1: "one thread per site", 2: "sites per lane", 3: "bulk-copy-fed"}


def _hop_config(wf, w, nrhs):
    c = wf.wf_hop_config(w.h, nrhs)
    if c is None:
        return None
    r = {"variant": HOP_VARIANTS.get(c[0], c[0]), "tile_rows": c[1], "kb_plus_kc_ms_x3": c[2]}
    if c[0] == 3:
        r["sources_per_unit"], r["stages"] = wf.wf_hop_pipe_config(w.h, nrhs)
    return r


def apply_roofline(wf, torch, w, nrhs, op, odd_sites, peak, steps=10):
    """Per-kernel CUDA-event times of the FP32 operator (op "schur": K-a, K-b, K-c of M-hat; "eo4d":
    the comparator's two half dslashes) over nrhs sources, with algorithmic bytes, GB/s and the
    fraction of peak per kernel and for the whole apply (bytes of all its kernels over the sum of
    their mean launch times). Outside every timed region."""
    half = w.L ** 3 * w.T // 2 * 12
    g = torch.Generator(device="cpu").manual_seed(7)
    x = torch.complex(torch.randn(nrhs * half, generator=g, dtype=torch.float64),
                      torch.randn(nrhs * half, generator=g, dtype=torch.float64)).cuda()
    out = torch.empty_like(x)
    fn = wf.wf_apply_eo4d_f32 if op == "eo4d" else wf.wf_apply_schur_f32
    model = eo4d_launch_bytes if op == "eo4d" else launch_bytes
    for _ in range(2):
        fn(w.h, x, out, 0, nrhs)
    torch.cuda.synchronize()
    wf.wf_profile(w.h, 1)
    for _ in range(steps):
        fn(w.h, x, out, 0, nrhs)
    prof = wf.wf_profile_get(w.h)
    wf.wf_profile(w.h, 0)
    rows, tot_b, tot_ms = {}, 0.0, 0.0
    for k, (n, ms) in prof.items():
        b = model(k, odd_sites, nrhs)
        if b is None or n == 0:
            continue
        avg = ms / n
        rows[k] = {"avg_launch_ms": avg, "algorithmic_bytes_per_launch": b, "achieved_gbs": b / (avg * 1e-3) / 1e9,
                   "frac": b / (avg * 1e-3) / 1e9 / peak}
        tot_b += b
        tot_ms += avg
    apply_gbs = tot_b / (tot_ms * 1e-3) / 1e9 if tot_ms else None
    return {"nrhs": nrhs, "kernels": rows, "apply_ms": tot_ms, "apply_bytes": tot_b, "apply_gbs": apply_gbs,
            "apply_frac": apply_gbs / peak if apply_gbs else None}


def _timed_solve(wf, torch, w, stream, rhs, x, method, prec, tol, reps=1):
    """(seconds per solve, iterations, true residuals) after one warm-up solve; method "full_sw":
    wf_solve_full_sw."""
    nr = rhs.shape[0]

    def call():
        if method == "full_sw":
            return wf.wf_solve_full_sw(w.h, rhs, x, nr, tol, prec)
        return wf.wf_solve(w.h, rhs, x, nr, tol, method, prec, 0)
    call()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        st, it, res = call()
    e1.record(stream)
    torch.cuda.synchronize()
    if st != wf.WF_OK or max(res) > tol:
        raise RuntimeError(f"solve failed: method {method}, status {st}, residuals {res}")
    return e0.elapsed_time(e1) / reps / 1e3, list(it), list(res)


METHOD_NAMES = {0: "unprec", 1: "eo4d", 2: "temporal", 3: "temporal_schur", 4: "temporal_ilu"}


def run_methods(args):
    """--mode methods: 16^3 x 128, xi = 3.5, one Gaussian source; every method in FP64 and in FP32
    with FP64 reliable updates, and the temporal + Schur method with FP16-stored spinors:
    iterations, time to solution, FP64 true residual."""
    import torch

    import paper_0910_0992_gb300 as wf
    import synthetic as S

    prm, U, eta = S.workload("wilson_16c128_xi3.5")
    stream = torch.cuda.Stream()
    w = wf.Wilson(prm["L"], prm["T"], prm["kappa_s"], kappa_t=prm["kappa_t"], bc=prm["bc"])
    w.set_stream(stream.cuda_stream)
    w.load_gauge(U)
    rhs = torch.from_numpy(eta).cuda()
    x = torch.empty_like(rhs)
    rows = []
    for prec, pname in ((wf.WF_FP64, "fp64"), (wf.WF_FP32, "fp32")):
        for method in (wf.WF_UNPREC, wf.WF_EO4D, wf.WF_TEMPORAL, wf.WF_TEMPORAL_SCHUR):
            t, it, res = _timed_solve(wf, torch, w, stream, rhs, x, method, prec, args.tol)
            rows.append({"method": METHOD_NAMES[method], "precision": pname, "iterations": it[0],
                         "time_s": t, "true_residual": res[0]})
    # FP16-stored spinors (FP32 arithmetic, FP32 and FP64 reliable updates): the temporal + Schur method
    t, it, res = _timed_solve(wf, torch, w, stream, rhs, x, wf.WF_TEMPORAL_SCHUR, wf.WF_FP16MIX, args.tol)
    rows.append({"method": "temporal_schur", "precision": "fp16mix", "iterations": it[0], "time_s": t,
                 "true_residual": res[0]})
    w.close()
    print(json.dumps({"mode": "methods", "workload": "wilson_16c128_xi3.5: 16^3x128, xi=3.5, 1 Gaussian source",
                      "tol": args.tol, "results": rows}))
    return 0


def run_sweep(args):
    """--mode sweep: xi in {1, 3, 4.5, 6} on 12^3 x 48, 16^3 x 96 and 16^3 x 128, four Gaussian
    sources per lattice in one call, kappa_s = 0.9 of the free critical value: temporal + 3-D Schur
    against 4-D even-odd (FP32 iterations, FP64 reliable updates, FP64 true residual)."""
    import torch

    import paper_0910_0992_gb300 as wf
    import synthetic as S

    rows, batches = [], []
    for xi in (1.0, 3.0, 4.5, 6.0):
        keep = []
        for L, T in ((12, 48), (16, 96), (16, 128)):
            name = f"sweep_xi{xi:g}_{L}c{T}"
            prm, U, eta = S.workload(name)
            stream = torch.cuda.Stream()
            w = wf.Wilson(L, T, prm["kappa_s"], kappa_t=prm["kappa_t"], bc=prm["bc"])
            w.set_stream(stream.cuda_stream)
            w.load_gauge(U)
            rhs = torch.from_numpy(eta).cuda()
            x = torch.empty_like(rhs)
            keep.append((w, rhs, x, stream))
            r = {"workload": name, "xi": xi, "L": L, "T": T, "kappa_s": prm["kappa_s"], "nsrc": eta.shape[0]}
            for method in (wf.WF_TEMPORAL_SCHUR, wf.WF_EO4D):
                t, it, res = _timed_solve(wf, torch, w, stream, rhs, x, method, wf.WF_FP32, args.tol, reps=3)
                r[METHOD_NAMES[method]] = {"time_s": t, "iterations": max(it), "max_true_residual": max(res)}
            r["time_ratio_eo4d_over_temporal_schur"] = r["eo4d"]["time_s"] / r["temporal_schur"]["time_s"]
            r["hop_kernels_autotuned"] = _hop_config(wf, w, eta.shape[0])
            r["iteration_ratio"] = r["eo4d"]["iterations"] / r["temporal_schur"]["iterations"]
            rows.append(r)
        # the three lattices of this xi in one ragged call
        seq = sum(rr["temporal_schur"]["time_s"] for rr in rows[-3:])
        batches.append(dict(xi=xi, **_ragged_times(wf, torch, keep, args.tol, seq)))
        for k in keep:
            k[0].close()

    # a ragged batch of small lattices (xi = 3.5, two Gaussian sources each), where single
    # solves do not fill the GPU
    xi = 3.5
    ks = 0.9 * S.kappa_critical_free(xi)
    keep, seq = [], 0.0
    for i, (L, T) in enumerate(((8, 16), (8, 24), (8, 32), (8, 48), (6, 64), (6, 96), (10, 40), (12, 24))):
        U = S.random_gauge(L, T, 0.25, 300 + i)
        eta = S.gaussian_source(L, T, 400 + i, nrhs=2)
        stream = torch.cuda.Stream()
        w = wf.Wilson(L, T, ks, kappa_t=xi * ks, bc=-1)
        w.set_stream(stream.cuda_stream)
        w.load_gauge(U)
        rhs = torch.from_numpy(eta).cuda()
        x = torch.empty_like(rhs)
        keep.append((w, rhs, x, stream))
        seq += _timed_solve(wf, torch, w, stream, rhs, x, wf.WF_TEMPORAL_SCHUR, wf.WF_FP32, args.tol, reps=3)[0]
    batches.append(dict(xi=xi, **_ragged_times(wf, torch, keep, args.tol, seq)))
    for k in keep:
        k[0].close()
    print(json.dumps({"mode": "sweep", "tol": args.tol, "results": rows, "ragged_calls": batches}))
    return 0


def _ragged_times(wf, torch, keep, tol, seq):
    """wf_solve_many over the handles in keep: the default path (a host thread and stream per
    lattice, their phases overlapping) and the joint solve (WF_JOINT=1: one launch per kernel and
    iteration across lattices), each the mean of three calls after a warm-up, against seq, the
    one-at-a-time total."""
    hs = [k[0].h for k in keep]
    rl, xl, nl = [k[1] for k in keep], [k[2] for k in keep], [k[1].shape[0] for k in keep]
    out = {"lattices": [f"{k[0].L}^3x{k[0].T}" for k in keep], "sources_per_lattice": nl}
    for key, joint in (("one_call_s", "0"), ("joint_launches_s", "1")):
        os.environ["WF_JOINT"] = joint
        try:
            wf.wf_solve_many(hs, rl, xl, nl, tol, wf.WF_TEMPORAL_SCHUR, wf.WF_FP32)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(3):
                st, per = wf.wf_solve_many(hs, rl, xl, nl, tol, wf.WF_TEMPORAL_SCHUR, wf.WF_FP32)
            torch.cuda.synchronize()
        finally:
            os.environ.pop("WF_JOINT", None)
        if st != wf.WF_OK or max(max(q[2]) for q in per) > tol:
            raise RuntimeError(f"ragged solve failed: status {st}")
        out[key] = (time.perf_counter() - t0) / 3
    out["one_at_a_time_s"] = seq
    out["speedup"] = seq / out["one_call_s"]
    out["speedup_joint_launches"] = seq / out["joint_launches_s"]
    return out


def run_force(args):
    """--mode force: the pseudofermion force on 8^3 x 32 and 16^3 x 64 (xi = 3), one Gaussian
    pseudofermion on the odd 3-D parity, FP64 and FP32-inner CG to 1e-12: time and iterations."""
    import numpy as np
    import torch

    import paper_0910_0992_gb300 as wf
    import synthetic as S

    rows = []
    for name in ("force_8c32_xi3", "force_16c64_xi3"):
        prm, U, _ = S.workload(name, with_sources=False)
        L, T = prm["L"], prm["T"]
        V = L ** 3 * T
        full = S.gaussian_source(L, T, prm["seed"] + 7)
        t_, z, y, x = np.meshgrid(np.arange(T), np.arange(L), np.arange(L), np.arange(L), indexing="ij")
        odd = ((x + y + z) % 2) == 1
        phi = torch.from_numpy(np.ascontiguousarray(full[odd])).cuda()
        w = wf.Wilson(L, T, prm["kappa_s"], kappa_t=prm["kappa_t"], bc=prm["bc"])
        w.load_gauge(U)
        F = torch.empty((V, 4, 8), dtype=torch.float64, device="cuda")
        r = {"workload": name, "L": L, "T": T}
        for prec, pname in ((wf.WF_FP64, "fp64"), (wf.WF_FP32, "fp32_inner")):
            wf.wf_force(w.h, phi, F, prec, 1e-12)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Sv, it = wf.wf_force(w.h, phi, F, prec, 1e-12)
            torch.cuda.synchronize()
            r[pname] = {"time_s": time.perf_counter() - t0, "cg_iterations": it, "action": Sv}
        w.close()
        rows.append(r)
    print(json.dumps({"mode": "force", "results": rows}))
    return 0


def spatial_plaquette(U):
    """<(1/3) Re tr U_ij> over sites and spatial planes i < j (input preparation for Eq. ClovCoeffs)."""
    import numpy as np
    acc, n = 0.0, 0
    for i, j in ((0, 1), (0, 2), (1, 2)):
        Ui, Uj = U[..., i, :, :], U[..., j, :, :]
        Uj_i = np.roll(Uj, -1, axis=3 - i)   # U_j(x + i); lattice axes 0..3 = t, z, y, x
        Ui_j = np.roll(Ui, -1, axis=3 - j)   # U_i(x + j)
        P = Ui @ Uj_i @ np.conj(np.swapaxes(Ui_j, -1, -2)) @ np.conj(np.swapaxes(Uj, -1, -2))
        acc += float(np.real(np.trace(P, axis1=-2, axis2=-1)).sum()) / 3.0
        n += P.shape[0] * P.shape[1] * P.shape[2] * P.shape[3]
    return acc / n


def run_clover(args):
    """--mode clover: the clover operator with partial temporal preconditioning and 3-D ILU on
    16^3 x 128, xi = 3.5, one Gaussian source, tree-level tadpole coefficients (Eq. ClovCoeffs,
    u_t = 1, gamma_g = gamma_f = xi, u_s from the spatial plaquette): FP64 and FP32 (FP64
    reliable updates) solves to 1e-10, against the 4-D Schur clover solve (the paper's
    comparator) and the Wilson temporal + 3-D Schur solve of the same source, and per-kernel CUDA-event times of one FP32 ILU solve (the clover apply kernel
    against HBM: half its chiral blocks, 576 B, and the spinor in and out, 192 B, per site in FP32)."""
    import torch

    import paper_0910_0992_gb300 as wf
    import synthetic as S

    name = "wilson_16c128_xi3.5"
    prm, U, eta = S.workload(name)
    xi = prm["kappa_t"] / prm["kappa_s"]
    u_s = spatial_plaquette(U) ** 0.25
    c_s = 1.0 / (u_s ** 3 * xi)
    c_t = (1.0 + 1.0 / xi) / (2.0 * u_s ** 2)
    stream = torch.cuda.Stream()
    w = wf.Wilson(prm["L"], prm["T"], prm["kappa_s"], kappa_t=prm["kappa_t"], bc=prm["bc"])
    w.set_stream(stream.cuda_stream)
    rhs = torch.from_numpy(eta).cuda()
    x = torch.empty_like(rhs)
    rows = []
    w.load_gauge(U)
    for prec, pname in ((wf.WF_FP64, "fp64"), (wf.WF_FP32, "fp32")):
        t, it, res = _timed_solve(wf, torch, w, stream, rhs, x, wf.WF_TEMPORAL_SCHUR, prec, args.tol)
        rows.append({"operator": "wilson", "method": "temporal_schur", "precision": pname, "iterations": it[0],
                     "time_s": t, "true_residual": res[0]})
    w.load_gauge_clover(U, c_s, c_t)
    for method in (wf.WF_TEMPORAL_ILU, wf.WF_EO4D, "full_sw"):
        for prec, pname in ((wf.WF_FP64, "fp64"), (wf.WF_FP32, "fp32")):
            t, it, res = _timed_solve(wf, torch, w, stream, rhs, x, method, prec, args.tol)
            rows.append({"operator": "clover", "method": METHOD_NAMES.get(method, method), "precision": pname,
                         "iterations": it[0], "time_s": t, "true_residual": res[0]})
    wf.wf_profile(w.h, 1)
    wf.wf_solve_full_sw(w.h, rhs, x, 1, args.tol, wf.WF_FP32)
    prof_full = wf.wf_profile_get(w.h)
    wf.wf_profile(w.h, 0)
    wf.wf_profile(w.h, 1)
    wf.wf_solve(w.h, rhs, x, 1, args.tol, wf.WF_TEMPORAL_ILU, wf.WF_FP32, 0)
    prof = wf.wf_profile_get(w.h)
    wf.wf_profile(w.h, 0)
    sites = prm["L"] ** 3 * prm["T"] // 2
    peak, kind = measured_peak()
    kern = {}
    for k, (n, ms) in sorted(prof.items(), key=lambda kv: -kv[1][1]):
        if n:  # names of the earlier profiled solve stay registered with no launches
            kern[k] = {"launches": n, "total_ms": ms, "avg_ms": ms / n}
    ca = kern.get("clover_apply_f32")
    if ca:
        gbs = 768.0 * sites / (ca["avg_ms"] * 1e-3) / 1e9
        ca.update({"gbs": gbs, "hbm_frac": gbs / peak, "hbm_peak": kind})
    kfull = {}
    for k, (n, ms) in sorted(prof_full.items(), key=lambda kv: -kv[1][1]):
        if n:
            kfull[k] = {"launches": n, "total_ms": ms, "avg_ms": ms / n}
    qa = kfull.get("qinv_apply_f32")
    if qa:
        # one source: per site the 12x12 block Sigma_t^-1 read once (1152 B in FP32; the kernel's
        # four sweeps read it twice whole and twice half) and the spinor in and out (96 B each)
        gbs = (1152.0 + 2 * 96.0) * sites / (qa["avg_ms"] * 1e-3) / 1e9
        qa.update({"gbs": gbs, "hbm_frac": gbs / peak, "hbm_peak": kind})
    w.close()
    print(json.dumps({"mode": "clover", "workload": f"{name}: 16^3x128, xi=3.5, 1 Gaussian source",
                      "c_s": c_s, "c_t": c_t, "u_s": u_s, "tol": args.tol, "results": rows,
                      "kernels_one_fp32_ilu_solve": kern, "kernels_one_fp32_full_sw_solve": kfull}))
    return 0


def run_fullsw(args):
    """--mode fullsw: full SW temporal preconditioning on 16^3 x 128, xi = 3.5, tree-level tadpole
    clover coefficients (as --mode clover). The factorisation of T_0 per precision, timed on a freshly
    loaded field; then per-kernel CUDA-event times of M-hat_full applies in FP32 and FP64 with 1 and
    12 sources (the factors are reused; each call checks their fingerprint), and the Q^-1 kernel
    against HBM in algorithmic bytes: per site the blocks Sigma_t^-1 and Z_t, each read once and
    shared by the line's sources, and per site and source the spinor in and out."""
    import torch

    import paper_0910_0992_gb300 as wf
    import synthetic as S

    name = "wilson_16c128_xi3.5"
    prm, U, _ = S.workload(name)
    xi = prm["kappa_t"] / prm["kappa_s"]
    u_s = spatial_plaquette(U) ** 0.25
    c_s = 1.0 / (u_s ** 3 * xi)
    c_t = (1.0 + 1.0 / xi) / (2.0 * u_s ** 2)
    stream = torch.cuda.Stream()
    w = wf.Wilson(prm["L"], prm["T"], prm["kappa_s"], kappa_t=prm["kappa_t"], bc=prm["bc"])
    w.set_stream(stream.cuda_stream)
    w.load_gauge_clover(U, c_s, c_t)
    half = wf.wf_half_elems(w.h)
    sites = prm["L"] ** 3 * prm["T"] // 2  # one parity: one launch of the Q^-1 kernel
    peak, kind = measured_peak()
    g = torch.Generator(device="cuda").manual_seed(7)
    setup = {}
    for f32 in (True, False):
        w.load_gauge_clover(U, c_s, c_t)  # a fresh field: the next call factors again
        x = torch.randn(1, half, dtype=torch.complex128, device="cuda", generator=g)
        wf.wf_profile(w.h, 1)
        (wf.wf_apply_schur_full_sw_f32 if f32 else wf.wf_apply_schur_full_sw)(w.h, x, torch.empty_like(x), 0, 1)
        prof = wf.wf_profile_get(w.h)
        wf.wf_profile(w.h, 0)
        setup["fp32" if f32 else "fp64"] = {k: {"launches": n, "total_ms": ms} for k, (n, ms) in prof.items()
                                            if n and (k.startswith("qinv_setup") or k == "fsw_fingerprint")}
    rows = []
    for nrhs in (1, 12):
        x = torch.randn(nrhs, half, dtype=torch.complex128, device="cuda", generator=g)
        out = torch.empty_like(x)
        for f32 in (True, False):
            fn = wf.wf_apply_schur_full_sw_f32 if f32 else wf.wf_apply_schur_full_sw
            for _ in range(max(1, args.warmup)):
                fn(w.h, x, out, 0, nrhs)
            wf.wf_profile(w.h, 1)
            reps = max(1, args.steps)
            for _ in range(reps):
                fn(w.h, x, out, 0, nrhs)
            prof = wf.wf_profile_get(w.h)
            wf.wf_profile(w.h, 0)
            kern = {k: {"launches": n, "avg_ms": ms / n} for k, (n, ms) in prof.items() if n}
            tag = "f32" if f32 else "f64"
            qa = kern.get("qinv_apply_" + tag)
            csz = 8 if f32 else 16
            if qa:
                byts = (2 * 144 * csz + nrhs * 2 * 12 * csz) * sites
                gbs = byts / (qa["avg_ms"] * 1e-3) / 1e9
                qa.update({"bytes_per_launch": byts, "gbs": gbs, "hbm_frac": gbs / peak, "hbm_peak": kind})
            apply_ms = sum(v["avg_ms"] * v["launches"] for k, v in kern.items()) / reps
            rows.append({"nrhs": nrhs, "precision": "fp32" if f32 else "fp64", "apply_ms": apply_ms, "kernels": kern})
    w.close()
    print(json.dumps({"mode": "fullsw", "workload": f"{name}: 16^3x128, xi=3.5, random odd fields",
                      "c_s": c_s, "c_t": c_t, "factorisation": setup, "results": rows}))
    return 0


# GB300 FP64 rate: 152 SMs x 2 FP64 FMA per clock x 2 FLOP x 2.07 GHz (maximum SM clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def run_logdet(args):
    """--mode logdet: log det(mu - D_t) and its force (wf_temporal_logdet) on 24^3 x 128 and the two
    force workloads, both frames: per-kernel CUDA-event times, and the force kernel against the
    FP64 rate (two 3x3 complex products and the projection, 448 FLOP per site) and against HBM
    (A(t) read 144 B, force written 256 B per site)."""
    import torch

    import paper_0910_0992_gb300 as wf
    import synthetic as S

    peak_bw, peak_kind = measured_peak()
    rows = []
    for name in (WORKLOAD, "force_8c32_xi3", "force_16c64_xi3"):
        prm, U, _ = S.workload(name, with_sources=False)
        L, T = prm["L"], prm["T"]
        V = L ** 3 * T
        F = torch.empty((V, 4, 8), dtype=torch.float64, device="cuda")
        for axial in (True, False):
            w = wf.Wilson(L, T, prm["kappa_s"], kappa_t=prm["kappa_t"], bc=prm["bc"], axial=axial)
            w.load_gauge(U)
            for _ in range(max(3, args.warmup)):
                w.temporal_logdet(F)
            torch.cuda.synchronize()
            n0 = wf.wf_launch_count(w.h)
            wf.wf_profile(w.h, 1)
            t0 = time.perf_counter()
            for _ in range(args.steps):
                val = w.temporal_logdet(F)
            call_ms = (time.perf_counter() - t0) / args.steps * 1e3
            prof = wf.wf_profile_get(w.h)
            wf.wf_profile(w.h, 0)
            kern = {k: {"launches": n, "avg_ms": ms / n} for k, (n, ms) in prof.items()}
            r = {"workload": name, "frame": "axial" if axial else "caller", "logdet": val, "call_ms": call_ms,
                 "launches_per_call": (wf.wf_launch_count(w.h) - n0) / args.steps, "kernels": kern}
            fk = kern.get("tdet_force_f64")
            if fk:
                sec = fk["avg_ms"] * 1e-3
                tflops = 448.0 * V / sec / 1e12
                gbs = 400.0 * V / sec / 1e9
                r["force_kernel"] = {"fp64_tflops": tflops, "fp64_peak_tflops": FP64_PEAK_TFLOPS,
                                     "fp64_frac": tflops / FP64_PEAK_TFLOPS, "hbm_gbs": gbs,
                                     "hbm_frac": gbs / peak_bw, "hbm_peak": peak_kind}
            rows.append(r)
            w.close()
        del F
    print(json.dumps({"mode": "logdet", "steps": args.steps, "results": rows}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp64", "fp16mix"], default="fp32")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the same-GPU 4-D even-odd comparison")
    ap.add_argument("--mode", choices=["solve", "apply", "methods", "sweep", "force", "logdet", "clover", "fullsw"], default="solve",
                    help="apply: only FP32 M-hat applies (for kernel profiling); methods: every solve method "
                         "on 16^3x128; sweep: temporal+Schur vs 4-D even-odd over xi; force: force timings; "
                         "logdet: the temporal-preconditioner determinant and its force; clover: the clover operator "
                         "with partial temporal preconditioning and 3-D ILU; fullsw: the applies of full SW temporal "
                         "preconditioning")
    ap.add_argument("--nrhs", type=int, default=1, help="sources per apply in --mode apply")
    ap.add_argument("--op", choices=["schur", "eo4d"], default="schur", help="operator of --mode apply")
    ap.add_argument("--workload", default=None, help="--mode apply only: another synthetic workload by name")
    args = ap.parse_args()

    import synthetic as S

    if args.mode in ("methods", "sweep", "force", "logdet", "clover", "fullsw"):
        return {"methods": run_methods, "sweep": run_sweep, "force": run_force, "logdet": run_logdet,
                "clover": run_clover, "fullsw": run_fullsw}[args.mode](args)
    name = WORKLOAD
    if args.workload:
        if args.mode != "apply" or args.workload not in S.WORKLOADS:
            ap.error("--workload needs --mode apply and a known workload name")
        name = args.workload
    prm = dict(S.WORKLOADS[name])
    if args.impl == "reference":
        return run_reference(args, prm)
    _, U, eta = S.workload(name, with_sources=args.mode == "solve")
    if args.mode == "apply":
        return run_apply(args, prm, U, eta)
    return run_ours(args, prm, U, eta)


if __name__ == "__main__":
    sys.exit(main())
