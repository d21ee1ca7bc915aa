"""Benchmark of the butterfly-factorization apply on GB300.

Default workload: 2-D FIO K = exp(2 pi i (x.xi + c(x)|xi|)), polar tree on Omega,
n = 256 (N = 65,536), depth L = 6, rank r = 24.  One *step* is one full apply
u = K_f g (all stages: (V^L)^*, (H^l)^*, M^h, G^l, U^L) of one batch of synthetic
input already resident in HBM.  The headline leg applies 64 RHS on the tensor cores
(split-BF16x3); a second leg applies 1 RHS with the FP32 SIMT kernel.  Factors (about
420 MB of complex64; 450 MB of tensor tiles) exceed the 129 MB L2, so no flush is
needed between steps.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle's FP64
factor apply on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from mbf_synth import SERVE_MIX, WORKLOADS, complex_normal, request_stream  # noqa: E402

METRIC = "MBF apply points·RHS/s & %HBM/TC roofline; serve p50/p99 at rel err ≤1e-4"
UNIT = "points*RHS/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="mbf", choices=["mbf", "reference"])
    p.add_argument("--workload", default="fio2_polar_n256_L6_r24")
    p.add_argument("--nrhs", type=int, default=0, help="override the workload's RHS count")
    p.add_argument("--precision", default="auto", choices=["auto", "fp32_simt", "bf16x3", "tf32"],
                   help="auto: FP32 SIMT below 8 RHS, split-BF16x3 tensor cores from 8 RHS")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-serve", action="store_true", help="skip the served-mix experiment")
    p.add_argument("--serve-requests", type=int, default=512)
    p.add_argument("--no-small", action="store_true", help="skip the 2-D DFT n = 64 latency leg")
    p.add_argument("--factor-file", default=None,
                   help="factor checkpoint to load (or write) instead of building: the workload's file, "
                        "or for the multiscale leg the files <path>.t<k>")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# arithmetic of each precision: (the type the MMAs / FMAs take, what it means)
DTYPES = {
    "bf16x3": ("bf16x3+f32", "complex64 data; tensor cores: each f32 operand split into bf16 hi + lo, "
                             "hi*hi + hi*lo + lo*hi, f32 accumulation; leaf kernels f32"),
    "tf32": ("tf32+f32", "complex64 data; tensor cores: tf32 operands, f32 accumulation; leaf kernels f32"),
    "fp32_simt": ("f32", "complex64 data; f32 FMA, f32 accumulation"),
}


def max_over_ranks(x, world, device):
    """The largest x over the ranks (the slowest replica sets the job's time); x itself
    on one rank.  Needs the default process group when world > 1."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


KERNEL_SOURCES = {"bf_apply_simt": ("apply_simt.cu", "layout.hpp"),
                  "bf_apply_tc": ("apply_tc.cu", "layout.hpp", "apply.hpp")}


def _code_only(text):
    """Source text without comments and blank lines: edits to comments leave it unchanged."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*", "", ln).rstrip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln)


def kernel_source_hash(kernel):
    """Hash of the code (comments stripped) of the sources a kernel is compiled from:
    its DRAM traffic record is only used while that code is unchanged."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1509_07925_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload, nrhs, kernel):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the
    current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    ent = d.get(f"{workload}/nrhs{nrhs}")
    if not ent or ent.get("kernel_hash") != kernel_source_hash(kernel):
        return None
    return ent.get("dram_bytes_per_launch")


def build_factors(bd, wl, factor_file=None):
    """Host FP64 construction of the workload's factors; with factor_file, loaded from
    that checkpoint when it exists (and matches), else built and written there."""
    tree = {"none": bd.MBF_TREE_UNIFORM, "polar": bd.MBF_TREE_POLAR}[wl.transform]
    return bd.HostFactors.build(wl.dim, wl.n, wl.L, wl.r, tree=tree, kernel=wl.kernel,
                                seed=wl.seed_build, factor_file=factor_file)


def oracle_apply_rate(hf, wl, nrhs, budget_s=15.0, threads=None):
    """Time the oracle's FP64 sparse factor apply (as it stands) on the same factors,
    its RHS split across `threads` host threads (default: every core; scipy's sparse
    products release the GIL), bounded by `budget_s` of wall time.
    Returns (points*RHS/s, sample text, threads)."""
    from concurrent.futures import ThreadPoolExecutor
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from gpu_util import export_factors  # noqa: WPS433
    from oracle import bf as B
    sb = B.SparseBF(export_factors(hf.arrays()))
    g = complex_normal(wl.N, nrhs, seed=wl.seed_g)
    nt = max(1, min(threads or os.cpu_count() or 1, nrhs))
    parts = [g[k::nt] for k in range(nt)]
    sb.apply(g[:1])                           # warm-up
    with ThreadPoolExecutor(nt) as ex:
        t0 = time.perf_counter()
        reps = 0
        while True:
            list(ex.map(sb.apply, parts))
            reps += 1
            if time.perf_counter() - t0 > budget_s or reps >= 50:
                break
        dt = (time.perf_counter() - t0) / reps
    sample = (f"{reps} FP64 sparse factor applies of {nrhs} RHS (N={wl.N}), scipy CSR, "
              f"RHS split over {nt} threads")
    return wl.N * nrhs / dt, sample, nt


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_1509_07925_gb300 import binding as bd
    from paper_1509_07925_gb300 import buildlib
    buildlib.build()
    wl = WORKLOADS[args.workload]
    nrhs = args.nrhs or 64
    hf = build_factors(bd, wl, args.factor_file)
    rates = []
    for k in range(args.warmup + args.steps):
        r, sample, cores = oracle_apply_rate(hf, wl, nrhs, budget_s=2.0)
        if k >= args.warmup:
            rates.append(r)
    v = statistics.median(rates)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wl.N * nrhs / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": wl.name, "n": wl.n, "N": wl.N, "L": wl.L,
                                            "r": wl.r, "nrhs": nrhs, "tree": wl.transform,
                                            "kernel": wl.kernel},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_applies(torch, op, g, u, nrhs, prec, steps, stream, adjoint=False):
    """Device time per apply over `steps` back-to-back applies (CUDA events on the stream)."""
    sp = stream.cuda_stream
    fn = op.apply_adjoint if adjoint else op.apply
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        fn(g.data_ptr(), u.data_ptr(), nrhs, prec, sp)
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / steps


def kernel_times(torch, op, g, u, nrhs, prec, steps, stream, adjoint=False):
    """Per-kernel device time per apply: a second pass with the library's kernel timing
    on (CUDA events around each launch, on the apply's stream)."""
    fn = op.apply_adjoint if adjoint else op.apply
    op.set_profiling(True)
    for _ in range(steps):
        fn(g.data_ptr(), u.data_ptr(), nrhs, prec, stream.cuda_stream)
    torch.cuda.synchronize()
    prof = op.profile()
    op.set_profiling(False)
    return {k: {"launches_per_apply": n / steps, "ms_per_apply": ms / steps}
            for k, (n, ms) in prof.items() if n}


def small_dft_leg(torch, bd, stream, steps, warmup, name="dft2_n64_L4_r16"):
    """The 2-D DFT at n = 64 (N = 4096, L = 4, r = 16), one RHS on the FP32 SIMT apply.
    Its factors (about 9 MB) stay in the 129 MB L2 between applies, so the figure of
    merit is the latency of one apply and the algorithmic bytes it moves per second,
    not a fraction of HBM bandwidth."""
    wl = WORKLOADS[name]
    op = bd.Operator(build_factors(bd, wl))
    info = op.info()
    sp = stream.cuda_stream
    g = torch.from_numpy(complex_normal(wl.N, 1, seed=wl.seed_g).astype(np.complex64)).cuda()
    u = torch.empty((1, wl.N), dtype=torch.complex64, device="cuda")
    for _ in range(max(3, warmup)):
        op.apply(g.data_ptr(), u.data_ptr(), 1, bd.MBF_PREC_FP32_SIMT, sp)
    op.check(sp)
    n = max(steps, 100)
    ms = timed_applies(torch, op, g, u, 1, bd.MBF_PREC_FP32_SIMT, n, stream)
    op.check(sp)
    alg = info.bytes_algorithmic + 16 * wl.N
    eps = op.estimate_error(wl.kernel, n_samples=wl.N, seed=wl.seed_s, stream=sp)
    op.close()
    return {"workload": name, "nrhs": 1, "precision": "fp32_simt", "applies": n,
            "latency_us": ms * 1e3, "value": wl.N / (ms * 1e-3), "unit": UNIT,
            "algorithmic_bytes": alg, "achieved_gbs": alg / (ms * 1e-3) / 1e9,
            "l2_resident": True, "eps_full_direct": eps,
            "timing": "back-to-back applies on one stream, CUDA events; factors L2-resident"}


def serve_experiment(torch, bd, ops, n_requests, loads=(0.5, 0.8, 1.1)):
    """The served mix: n_requests seeded requests (operator uniform over `ops`, RHS
    uniform 1..32), first as a closed-loop flood (all submitted at once) to find the
    saturation rate, then as Poisson arrivals at fractions of it.  Latency = device
    completion - submission, from the server's own clock.  A few results are checked
    against the same request applied alone."""
    names = [nm for nm, _ in ops]
    base = request_stream(n_requests, names, rate_hz=1.0, max_rhs=32, seed=2)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2)
    byname = dict(ops)
    bufs = []
    for _, nm, R in base:
        op, N = byname[nm]
        g = torch.randn((R, N), dtype=torch.complex64, device="cuda", generator=gen)
        u = torch.empty((R, N), dtype=torch.complex64, device="cuda")
        bufs.append((g, u))
    torch.cuda.synchronize()
    work = sum(byname[nm][1] * R for _, nm, R in base)     # points x RHS of all requests

    def run(arrivals):
        srv = bd.Server(staging_budget_bytes=4 << 30, max_inflight=4, max_batch_rhs=64)
        pending, lat, t_first, t_last = {}, [], None, 0.0
        k = 0
        t0 = time.perf_counter()
        while k < len(base) or pending:
            now = time.perf_counter() - t0
            while k < len(base) and arrivals[k] <= now:
                _, nm, R = base[k]
                g, u = bufs[k]
                try:
                    tk = srv.submit(byname[nm][0], g.data_ptr(), u.data_ptr(), R)
                except bd.MbfError as e:
                    if e.code != bd.MBF_ERR_BUSY:
                        raise
                    break                                   # retry at the next sweep
                pending[tk] = k
                k += 1
            for tk in list(pending):
                st = srv.poll(tk)
                if st.state == bd.MBF_REQ_DONE:
                    lat.append(st.t_done - st.t_submit)
                    t_first = st.t_submit if t_first is None else min(t_first, st.t_submit)
                    t_last = max(t_last, st.t_done)
                    del pending[tk]
                elif st.state == bd.MBF_REQ_ERROR:
                    raise RuntimeError(f"served request failed: status {st.error}")
        stats = srv.stats()
        srv.close()
        wall = t_last - t_first
        lat_ms = np.array(lat) * 1e3
        return {"p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
                "value": work / wall, "requests_per_s": len(base) / wall, "wall_s": wall,
                "batches": int(stats.batches), "coalesced_requests": int(stats.coalesced_requests),
                "max_batch_requests": int(stats.max_batch_requests),
                "max_concurrent_batches": int(stats.max_concurrent_batches),
                "graph_launches": int(stats.graph_launches), "rejected_busy": int(stats.rejected_busy)}

    run([0.0] * len(base))                                 # warm-up (graphs, workspaces)
    flood = run([0.0] * len(base))
    sat = flood["requests_per_s"]
    out = {"requests": len(base), "operators": names, "rhs": "uniform 1..32", "flood": flood, "loads": []}
    for f in loads:
        arr = [t / (f * sat) for t, _, _ in base]           # unit-rate Poisson times, rescaled
        r = run(arr)
        r["offered"] = f
        out["loads"].append(r)
    # spot check: a few served results equal the same request applied alone
    worst = 0.0
    for k in range(0, len(base), max(1, len(base) // 8)):
        _, nm, R = base[k]
        g, u = bufs[k]
        ref = torch.empty_like(u)
        byname[nm][0].apply(g.data_ptr(), ref.data_ptr(), R, bd.MBF_PREC_AUTO,
                            torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        worst = max(worst, float(torch.linalg.norm(u - ref) / torch.linalg.norm(ref)))
    out["served_vs_alone_max_rel"] = worst
    return out


MSBF_WORKLOAD = "fio2_msbf_n512_r24_x32"


def msbf_bench(args, torch, bd, stream, peak, peak_kind):
    """The multiscale workload: 2-D isotropic FIO, n = 512, r = 24, 16 x 16 centre,
    coronas t = 0..4, 32 RHS on the tensor cores (split-BF16x3).  Not a default leg: its
    host construction takes minutes.  One step = one apply of eq. (f1) (every corona's
    factorization plus the dense centre) to a 32-RHS panel."""
    n, r, nrhs = 512, 24, args.nrhs or 32
    N = n * n
    t0 = time.time()
    m = bd.MsBF.build(n, r, kernel="fio_iso", n_center=16, seed=7, factor_file=args.factor_file)
    t_build = time.time() - t0
    info = m.info()
    sp = stream.cuda_stream
    g = torch.from_numpy(complex_normal(N, nrhs, seed=0).astype(np.complex64)).cuda()
    u = torch.empty((nrhs, N), dtype=torch.complex64, device="cuda")
    for _ in range(max(3, args.warmup)):
        m.apply(g.data_ptr(), u.data_ptr(), nrhs, bd.MBF_PREC_BF16X3, sp)
    m.check(sp)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    ev0.record(stream)
    for _ in range(args.steps):
        m.apply(g.data_ptr(), u.data_ptr(), nrhs, bd.MBF_PREC_BF16X3, sp)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    m.check(sp)
    # end to end: pinned host panel in, result out, inside the timed region
    gh = g.cpu().pin_memory()
    uh = torch.empty((nrhs, N), dtype=torch.complex64).pin_memory()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _ in range(max(3, args.steps // 2)):
        g.copy_(gh, non_blocking=True)
        m.apply(g.data_ptr(), u.data_ptr(), nrhs, bd.MBF_PREC_BF16X3, sp)
        uh.copy_(u, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t1) / max(3, args.steps // 2)
    fac_bytes = info.bytes_algorithmic + 8 * info.n_center_points * N
    step_bytes = fac_bytes + 16 * N * nrhs
    achieved = step_bytes / (ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": N * nrhs / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES["bf16x3"][0], "dtype_detail": DTYPES["bf16x3"][1],
        "data": "synthetic",
        "config": {"workload": MSBF_WORKLOAD, "kernel": "fio_iso", "tree": "multiscale", "n": n, "N": N, "r": r,
                   "n_center": 16, "coronas": [int(info.part_t[i]) for i in range(info.n_parts)],
                   "corona_depths": [int(info.part_L[i]) for i in range(info.n_parts)], "nrhs": nrhs,
                   "precision": "bf16x3", "l2": f"inputs larger than L2: factors {fac_bytes / 1e9:.1f} GB",
                   "factor_bytes_algorithmic": fac_bytes, "host_build_s": t_build},
        "roofline": {"bound": "hbm", "kernel": "whole apply (every kernel of the step)", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "peak_kind": f"{peak_kind} hbm_gbs (burst copy)", "algorithmic_bytes_per_launch": step_bytes,
                     "algorithmic_bytes": "8 B x nonzeros of every corona's factors + 8 B x the dense centre "
                                          "entries + 8 B in + 8 B out per point and RHS, per step"},
        "e2e": {"value": N * nrhs / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * N * nrhs,
                "d2h_bytes_per_step": 8 * N * nrhs},
        "gpu_launches": None, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    m.close()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1509_07925_gb300 import binding as bd
    from paper_1509_07925_gb300 import buildlib
    if rank == 0:
        buildlib.build()
    if world > 1:
        torch.distributed.barrier()
    buildlib.build()
    if args.workload == MSBF_WORKLOAD:
        peak, peak_kind = measured_peaks()
        return msbf_bench(args, torch, bd, torch.cuda.current_stream(), peak, peak_kind)
    wl = WORKLOADS[args.workload]
    N = wl.N
    hf = build_factors(bd, wl, args.factor_file)
    op = bd.Operator(hf)
    info = op.info()
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    peak, peak_kind = measured_peaks()

    # legs: the headline (64 RHS on tensor cores, or --nrhs / --precision) and the
    # single-RHS FP32 SIMT apply it is compared with
    nrhs = args.nrhs or 64
    if args.precision == "auto":
        args.precision = "bf16x3" if nrhs >= 8 else "fp32_simt"
    prec = {"fp32_simt": bd.MBF_PREC_FP32_SIMT, "bf16x3": bd.MBF_PREC_BF16X3,
            "tf32": bd.MBF_PREC_TF32}[args.precision]
    legs = [("headline", nrhs, prec, args.precision)]
    if not (nrhs == 1 and args.precision == "fp32_simt"):
        legs.append(("simt_1rhs", 1, bd.MBF_PREC_FP32_SIMT, "fp32_simt"))
    if nrhs >= 8 and args.precision == "bf16x3":
        # the same panel with TF32 operands (precision sweep: about 1e-3 relative error
        # against 1e-5 for split-BF16x3, measured by the full-size GPU test)
        legs.append(("tf32", nrhs, bd.MBF_PREC_TF32, "tf32"))
        # the adjoint K^* u of the same panel on the tensor cores
        legs.append(("adjoint", nrhs, bd.MBF_PREC_BF16X3, "bf16x3"))
    res = {}
    clocks = ClockSampler(local)
    clk = None
    for name, R, pr, prname in legs:
        adj = name == "adjoint"
        apply_fn = op.apply_adjoint if adj else op.apply
        g = torch.from_numpy(complex_normal(N, R, seed=wl.seed_g).astype(np.complex64)).cuda()
        u = torch.empty((R, N), dtype=torch.complex64, device="cuda")
        for _ in range(max(3, args.warmup)):
            apply_fn(g.data_ptr(), u.data_ptr(), R, pr, sp)
        op.check(sp)
        torch.cuda.synchronize()
        if name == "headline":
            clocks.start()
            time.sleep(0.3)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ms = timed_applies(torch, op, g, u, R, pr, args.steps, stream, adjoint=adj)
        if world > 1:
            torch.distributed.barrier()
        ms = max_over_ranks(ms, world, "cuda")
        if name == "headline":
            clk = clocks.stop()
        op.check(sp)
        kt = kernel_times(torch, op, g, u, R, pr, args.steps, stream, adjoint=adj)
        op.check(sp)
        res[name] = {"nrhs": R, "precision": prname, "ms": ms, "value": world * N * R / (ms * 1e-3),
                     "kernels": kt}
        del g, u

    # roofline of the dominant kernel of the headline leg: algorithmic bytes are the
    # factor nonzeros it applies (8 B each, complex64), the method's O(N log N) work
    head = res["headline"]
    R = head["nrhs"]
    nL = info.c ** info.L
    vec_bytes = 8 * R * nL * (info.RV[info.L] + info.RU[info.L])   # level-L vectors in and out
    if head["precision"] in ("bf16x3", "tf32"):
        kname = "bf_apply_tc"
        nnz_tc = sum(info.nnz_stage[s] for s in range(1, info.n_stages)) - info.nnz_leaf_u
        alg_bytes = 8 * nnz_tc
        alg_note = ("8 B x nonzeros of the G/H factors (S folded into G^h), per launch (one "
                    "64-RHS panel); the level-L coefficient vectors it reads and writes are "
                    "reported apart (level_L_vector_bytes)")
    else:
        kname = "bf_apply_simt"
        alg_bytes = info.bytes_algorithmic + 16 * N * R
        alg_note = "8 B x nonzeros of all factors + 8 B in + 8 B out per point and RHS"
    k_ms = head["kernels"][kname]["ms_per_apply"] / head["kernels"][kname]["launches_per_apply"]
    achieved = alg_bytes / (k_ms * 1e-3) / 1e9
    traffic = recorded_traffic(wl.name, R, kname)
    step_bytes = info.bytes_algorithmic + 16 * N * R
    step_gbs = step_bytes / (head["ms"] * 1e-3) / 1e9

    # factorization error of the benchmarked operator (§3.3 estimator: one FP32 apply
    # against the direct sum on sampled outputs), so that the throughput is read with it
    eps = op.estimate_error(wl.kernel, n_samples=wl.n_sample or 256, seed=wl.seed_s, stream=sp)

    # end to end through the C ABI with host buffers (copies inside the timed region)
    g_host = torch.from_numpy(complex_normal(N, R, seed=wl.seed_g).astype(np.complex64)).pin_memory()
    u_host = torch.empty((R, N), dtype=torch.complex64).pin_memory()
    import ctypes as C
    lib = bd.lib()
    hprec = {"fp32_simt": bd.MBF_PREC_FP32_SIMT, "bf16x3": bd.MBF_PREC_BF16X3,
             "tf32": bd.MBF_PREC_TF32}[head["precision"]]
    for _ in range(2):
        bd._check(lib.mbf_apply_host(op.handle, C.c_void_p(g_host.data_ptr()),
                                     C.c_void_p(u_host.data_ptr()), R, hprec, C.c_void_p(sp)))
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    n_single = max(3, args.steps // 2)
    for _ in range(n_single):
        bd._check(lib.mbf_apply_host(op.handle, C.c_void_p(g_host.data_ptr()),
                                     C.c_void_p(u_host.data_ptr()), R, hprec, C.c_void_p(sp)))
    single_s = max_over_ranks((time.perf_counter() - t0) / n_single, world, "cuda")
    # the pipelined host API: K panels (one per step, each its own page-locked block)
    # in one call; the copy engines move panel k+1 in and panel k-1 out while panel k is
    # applied, and every byte of every panel crosses the host link inside the timed call
    n_e2e = max(4, args.steps)
    g_batch = g_host.unsqueeze(0).repeat(n_e2e, 1, 1).pin_memory()
    u_batch = torch.empty((n_e2e, R, N), dtype=torch.complex64).pin_memory()
    for _ in range(2):
        bd._check(lib.mbf_apply_host_batch(op.handle, C.c_void_p(g_batch.data_ptr()),
                                           C.c_void_p(u_batch.data_ptr()), min(n_e2e, 3), R, hprec,
                                           C.c_void_p(sp)))
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    bd._check(lib.mbf_apply_host_batch(op.handle, C.c_void_p(g_batch.data_ptr()),
                                       C.c_void_p(u_batch.data_ptr()), n_e2e, R, hprec, C.c_void_p(sp)))
    e2e_s = max_over_ranks((time.perf_counter() - t0) / n_e2e, world, "cuda")
    e2e_err = float(np.max(np.abs(u_batch[-1].numpy() - u_host.numpy())) /
                    max(1e-30, float(np.max(np.abs(u_host.numpy())))))

    launches = sum(k["launches_per_apply"] for k in head["kernels"].values())
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[head["precision"]][0],
        "dtype_detail": DTYPES[head["precision"]][1], "data": "synthetic",
        "config": {"workload": wl.name, "kernel": wl.kernel, "tree": wl.transform, "n": wl.n, "N": N,
                   "L": wl.L, "r": wl.r, "nrhs": R, "precision": head["precision"],
                   "parallelism": f"replicas{world}",
                   "l2": f"inputs larger than L2: packed factors {info.bytes_packed / 1e6:.0f} MB "
                         f"(tensor tiles {info.bytes_tensor / 1e6:.0f} MB) > 129 MB",
                   "factor_bytes_algorithmic": info.bytes_algorithmic,
                   "factor_bytes_packed": info.bytes_packed},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": f"{peak_kind} hbm_gbs (burst copy)",
                     "algorithmic_bytes_per_launch": alg_bytes, "algorithmic_bytes": alg_note,
                     "kernel_ms_per_launch": k_ms,
                     "level_L_vector_bytes": vec_bytes if kname == "bf_apply_tc" else None,
                     "step": {"algorithmic_bytes": step_bytes, "ms": head["ms"], "achieved": step_gbs,
                              "frac": step_gbs / peak,
                              "note": "whole apply (all kernels): 8 B x nonzeros of every factor + "
                                      "8 B in + 8 B out per point and RHS, over the step time"}},
        "legs": res,
        "e2e": {"value": world * N * R / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * N * R,
                "d2h_bytes_per_step": 8 * N * R, "api": "mbf_apply_host_batch", "panels_per_call": n_e2e,
                "ms_per_panel": e2e_s * 1e3, "max_rel_diff_vs_single_call": e2e_err,
                "single_call": {"api": "mbf_apply_host", "value": world * N * R / single_s,
                                "ms_per_call": single_s * 1e3}},
        "gpu_launches": int(round(launches * args.steps)),
        "clocks": clk,
    }
    if "simt_1rhs" in res:
        line["speedup_vs_simt_1rhs"] = head["value"] / res["simt_1rhs"]["value"]
    line["eps"] = {"value": eps, "samples": wl.n_sample or 256,
                   "what": "relative L2 error of the operator (one FP32 apply) against the direct "
                           "sum u = K g on sampled outputs, the error estimator of §3.3; the "
                           "factorization error of this operator, not an arithmetic error"}
    if not args.no_small and world == 1:
        line["small_dft"] = small_dft_leg(torch, bd, stream, args.steps, args.warmup)
    if not args.no_serve and world == 1:
        serve_ops, keep = [], []
        for nm in SERVE_MIX:
            if nm == wl.name:
                serve_ops.append((nm, (op, N)))
            else:
                w2 = WORKLOADS[nm]
                o2 = bd.Operator(build_factors(bd, w2))
                keep.append(o2)
                serve_ops.append((nm, (o2, w2.N)))
        line["serve"] = serve_experiment(torch, bd, serve_ops, args.serve_requests)
        for o2 in keep:
            o2.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            v, sample, cores = oracle_apply_rate(hf, wl, R)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": sample}
        except Exception as e:  # the baseline must not hide the GPU number
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 0, "kind": "oracle",
                                    "sample": f"failed: {e}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    op.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
