#!/usr/bin/env python3
"""Throughput of sttsm, C := [A; X, X, X], on the large single-instance workload.

Workload: m = 3, n = p = 768, A symmetric Uniform(-1,1) in BCSS (FP32),
X N(0, 1/n) (FP32), block size b from {32, 48, 64} (chosen by a short
measurement unless --b is given), BF16X6 split-precision tensor-core path.
A step is one sttsm_bcss call: the X split plus the m level launches of the
algorithm-by-blocks.  Useful flops are the paper's BCSS count (Tbl. 4,
MinCosts) — `sttsm_flops`.  Inputs (A: >= 340 MB) are larger than the 129 MB
L2, so no flush is needed between steps.

Also reported: the plain FP64 GPU path on the same workload, the sampled
relative error of both paths against the FP64 oracle, an end-to-end figure
through the host-buffer entry point (H2D of A and X, D2H of C inside the
timed region), the roofline of the dominant kernel from CUDA events the
library records on its launch stream, SM clocks sampled during the timed
region, and the FP64 CPU oracle timed on this host (cpu_baseline).

Multi-GPU (torchrun): every rank runs its own independent instance
(replicas, weak scaling); value = all ranks' useful flops / max time.

`--impl reference` times the FP64 CPU oracle (the dense successive
mode-product chain) on bounded slices of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sttsm TFLOP/s (paper's BCSS flop count) & % peak, BF16x3 vs FP64 at stated rel err; p99 ms"
M, N, P = 3, 768, 768
SEED_A, SEED_X, SEED_J = 0, 1, 2


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--b", default="auto", help="block size or 'auto'")
    ap.add_argument("--prec", default="bf16x6", choices=["bf16x6", "bf16x3", "bf16x6_r64", "bf16x3_r64"])
    ap.add_argument("--no-check", action="store_true", help="skip the oracle error check and CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU-baseline sample time")
    ap.add_argument("--workload", default="single",
                    choices=["single", "m4", "abo", "batch", "serve", "symmetry", "pack"],
                    help="single: m=3 n=p=768 instance (default); m4: m=4 n=128 p=64 compressing instance; "
                         "abo: all modes but one on the m=3 n=p=768 instance; batch: 4096 mixed instances; "
                         "serve: Poisson stream")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--pack-n", type=int, default=768, help="n of the m = 3 FP32 tensor of --workload pack")
    ap.add_argument("--ws-gb", type=float, default=48.0, help="batch workspace budget (GiB)")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-budget-gb", type=float, default=40.0)
    ap.add_argument("--fused-tail", type=int, default=1, choices=[0, 1, 2],
                    help="short contractions' last two levels: 0 two launches, 1 fused in single calls "
                         "(library default), 2 fused in batch plans and serving too")
    ap.add_argument("--inblock-sym", type=int, default=0, choices=[0, 1],
                    help="short contractions: 1 computes the canonical entries of diagonal blocks only "
                         "(sttsm_set_inblock_symmetry), 0 every entry (library default)")
    ap.add_argument("--no-configs", action="store_true",
                    help="leave the m4 / batch / serve short forms out of the default line")
    ap.add_argument("--configs-serve-seconds", type=float, default=10.0,
                    help="length of the serving stream in the default line's short form")
    ap.add_argument("--no-extras", action="store_true",
                    help="time the headline step only (no e2e, FP64 path, check or CPU baseline); for profiling")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def prec_code(st, name):
    return {"bf16x6": st.STTSM_BF16X6, "bf16x3": st.STTSM_BF16X3, "bf16x6_r64": st.STTSM_BF16X6_R64,
            "bf16x3_r64": st.STTSM_BF16X3_R64}[name]


def tensor_peak(pk, pk_src, clk, timed_ms):
    """The BF16 tensor peak that matches a timed region: the burst figure (a cuBLAS
    GEMM timed alone, at full clock) for a region that is short and saw no power
    cap, the sustained one (seconds of GEMMs under the power cap) otherwise."""
    burst = float(pk.get("bf16_tflops", 1900.0))
    sustained = float(pk.get("bf16_tflops_sustained", 1700.0))
    capped = "sw_power_cap" in (clk.get("reasons") or [])
    if timed_ms < 2000.0 and not capped:
        return burst, ("bf16_tflops (burst) of %s MEASURED_PEAKS: timed region %.0f ms, median SM clock %s MHz, "
                       "no power cap seen" % (pk_src, timed_ms, clk.get("sm_mhz")))
    return sustained, ("bf16_tflops_sustained of %s MEASURED_PEAKS: timed region %.0f ms%s"
                       % (pk_src, timed_ms, ", sw_power_cap seen" if capped else ""))


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100"]
            vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
            if vis and "," not in vis:
                cmd += ["-i", vis]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        first = rows[0][0]
        rows = [r for r in rows if r[0] == first]

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ---------------------------------------------------------------- inputs

def xcol32(X):
    return np.asfortranarray(X).reshape(-1, order="F").astype(np.float32)


def make_device_inputs(st, torch, b, dtype):
    import synth
    dense = torch.empty(N ** M, dtype=dtype, device="cuda")
    synth.dev_sym_uniform_dense(dense.data_ptr(), M, N, SEED_A, "f64" if dtype == torch.float64 else "f32",
                                torch.cuda.current_stream().cuda_stream)
    A = torch.empty(st.bcss_num_elems(M, N, b), dtype=dtype, device="cuda")
    st.bcss_pack(dense, A, M, N, b)
    torch.cuda.synchronize()
    del dense
    torch.cuda.empty_cache()
    return A


def pack_bandwidth(st, torch, b, pk, pk_src, reps=5, n=None):
    """bcss_pack (dense -> BCSS) and bcss_unpack (BCSS -> dense) of the FP32
    workload tensor, CUDA events on the current stream, mean of reps launches
    after one untimed launch.  Algorithmic bytes: pack reads and writes each
    stored entry once (4 B each way); unpack writes each dense entry and reads
    its canonical stored entry (4 B each way)."""
    import synth
    n = N if n is None else n
    stream = torch.cuda.current_stream()
    dense = torch.empty(n ** M, dtype=torch.float32, device="cuda")
    synth.dev_sym_uniform_dense(dense.data_ptr(), M, n, SEED_A, "f32", stream.cuda_stream)
    A = torch.empty(st.bcss_num_elems(M, n, b), dtype=torch.float32, device="cuda")
    out = torch.empty_like(dense)
    res = {}
    for name, fn, nbytes in (("pack", lambda: st.bcss_pack(dense, A, M, n, b), 8.0 * A.numel()),
                             ("unpack", lambda: st.bcss_unpack(A, out, M, n, b), 8.0 * dense.numel())):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        gbs = nbytes / (ms * 1e-3) / 1e9
        res[name] = {"ms": ms, "achieved_gbs": gbs, "algorithmic_bytes": nbytes,
                     "frac_of_hbm": gbs / float(pk.get("hbm_gbs", 6800.0))}
    res["bound"] = "hbm"
    res["peak_gbs"] = float(pk.get("hbm_gbs", 6800.0))
    res["peak_source"] = "hbm_gbs of %s MEASURED_PEAKS" % pk_src
    res["bit_exact_round_trip"] = bool(torch.equal(out, dense))
    del dense, A, out
    torch.cuda.empty_cache()
    return res


def bcss_pos(j, b):
    import math
    s = sorted(int(x) for x in j)
    rank = sum(math.comb(s[t] // b + t, t + 1) for t in range(M))
    return rank * b ** M + sum((s[t] % b) * b ** t for t in range(M))


# ---------------------------------------------------------------- CPU oracle (baseline)

def oracle_slice_rate(A_dense, X, target_s, max_slices=None):
    """Times the oracle's dense mode-product chain on S slices C[:, :, j] (j a
    seeded sample of rows of X for the last mode), S sized from one timed
    slice to take about target_s seconds; returns (seconds, S)."""
    import oracle
    rng = np.random.default_rng(SEED_J)
    t0 = time.perf_counter()
    oracle.ttm_chain(A_dense, [X, X, X[rng.integers(0, P, size=1)]], M)
    one = time.perf_counter() - t0
    S = max(1, int(target_s / max(one, 1e-3)))
    if max_slices:
        S = min(S, max_slices)
    rows = rng.integers(0, P, size=S)
    t0 = time.perf_counter()
    oracle.ttm_chain(A_dense, [X, X, X[rows]], M)
    dt = time.perf_counter() - t0
    return dt, S


def cpu_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import synth
    import oracle
    b = 64 if args.b == "auto" else int(args.b)
    F = bcss_flops_host(b)
    A = synth.sym_uniform_dense(M, N, SEED_A)
    X = synth.x_gaussian(SEED_X, P, N).astype(np.float32).astype(np.float64)
    oracle.build()
    per_step = max(2.0, min(10.0, 120.0 / max(1, args.steps + args.warmup)))
    _, S = oracle_slice_rate(A, X, per_step)
    times = []
    for i in range(args.warmup + args.steps):
        dt = _timed_slices(A, X, S, i)
        if i >= args.warmup:
            times.append(dt)
    t = float(np.mean(times))
    value = F * S / P / t / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "sttsm m=3 n=p=768 b=%d" % b, "m": M, "n": N, "p": P, "b": b},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": "FP64 oracle dense mode-product chain on %d of %d slices C[:,:,j] per step; "
                                       "value scales the BCSS flop count by %d/%d" % (S, P, S, P)},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _timed_slices(A, X, S, i):
    import oracle
    rng = np.random.default_rng(SEED_J + 1 + i)
    rows = rng.integers(0, P, size=S)
    t0 = time.perf_counter()
    oracle.ttm_chain(A, [X, X, X[rows]], M)
    return time.perf_counter() - t0


def bcss_flops_host(b):
    """Tbl. 4 (MinCosts) BCSS flop count, restated for the reference leg (no library load)."""
    import math
    nbar, pbar = -(-N // b), -(-P // b)
    s = sum(math.comb(pbar + d, d + 1) * math.comb(nbar + M - d - 2, M - d - 1) for d in range(M))
    return 2.0 * nbar * b ** (M + 1) * s


# ---------------------------------------------------------------- our arm

def max_over_ranks(total_ms, device):
    """The slowest rank's timed-region duration (all ranks call it; needs an
    initialised process group: NCCL on the GPU, gloo in the CPU tests)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(flops_per_rank_step, world, total_ms, steps):
    """Whole-job TFLOP/s: every rank ran `steps` steps of `flops_per_rank_step`
    useful flops (replicas: weak scaling) in the slowest rank's `total_ms`."""
    return flops_per_rank_step * world * steps / (total_ms * 1e-3) / 1e12


def time_steps(torch, fn, steps, warmup, per_step_events=True):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    t_all0.record()
    for i in range(steps):
        ev[i][0].record()
        fn()
        ev[i][1].record()
    t_all1.record()
    torch.cuda.synchronize()
    per = [a.elapsed_time(b_) for a, b_ in ev]
    return t_all0.elapsed_time(t_all1), per


def profiled_traffic(b, prec, kinds):
    """DRAM bytes (read + write) per launch of the level kernel (mean of the m level
    launches of a step), from the committed ncu summary of this workload
    (profiles/traffic.json), or None when no capture of the current kernel for this
    block size exists."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    key = "%s_b%d_%s" % (kinds[0] if kinds else "", b, prec)
    v = d.get(key)
    return v.get("dram_bytes_per_launch") if isinstance(v, dict) else None


def end_to_end(st, torch, A, C, Xh, ws, b, F, prec, world, steps):
    """Same metric through sttsm_bcss_host: every step copies its A and X from
    pinned host buffers to the device, computes, and copies its C back, all inside
    the timed region.  Two forms, each timed over the same number of steps between
    a barrier and a device synchronisation (slowest rank's time):
      * "one stream": the steps one after another on one stream;
      * "two streams": steps alternate between two streams with their own device
        buffers and workspaces, so one step's copies can overlap the neighbouring
        steps' computation, as a pipelined caller would run them.
    The better one is the reported value; the other is kept beside it, with the
    copy bandwidth of each direction measured alone and both at once."""
    hA = A.cpu().pin_memory()
    hX = torch.from_numpy(xcol32(Xh)).pin_memory()
    hC = [torch.empty(C.numel(), dtype=torch.float32).pin_memory() for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    dev = [(torch.empty_like(A), torch.empty(hX.numel(), dtype=torch.float32, device="cuda"), torch.empty_like(C),
            ws if k == 0 else torch.empty_like(ws)) for k in range(2)]

    def step_on(i, k):
        dA2, dX2, dC2, w2 = dev[k]
        st.sttsm_bcss_host(hA, hX, M, N, P, b, hC[i & 1], prec, dA2, dX2, dC2, w2, streams[k].cuda_stream)

    forms = {"two streams": lambda i: step_on(i, i & 1), "one stream": lambda i: step_on(i, 0)}

    def timed(fn, nsteps):
        for i in range(3):
            fn(i)
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(nsteps):
            fn(i)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / nsteps
        return max_over_ranks(ms, "cuda") if world > 1 else ms

    res = {name: timed(fn, steps) for name, fn in forms.items()}
    assert np.array_equal(hC[0].numpy(), C.cpu().numpy()) and np.array_equal(hC[1].numpy(), C.cpu().numpy())
    # copy bandwidth alone: H2D of A, D2H of C, and both directions at once (two streams)
    h2d_bytes, d2h_bytes = hA.numel() * 4, hC[0].numel() * 4

    def copy_ms(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3 / reps

    def both():
        with torch.cuda.stream(streams[0]):
            dev[0][0].copy_(hA, non_blocking=True)
        with torch.cuda.stream(streams[1]):
            hC[1].copy_(dev[1][2], non_blocking=True)

    t_h2d = copy_ms(lambda: dev[0][0].copy_(hA, non_blocking=True))
    t_d2h = copy_ms(lambda: hC[0].copy_(dev[0][2], non_blocking=True))
    t_both = copy_ms(both)
    best = min(res, key=res.get)
    ms = res[best]
    return {"value": F / (ms * 1e-3) / 1e12 * world, "unit": "TFLOP/s", "ms_per_step": ms, "form": best,
            "ms_per_step_by_form": res,
            "value_by_form": {k: F / (v * 1e-3) / 1e12 * world for k, v in res.items()},
            "h2d_bytes_per_step": int(h2d_bytes + hX.numel() * 4), "d2h_bytes_per_step": int(d2h_bytes),
            "timer": "host wall clock over the steps, barrier and device synchronisation at both ends, max over ranks",
            "copy_gbs": {"h2d_alone": h2d_bytes / (t_h2d * 1e-3) / 1e9, "d2h_alone": d2h_bytes / (t_d2h * 1e-3) / 1e9,
                         "h2d_and_d2h_at_once": (h2d_bytes + d2h_bytes) / (t_both * 1e-3) / 1e9,
                         "what": "pinned host <-> device copies of the workload's A (H2D) and C (D2H), 5 reps each"},
            "steps": steps}


def fp64_path(st, torch, Xh, b, F, ms):
    """The plain FP64 GPU path (CUDA-core FMAs) on the same workload."""
    A64 = make_device_inputs(st, torch, b, torch.float64)
    dX64 = torch.from_numpy(np.asfortranarray(Xh).reshape(-1, order="F").copy()).cuda()
    C64 = torch.empty(st.bcss_num_elems(M, P, b), dtype=torch.float64, device="cuda")
    ws64 = st.workspace_tensor(M, N, P, b, st.STTSM_FP64)
    tot64, _ = time_steps(torch, lambda: st.sttsm_bcss(A64, dX64, M, N, P, b, C64, st.STTSM_FP64, ws64), 2, 1)
    ms64 = tot64 / 2
    # FP64 reference rate on this GPU: a library FP64 GEMM (4096^3) timed the same way
    g = 4096
    ga = torch.randn(g, g, dtype=torch.float64, device="cuda")
    gb = torch.randn(g, g, dtype=torch.float64, device="cuda")
    totg, _ = time_steps(torch, lambda: torch.matmul(ga, gb), 3, 1)
    dgemm = 2.0 * g ** 3 / (totg / 3 * 1e-3) / 1e12
    del ga, gb
    value = F / (ms64 * 1e-3) / 1e12
    return ({"value": value, "unit": "TFLOP/s", "ms_per_step": ms64, "speedup_of_split_path": ms64 / ms,
             "library_fp64_gemm_tflops": dgemm, "frac_of_library_fp64_gemm": value / dgemm}, C64)


def check_and_baseline(args, C, C64, Xh, X32, b, F, world, C_r64=None):
    """Sampled relative error of both paths against the FP64 oracle, and the
    oracle itself timed on this host's cores (N = 1 only)."""
    import oracle
    import synth
    oracle.build()
    A_dense = synth.sym_uniform_dense(M, N, SEED_A)
    J = np.sort(np.random.default_rng(SEED_J).integers(0, P, size=(256, M)), axis=1)
    ref32 = oracle.sttsm_entries(A_dense, X32, M, J)
    c32 = C.double().cpu().numpy()
    got32 = np.array([c32[bcss_pos(j, b)] for j in J])
    rel_err = {"samples": 256, args.prec: float(np.linalg.norm(got32 - ref32) / np.linalg.norm(ref32)),
               "tolerance": {args.prec: 1e-6, "fp64": 1e-12},
               "elementwise": {args.prec: float(np.max(np.abs(got32 - ref32)) / np.max(np.abs(ref32)))}}
    if C_r64 is not None:
        cr = C_r64.double().cpu().numpy()
        gotr = np.array([cr[bcss_pos(j, b)] for j in J])
        rel_err["bf16x6_r64"] = float(np.linalg.norm(gotr - ref32) / np.linalg.norm(ref32))
        rel_err["elementwise"]["bf16x6_r64"] = float(np.max(np.abs(gotr - ref32)) / np.max(np.abs(ref32)))
    if C64 is not None:
        ref64 = oracle.sttsm_entries(A_dense, Xh, M, J)
        c64 = C64.cpu().numpy()
        got64 = np.array([c64[bcss_pos(j, b)] for j in J])
        rel_err["fp64"] = float(np.linalg.norm(got64 - ref64) / np.linalg.norm(ref64))
        rel_err["elementwise"]["fp64"] = float(np.max(np.abs(got64 - ref64)) / np.max(np.abs(ref64)))
    cpu_base = None
    if world == 1:
        dt, S = oracle_slice_rate(A_dense, X32, args.cpu_seconds)
        cpu_base = {"value": F * S / P / dt / 1e12, "unit": "TFLOP/s", "cores": cpu_threads(), "kind": "oracle",
                    "sample": "FP64 oracle dense mode-product chain (A x_2 X_S x_1 X x_0 X) for %d of %d "
                              "slices C[:,:,j], %.1f s; value = BCSS flop count x %d/%d / time" % (S, P, dt, S, P)}
        one = oracle_one_core(2)
        if one:
            cpu_base["one_core"] = {"value": F * 2 / P / one / 1e12, "unit": "TFLOP/s", "cores": 1,
                                    "sample": "same chain, 2 slices, %.1f s, OMP_NUM_THREADS=1 in a child process" % one}
    return rel_err, cpu_base


def oracle_one_core(slices):
    """The same oracle chain on one host core (a child process started with
    OMP_NUM_THREADS=1, since the thread count is fixed at the first parallel
    region); returns seconds for `slices` slices, or None on failure."""
    code = ("import sys, time, numpy as np; sys.path.insert(0, %r); import synth, oracle; oracle.build(); "
            "A = synth.sym_uniform_dense(%d, %d, %d); "
            "X = synth.x_gaussian(%d, %d, %d).astype(np.float32).astype(np.float64); "
            "rows = np.random.default_rng(%d).integers(0, %d, size=%d); t0 = time.perf_counter(); "
            "oracle.ttm_chain(A, [X, X, X[rows]], %d); print(time.perf_counter() - t0)"
            % (ROOT, M, N, SEED_A, SEED_X, P, N, SEED_J + 1, P, slices, M))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        return float(out.stdout.strip().splitlines()[-1]) if out.returncode == 0 else None
    except (subprocess.TimeoutExpired, ValueError, IndexError):
        return None


def bcss_pos_m(j, b, m):
    import math
    s = sorted(int(x) for x in j)
    rank = sum(math.comb(s[t] // b + t, t + 1) for t in range(m))
    return rank * b ** m + sum((s[t] % b) * b ** t for t in range(m))


def run_m4(args, emit=True, short=False):
    """The compressing single instance m = 4, n = 128, p = 64 (X with orthonormal
    rows), b in {8, 16, 32}, BF16X6 and FP64: TFLOP/s per (b, precision) and the
    error of 64 sampled C entries against the FP64 oracle.  short: at most 10
    timed steps per case (the form the default bench line carries)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1301_7744_gb300 as st
    st.sttsm_set_fused_tail(args.fused_tail)
    st.sttsm_set_inblock_symmetry(args.inblock_sym)
    import synth
    import oracle
    m, n, p = 4, 128, 64
    stream = torch.cuda.current_stream().cuda_stream
    Xh = synth.x_orthonormal_rows(SEED_X, p, n)
    X32 = Xh.astype(np.float32).astype(np.float64)
    steps, warm = max(3, min(args.steps, 10 if short else 50)), max(3, args.warmup)
    res, keep = {}, {}
    clocks = ClockSampler()
    clocks.start()
    for b in (8, 16, 32):
        for prec, name, dt in ((st.STTSM_BF16X6, "bf16x6", torch.float32), (st.STTSM_FP64, "fp64", torch.float64)):
            dense = torch.empty(n ** m, dtype=dt, device="cuda")
            synth.dev_sym_uniform_dense(dense.data_ptr(), m, n, SEED_A, "f64" if dt == torch.float64 else "f32", stream)
            A = torch.empty(st.bcss_num_elems(m, n, b), dtype=dt, device="cuda")
            st.bcss_pack(dense, A, m, n, b)
            del dense
            Xsrc = Xh if name == "fp64" else X32
            X = torch.from_numpy(np.asfortranarray(Xsrc).reshape(-1, order="F").copy()).to(device="cuda", dtype=dt)
            C = torch.empty(st.bcss_num_elems(m, p, b), dtype=dt, device="cuda")
            ws = st.workspace_tensor(m, n, p, b, prec)
            st.sttsm_profile_enable(True)
            st.sttsm_bcss(A, X, m, n, p, b, C, prec, ws)
            torch.cuda.synchronize()
            kinds = sorted({r["kind"] for r in st.sttsm_profile_read() if r["kind"] != "split"})
            st.sttsm_profile_enable(False)
            tot, per = time_steps(torch, lambda: st.sttsm_bcss(A, X, m, n, p, b, C, prec, ws), steps, warm)
            F = st.sttsm_flops(m, n, p, b)
            res["%s_b%d" % (name, b)] = {"tflops": F / (tot / steps * 1e-3) / 1e12, "ms_per_step": tot / steps,
                                         "p99_ms": float(np.percentile(per, 99)), "level_kernel": kinds}
            keep[(name, b)] = C.double().cpu().numpy()
            del A, C, ws, X
            torch.cuda.empty_cache()
    clk = clocks.stop()
    oracle.build()
    A_dense = synth.sym_uniform_dense(m, n, SEED_A)
    J = np.sort(np.random.default_rng(SEED_J).integers(0, p, size=(64, m)), axis=1)
    ref = {"bf16x6": oracle.sttsm_entries(A_dense, X32, m, J), "fp64": oracle.sttsm_entries(A_dense, Xh, m, J)}
    for (name, b), c in keep.items():
        got = np.array([c[bcss_pos_m(j, b, m)] for j in J])
        res["%s_b%d" % (name, b)]["rel_err"] = float(np.linalg.norm(got - ref[name]) / np.linalg.norm(ref[name]))
    best = max((k for k in res if k.startswith("bf16x6")), key=lambda k: res[k]["tflops"])
    fastest = min((k for k in res if k.startswith("bf16x6")), key=lambda k: res[k]["ms_per_step"])
    line = {"metric": "sttsm TFLOP/s, m=4 n=128 p=64 (compressing)", "value": res[best]["tflops"], "unit": "TFLOP/s",
            "n_gpus": 1, "steps": steps, "warmup": warm, "higher_is_better": True, "dtype": "bf16x6",
            "data": "synthetic", "config": {"workload": "sttsm m=4 n=128 p=64, X orthonormal rows, b in {8,16,32}",
                                            "best": best, "tolerance": {"bf16x6": 1e-6, "fp64": 1e-12},
                                            "oracle_samples": 64},
            "time_to_solution": {"case": fastest, "ms_per_step": res[fastest]["ms_per_step"],
                                 "tflops": res[fastest]["tflops"]},
            "results": res, "clocks": clk}
    if emit:
        print(json.dumps(line), flush=True)
        return 0
    return line


def run_abo(args):
    """Multiplication in all modes but one, B = A x_1 X x_2 X on the m = 3, n = p = 768
    instance (b = 64, BF16X6): TFLOP/s of levels 0 .. m-2 and the error of a 4 x 4 x 4
    grid of sampled entries against the FP64 oracle's chain restricted to those rows."""
    import math
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1301_7744_gb300 as st
    st.sttsm_set_fused_tail(args.fused_tail)
    st.sttsm_set_inblock_symmetry(args.inblock_sym)
    import synth
    import oracle
    b = 64 if args.b == "auto" else int(args.b)
    prec = prec_code(st, args.prec)
    Xh = synth.x_gaussian(SEED_X, P, N)
    X32 = Xh.astype(np.float32).astype(np.float64)
    dX = torch.from_numpy(xcol32(Xh)).cuda()
    A = make_device_inputs(st, torch, b, torch.float32)
    T = torch.empty(st.sttsm_all_but_one_elems(M, N, P, b), dtype=torch.float32, device="cuda")
    ws = st.workspace_tensor(M, N, P, b, prec)
    F = st.sttsm_all_but_one_flops(M, N, P, b)
    steps, warm = max(3, min(args.steps, 100)), max(3, args.warmup)
    clocks = ClockSampler()
    clocks.start()
    tot, per = time_steps(torch, lambda: st.sttsm_bcss_all_but_one(A, dX, M, N, P, b, T, prec, ws), steps, warm)
    clk = clocks.stop()
    ms = tot / steps
    rng = np.random.default_rng(SEED_J)
    ri, rj = np.sort(rng.integers(0, N, size=4)), np.sort(rng.integers(0, P, size=4))
    oracle.build()
    A_dense = synth.sym_uniform_dense(M, N, SEED_A)
    ref = oracle.ttm_chain(A_dense, [np.eye(N)[ri], X32[rj], X32[rj]], M).reshape(4, 4, 4, order="F")
    t = T.double().cpu().numpy()
    nbar = -(-N // b)
    got = np.empty_like(ref)
    for a, i in enumerate(ri):
        for c1, j1 in enumerate(rj):
            for c2, j2 in enumerate(rj):
                lo, hi = sorted((int(j1), int(j2)), key=lambda v: v // b)
                node = math.comb(lo // b + 0, 1) + math.comb(hi // b + 1, 2)
                off = int(i) % b + (lo % b) * b + (hi % b) * b * b
                got[a, c1, c2] = t[(node * nbar + int(i) // b) * b ** M + off]
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    line = {"metric": "sttsm all-but-one TFLOP/s (A x_1 X x_2 X, Tbl. 4 count of levels 0..m-2)", "value": F / (ms * 1e-3) / 1e12,
            "unit": "TFLOP/s", "n_gpus": 1, "steps": steps, "warmup": warm, "ms_per_step": ms,
            "p99_ms_per_step": float(np.percentile(per, 99)), "higher_is_better": True, "dtype": args.prec,
            "data": "synthetic", "config": {"workload": "all modes but one, m=3 n=p=768 b=%d %s" % (b, args.prec.upper()),
                                            "useful_flops_per_step": F},
            "rel_err": {"samples": 64, args.prec: err, "tolerance": 1e-6}, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args, emit=True, short=False):
    """Batched workload: count instances, m in {3,4,5} (weights .5/.3/.2), n in U{8..64},
    p in U{8..n}, b per instance by sttsm_autotune_b over {4, 8, 16}; BF16X6; one
    sttsm_batch_run (a CUDA-graph replay) per step.  Compared with a per-instance loop
    of the plain FP64 path (sttsm_bcss per instance).  short: no FP64 loop and no
    tcgen05 comparison (the form the default bench line carries)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1301_7744_gb300 as st
    st.sttsm_set_fused_tail(args.fused_tail)
    st.sttsm_set_inblock_symmetry(args.inblock_sym)
    import synth
    prec = st.STTSM_BF16X6
    shapes = synth.batch_shapes(3, args.batch_count)
    maxdense = max(n ** m for m, n, _ in shapes)
    scratch32 = torch.empty(maxdense, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    insts, xs = [], []
    bcount = {}
    for i, (m, n, p) in enumerate(shapes):
        b = st.sttsm_autotune_b(m, n, p, prec, (4, 8, 16))
        bcount[b] = bcount.get(b, 0) + 1
        d = scratch32[: n ** m]
        synth.dev_sym_uniform_dense(d.data_ptr(), m, n, 1000 + i, "f32", stream)
        A = torch.empty(st.bcss_num_elems(m, n, b), dtype=torch.float32, device="cuda")
        st.bcss_pack(d, A, m, n, b)
        X = synth.x_gaussian(5000 + i, p, n)
        xs.append(X)
        dX = torch.from_numpy(xcol32(X)).cuda()
        C = torch.empty(st.bcss_num_elems(m, p, b), dtype=torch.float32, device="cuda")
        insts.append((A, dX, C, m, n, p, b))
    torch.cuda.synchronize()
    del scratch32
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    plan = st.BatchPlan(insts, prec, ws_budget=int(args.ws_gb * 2 ** 30))
    plan_s = time.perf_counter() - t0
    info = plan.info()
    ws = torch.empty(max(plan.workspace_size(), 1), dtype=torch.uint8, device="cuda")
    F = info["useful_flops"]
    t0 = time.perf_counter()
    plan.run(ws)                       # captures the graph
    torch.cuda.synchronize()
    capture_s = time.perf_counter() - t0
    steps = max(3, min(args.steps, 20))
    tot_tc = tot_unfused = None
    if not args.no_extras and not short:
        # the tcgen05 small-tile kernel for the same plan (for comparison)
        st.sttsm_set_small_kernel(st.SMALL_TCGEN05)
        plan_tc = st.BatchPlan(insts, prec, ws_budget=int(args.ws_gb * 2 ** 30))
        tot_tc, _ = time_steps(torch, lambda: plan_tc.run(ws), 3, 2)
        plan_tc.destroy()
        st.sttsm_set_small_kernel(st.SMALL_F32)
        # the last two levels fused in the batch (for comparison)
        st.sttsm_set_fused_tail(st.FUSED_TAIL_ALL)
        plan_uf = st.BatchPlan(insts, prec, ws_budget=int(args.ws_gb * 2 ** 30))
        tot_unfused, _ = time_steps(torch, lambda: plan_uf.run(ws), 3, 2)
        plan_uf.destroy()
        st.sttsm_set_fused_tail(args.fused_tail)
        st.sttsm_set_inblock_symmetry(args.inblock_sym)
    clocks = ClockSampler()
    clocks.start()
    total_ms, per = time_steps(torch, lambda: plan.run(ws), steps, max(3, args.warmup))
    clk = clocks.stop()
    ms = total_ms / steps
    value = F / (ms * 1e-3) / 1e12
    if args.no_extras:
        print(json.dumps({"metric": "sttsm batch TFLOP/s", "value": value, "ms_per_step": ms, "instances": len(shapes),
                          "useful_flops_per_step": F}), flush=True)
        plan.destroy()
        return 0
    # accuracy on a sample of instances against the oracle
    import oracle
    rng = np.random.default_rng(0)
    errs, errs_el = [], []
    small = [i for i, (m, n, p) in enumerate(shapes) if n ** m <= 2e7]
    for i in rng.choice(small, size=min(16, len(small)), replace=False):
        A_, dX_, C_, m, n, p, b = insts[i]
        X32 = xs[i].astype(np.float32).astype(np.float64)
        Ad = synth.sym_uniform_dense(m, n, 1000 + int(i))
        ref = oracle.bcss_pack(oracle.sttsm_chain(Ad, X32, m), m, p, b)
        got = C_.double().cpu().numpy()
        errs.append(float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
        errs_el.append(float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))))
    tot64 = None
    if not short:
        # the per-instance loop of the plain FP64 path
        scratch64 = torch.empty(maxdense, dtype=torch.float64, device="cuda")
        f64 = []
        for i, (A_, dX_, C_, m, n, p, b) in enumerate(insts):
            d = scratch64[: n ** m]
            synth.dev_sym_uniform_dense(d.data_ptr(), m, n, 1000 + i, "f64", stream)
            A64 = torch.empty(st.bcss_num_elems(m, n, b), dtype=torch.float64, device="cuda")
            st.bcss_pack(d, A64, m, n, b)
            X64 = torch.from_numpy(np.asfortranarray(xs[i]).reshape(-1, order="F").copy()).cuda()
            C64 = torch.empty(st.bcss_num_elems(m, p, b), dtype=torch.float64, device="cuda")
            f64.append((A64, X64, C64, m, n, p, b, st.workspace_tensor(m, n, p, b, st.STTSM_FP64)))
        del scratch64
        torch.cuda.synchronize()

        def loop64():
            for (A64, X64, C64, m, n, p, b, w64) in f64:
                st.sttsm_bcss(A64, X64, m, n, p, b, C64, st.STTSM_FP64, w64)

        tot64, _ = time_steps(torch, loop64, 1, 1)
        del f64
    # executed FMAs of the small-contraction kernel (tile rows x compile-time column
    # width x contraction padded to 4) and the algorithmic bytes (parents read, outputs
    # written, FP32) of every level of every instance, from the library's own plans
    exec_flops, alg_bytes = 0.0, 0.0
    for (_, _, _, m, n, p, b) in insts:
        Kc = ((-(-n // b)) * b + 3) // 4 * 4
        for d in range(m):
            tiles, _, li = st.sttsm_plan_level(m, n, p, b, prec, d)
            w = np.select([tiles[:, 5] <= 8, tiles[:, 5] <= 16, tiles[:, 5] <= 24, tiles[:, 5] <= 32, tiles[:, 5] <= 48],
                          [8, 16, 24, 32, 48], 64)
            exec_flops += 2.0 * 128 * Kc * float(w.sum())
            alg_bytes += 4.0 * (li["nodes_parent"] * li["P_parent"] + li["nodes_out"] * li["P_out"]) * li["bm"]
    pk, pk_src = peaks()
    fp32_peak = 152 * 128 * 2 * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    line = {"metric": "sttsm batch TFLOP/s (paper's BCSS flop count), BF16X6, one graph replay per step",
            "value": value, "unit": "TFLOP/s", "n_gpus": 1, "steps": steps, "warmup": max(3, args.warmup),
            "ms_per_step": ms, "p99_ms_per_step": float(np.percentile(per, 99)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x6", "data": "synthetic",
            "config": {"workload": "batch of %d sttsm instances: m in {3,4,5} (.5/.3/.2), n U{8..64}, p U{8..n}, "
                                   "b autotuned from {4,8,16}" % len(shapes),
                       "b_counts": {str(k): v for k, v in sorted(bcount.items())}, "useful_flops_per_step": F,
                       "waves": info["waves"], "workspace_gb": plan.workspace_size() / 2 ** 30,
                       "plan_seconds": plan_s, "graph_capture_seconds": capture_s},
            "fp64_per_instance_loop": {"value": F / (tot64 * 1e-3) / 1e12, "unit": "TFLOP/s", "ms": tot64,
                                       "speedup_of_batch": tot64 / ms} if tot64 else None,
            "small_kernel": "fp32 cuda-core (n̄b <= 64 contractions)",
            "median_ms_per_step": float(np.median(per)),
            "roofline": {"bound": "alu", "achieved": exec_flops / (ms * 1e-3) / 1e12, "peak": fp32_peak,
                         "unit": "TFLOP/s", "frac": exec_flops / (ms * 1e-3) / 1e12 / fp32_peak, "traffic": None,
                         "kernel": "level_small_f32_kernel (all levels of all instances)",
                         "achieved_counts": "executed FP32 FMAs x 2 (tile rows x compile-time column width x "
                                            "contraction padded to 4) per step / step time",
                         "peak_source": "152 SMs x 128 FP32 lanes x 2 x sm_max_mhz of %s MEASURED_PEAKS" % pk_src,
                         "useful_over_executed": F / exec_flops if exec_flops else None},
            "hbm": {"algorithmic_bytes_per_step": alg_bytes, "achieved_gbs": alg_bytes / (ms * 1e-3) / 1e9,
                    "peak_gbs": float(pk.get("hbm_gbs", 6800.0)),
                    "counts": "FP32 parents read + outputs written, every level of every instance"},
            "tcgen05_small_tile_kernel": {"value": F / (tot_tc / 3 * 1e-3) / 1e12, "unit": "TFLOP/s",
                                          "ms_per_step": tot_tc / 3} if tot_tc else None,
            "last_two_levels_fused": {"value": F / (tot_unfused / 3 * 1e-3) / 1e12, "unit": "TFLOP/s",
                                      "ms_per_step": tot_unfused / 3} if tot_unfused else None,
            "rel_err": {"instances_checked": len(errs), "max": max(errs), "median": float(np.median(errs)),
                        "max_elementwise": max(errs_el), "tolerance": 1e-6},
            "clocks": clk}
    plan.destroy()
    if emit:
        print(json.dumps(line), flush=True)
        return 0
    return line


SERVE_B = {3: (16, 32, 64), 4: (8, 16, 32), 5: (4, 8, 16), 6: (4, 8)}


def run_serve(args, emit=True, seconds=None, serve_prec=None):
    """Serving workload: Poisson arrivals (rate, seconds), uniform over the classes
    m=3 (n,p in [64,512]), m=4 ([32,160]), m=5 ([16,64]), m=6 ([8,32]); BF16X6; the
    server admits by HBM budget and batches continuously.  Inputs come from a pool of
    pre-generated instances per class (shapes drawn from the class ranges); each
    request uses pool entry (class, index mod pool size) with its own output buffer."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1301_7744_gb300 as st
    st.sttsm_set_fused_tail(args.fused_tail)
    st.sttsm_set_inblock_symmetry(args.inblock_sym)
    import synth
    prec = prec_code(st, serve_prec or "bf16x6")
    seconds = float(seconds or args.serve_seconds)
    reqs = synth.serve_requests(4, args.serve_rate, seconds)
    pool_n, cbuf = 32, 8
    rng = np.random.default_rng(11)
    stream = torch.cuda.current_stream().cuda_stream
    pool = {}
    for m, lo, hi in synth.SERVE_CLASSES:
        entries = []
        for e in range(pool_n):
            n, p = int(rng.integers(lo, hi + 1)), int(rng.integers(lo, hi + 1))
            b = st.sttsm_autotune_b(m, n, p, prec, SERVE_B[m])
            d = torch.empty(n ** m, dtype=torch.float32, device="cuda")
            synth.dev_sym_uniform_dense(d.data_ptr(), m, n, 7000 + 100 * m + e, "f32", stream)
            A = torch.empty(st.bcss_num_elems(m, n, b), dtype=torch.float32, device="cuda")
            st.bcss_pack(d, A, m, n, b)
            del d
            X = torch.from_numpy(xcol32(synth.x_gaussian(8000 + 100 * m + e, p, n))).cuda()
            Cs = [torch.empty(st.bcss_num_elems(m, p, b), dtype=torch.float32, device="cuda") for _ in range(cbuf)]
            entries.append(dict(A=A, X=X, C=Cs, m=m, n=n, p=p, b=b, F=st.sttsm_flops(m, n, p, b)))
        pool[m] = entries
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    srv = st.Server(int(args.serve_budget_gb * 2 ** 30), prec)
    # warm-up: one request per pool entry (plans, G tables, TMEM/attribute set-up)
    warm = []
    for m in pool:
        for e in pool[m]:
            warm.append(srv.submit(e["A"], e["X"], e["C"][0], e["m"], e["n"], e["p"], e["b"]))
    while not all(srv.poll(t)[0] for t in warm):
        time.sleep(0.001)
    count = {m: 0 for m in pool}
    used = set()
    tickets, flops = [], 0.0
    busy = 0
    clocks = ClockSampler()
    clocks.start()
    t0 = time.perf_counter()
    max_queue, max_active, max_arena = 0, 0, 0
    for i, (ta, m, _n, _p) in enumerate(reqs):
        while True:
            dt = t0 + ta - time.perf_counter()
            if dt <= 0:
                break
            if dt > 2e-4:
                time.sleep(dt - 1e-4)
        e = pool[m][count[m] % pool_n]
        c = e["C"][(count[m] // pool_n) % cbuf]
        used.add((m, count[m] % pool_n, (count[m] // pool_n) % cbuf))
        count[m] += 1
        while True:
            try:
                tickets.append(srv.submit(e["A"], e["X"], c, e["m"], e["n"], e["p"], e["b"]))
                break
            except st.SttsmError as err:
                if err.code != st.STTSM_ERR_BUSY:
                    raise
                busy += 1
                time.sleep(1e-4)
        flops += e["F"]
        if i % 256 == 0:
            sts = srv.stats()
            max_queue = max(max_queue, sts["queued"])
            max_active = max(max_active, sts["active"])
            max_arena = max(max_arena, sts["arena_bytes"])
    t_sub = time.perf_counter() - t0
    lat = []
    pending = list(tickets)
    while pending:
        nxt = []
        for t in pending:
            done, ms = srv.poll(t)
            if done:
                lat.append(ms)
            else:
                nxt.append(t)
        pending = nxt
        if pending:
            time.sleep(0.001)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    srv.destroy()
    lat = np.array(lat)
    # accuracy: per class the two pool entries with the smallest dense sizes, every C
    # buffer a request wrote, all stored entries against the oracle's dense chain
    import oracle
    oracle.build()
    errs = []
    for m in pool:
        small = sorted(range(pool_n), key=lambda k: max(pool[m][k]["n"], pool[m][k]["p"]))[:2]
        for k in small:
            E = pool[m][k]
            n, p, b = E["n"], E["p"], E["b"]
            Ad = synth.sym_uniform_dense(m, n, 7000 + 100 * m + k)
            X32 = synth.x_gaussian(8000 + 100 * m + k, p, n).astype(np.float32).astype(np.float64)
            ref = oracle.bcss_pack(oracle.sttsm_chain(Ad, X32, m), m, p, b)
            for j in sorted({0} | {u[2] for u in used if u[0] == m and u[1] == k}):
                got = E["C"][j].double().cpu().numpy()
                errs.append((float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                             float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))))
    line = {"metric": "sttsm serving latency p50/p99 (ms) and throughput, Poisson %.0f req/s for %.0f s"
                      % (args.serve_rate, seconds),
            "value": float(np.percentile(lat, 99)), "unit": "ms (p99 latency)", "higher_is_better": False,
            "n_gpus": 1, "dtype": st.PREC_NAMES[prec], "data": "synthetic",
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "p999_ms": float(np.percentile(lat, 99.9)), "mean_ms": float(lat.mean()),
            "requests": len(lat), "throughput_req_s": len(lat) / wall, "useful_tflops": flops / wall / 1e12,
            "submit_seconds": t_sub, "wall_seconds": wall, "busy_retries": busy,
            "max_queued": max_queue, "max_active": max_active, "max_arena_gb": max_arena / 2 ** 30,
            "rel_err": {"outputs_checked": len(errs), "max_fro": max(e[0] for e in errs),
                        "max_elementwise": max(e[1] for e in errs), "tolerance": 1e-6,
                        "what": "full C of the two smallest pool entries per class vs the FP64 oracle's dense chain; "
                                "elementwise = max |C - C_oracle| / max |C_oracle|"},
            "config": {"workload": "Poisson stream, classes m=3 n,p in [64,512]; m=4 [32,160]; m=5 [16,64]; "
                                   "m=6 [8,32]; b autotuned per pool entry",
                       "hbm_budget_gb": args.serve_budget_gb, "pool_per_class": pool_n,
                       "b_candidates": {str(k): v for k, v in SERVE_B.items()}},
            "clocks": clk}
    if emit:
        print(json.dumps(line), flush=True)
        return 0
    return line


SYM_SHAPES = [(5, 64, 64, 16), (5, 64, 64, 8), (5, 64, 64, 4), (4, 64, 64, 16), (4, 64, 64, 8), (3, 64, 64, 32),
              (3, 64, 64, 16), (5, 32, 32, 16), (4, 48, 48, 16)]


def run_symmetry(args):
    """Symmetry inside diagonal blocks (sttsm_set_inblock_symmetry) on single short-
    contraction instances: per shape the time of one sttsm_bcss call (BF16X6) with the
    mode off and on (CUDA events, 30 calls, best of two alternating rounds), the Tbl. 4
    flops, the flops the mode's tiles issue (canonical rows x all columns x 2 n̄ b) and the
    minimum of Sec. 6 (unique entries only, 2 n sum_d C(p+d, d+1) C(n+m-d-2, m-d-1)),
    and the relative error against the oracle for the smallest shape with the mode on."""
    import math
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1301_7744_gb300 as st
    import synth
    import oracle
    prec = st.STTSM_BF16X6
    out = {}
    for (m, n, p, b) in SYM_SHAPES:
        X = synth.x_gaussian(SEED_X, p, n)
        d = torch.empty(n ** m, dtype=torch.float32, device="cuda")
        synth.dev_sym_uniform_dense(d.data_ptr(), m, n, SEED_A, "f32", torch.cuda.current_stream().cuda_stream)
        Ab = torch.empty(st.bcss_num_elems(m, n, b), dtype=torch.float32, device="cuda")
        st.bcss_pack(d, Ab, m, n, b)
        del d
        dX = torch.from_numpy(xcol32(X)).cuda()
        C = torch.empty(st.bcss_num_elems(m, p, b), dtype=torch.float32, device="cuda")
        ws = st.workspace_tensor(m, n, p, b, prec)
        best = {0: float("inf"), 1: float("inf")}
        for sym in (0, 1, 0, 1):
            st.sttsm_set_inblock_symmetry(sym)
            tot, _ = time_steps(torch, lambda: st.sttsm_bcss(Ab, dX, m, n, p, b, C, prec, ws), 30, 5,
                                per_step_events=False)
            best[sym] = min(best[sym], tot / 30)
        st.sttsm_set_inblock_symmetry(1)
        nbar = -(-n // b)
        issued = 0
        for lv in range(m):
            tiles, _, info = st.sttsm_plan_level(m, n, p, b, prec, lv)
            rows = np.minimum(info["BM"], tiles[:, 7].astype(np.int64) - tiles[:, 3])
            issued += int(2 * (rows * tiles[:, 5].astype(np.int64)).sum()) * nbar * b
        st.sttsm_set_inblock_symmetry(0)
        minimum = 2 * n * sum(math.comb(p + dd, dd + 1) * math.comb(n + m - dd - 2, m - dd - 1) for dd in range(m))
        out[f"m{m}_n{n}_p{p}_b{b}"] = {"ms_off": best[0], "ms_on": best[1], "speedup": best[0] / best[1],
                                       "tbl4_gflop": st.sttsm_flops(m, n, p, b) / 1e9,
                                       "issued_gflop_on": issued / 1e9, "minimum_gflop": minimum / 1e9}
    # accuracy with the mode on, smallest shape
    m, n, p, b = min(SYM_SHAPES, key=lambda s: s[1] ** s[0])
    A = synth.sym_uniform_dense(m, n, SEED_A)
    X32 = synth.x_gaussian(SEED_X, p, n).astype(np.float32).astype(np.float64)
    d = torch.from_numpy(A.astype(np.float32)).cuda()
    Ab = torch.empty(st.bcss_num_elems(m, n, b), dtype=torch.float32, device="cuda")
    st.bcss_pack(d, Ab, m, n, b)
    C = torch.empty(st.bcss_num_elems(m, p, b), dtype=torch.float32, device="cuda")
    st.sttsm_set_inblock_symmetry(1)
    st.sttsm_bcss(Ab, torch.from_numpy(xcol32(X32)).cuda(), m, n, p, b, C, prec, st.workspace_tensor(m, n, p, b, prec))
    torch.cuda.synchronize()
    st.sttsm_set_inblock_symmetry(0)
    ref = oracle.bcss_pack(oracle.sttsm_chain(A, X32, m), m, p, b)
    err = float(np.linalg.norm(C.double().cpu().numpy() - ref) / np.linalg.norm(ref))
    print(json.dumps({"metric": "sttsm single-call ms, in-block symmetry off / on", "unit": "ms",
                      "higher_is_better": False, "dtype": "f32 (BF16X6 products)", "data": "synthetic",
                      "results": out, "rel_err_on": {"shape": [m, n, p, b], "rel_fro": err}}), flush=True)
    return 0


def run_pack(args):
    """bcss_pack and bcss_unpack of the m = 3 FP32 symmetric tensor of dimension --pack-n
    (block size --b, default 64): GB/s of algorithmic bytes and fraction of the measured
    HBM copy peak, and the bit-exact round trip."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1301_7744_gb300 as st
    pk, pk_src = peaks()
    b = 64 if args.b == "auto" else int(args.b)
    res = pack_bandwidth(st, torch, b, pk, pk_src, reps=5, n=args.pack_n)
    print(json.dumps({"metric": "bcss pack / unpack GB/s", "unit": "GB/s", "higher_is_better": True,
                      "config": {"workload": "pack_unpack", "m": M, "n": args.pack_n, "b": b, "dtype": "f32"},
                      "results": res}), flush=True)
    return 0


def main():
    args = parse_args()
    if args.workload == "pack":
        return run_pack(args)
    if args.workload == "symmetry":
        return run_symmetry(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "m4":
        return run_m4(args)
    if args.workload == "abo":
        return run_abo(args)
    import torch
    import torch.distributed as dist

    import __graft_entry__
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # each rank's GPU is current before any NCCL call (the barrier below runs on it)
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.init_process_group("nccl")
        dist.barrier()
        if rank != 0:
            __graft_entry__.build()
    import paper_1301_7744_gb300 as st
    st.sttsm_set_fused_tail(args.fused_tail)
    st.sttsm_set_inblock_symmetry(args.inblock_sym)

    prec = prec_code(st, args.prec)
    import synth
    Xh = synth.x_gaussian(SEED_X, P, N)
    X32 = Xh.astype(np.float32).astype(np.float64)
    dX = torch.from_numpy(xcol32(Xh)).cuda()

    # ---- block size: the library's measured autotuner over {32, 48, 64}
    sweep = {}
    b_fastest = None
    if args.b == "auto":
        # the library picks the fastest b; the metric is TFLOP/s of the b-dependent Tbl. 4
        # count, so the line reports the b with the highest rate among the measured ones
        b_fastest, times = st.sttsm_autotune_b_measured(M, N, P, prec, (32, 48, 64), reps=3)
        sweep = {c: st.sttsm_flops(M, N, P, c) / (t * 1e-3) / 1e12 for c, t in times.items() if t}
        b = max(sweep, key=sweep.get)
        torch.cuda.empty_cache()
    else:
        b = int(args.b)
    if world > 1:
        # every replica runs rank 0's block size, so all ranks do the same work
        tb = torch.tensor([b], device="cuda", dtype=torch.int64)
        dist.broadcast(tb, 0)
        b = int(tb.item())
    F = st.sttsm_flops(M, N, P, b)

    A = make_device_inputs(st, torch, b, torch.float32)
    C = torch.empty(st.bcss_num_elems(M, P, b), dtype=torch.float32, device="cuda")
    ws = st.workspace_tensor(M, N, P, b, prec)

    def step():
        st.sttsm_bcss(A, dX, M, N, P, b, C, prec, ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler()
    clocks.start()
    st.sttsm_profile_enable(True)
    total_ms, per = time_steps(torch, step, args.steps, 0)
    st.sttsm_profile_enable(False)
    clk = clocks.stop()
    if world > 1:
        total_ms = max_over_ranks(total_ms, "cuda")
        dist.barrier()
    ms = total_ms / args.steps
    value = job_rate(F, world, total_ms, args.steps)

    # ---- dominant kernel roofline from the library's per-launch events
    recs = st.sttsm_profile_read()
    tc = [r for r in recs if r["kind"] in ("tc", "tma")]
    kinds = sorted({r["kind"] for r in tc})
    kern_ms = sum(r["ms"] for r in tc)
    kern_flops = sum(r["useful_flops"] for r in tc)
    nprod = 6 if args.prec.startswith("bf16x6") else 3
    pk, pk_src = peaks()
    mma_tflops = kern_flops * nprod / (kern_ms * 1e-3) / 1e12 if kern_ms > 0 else 0.0
    peak, peak_source = tensor_peak(pk, pk_src, clk, total_ms)
    per_level = {}
    for r in tc:
        d = per_level.setdefault(r["level"], {"ms": 0.0, "flops": 0.0, "n": 0})
        d["ms"] += r["ms"]
        d["flops"] += r["useful_flops"]
        d["n"] += 1
    levels = {str(k): {"ms_per_launch": v["ms"] / v["n"],
                       "useful_tflops": v["flops"] / (v["ms"] * 1e-3) / 1e12,
                       "mma_frac_of_peak": v["flops"] * nprod / (v["ms"] * 1e-3) / 1e12 / peak}
              for k, v in sorted(per_level.items())}
    traffic = profiled_traffic(b, args.prec, kinds)
    # algorithmic bytes per level launch (mean): parent BF16 pieces read + output written
    # (pieces, or FP32 C at the last level), from the level sizes
    alg = 0.0
    npc = 3 if args.prec.startswith("bf16x6") else 2
    for d in range(M):
        _, _, info = st.sttsm_plan_level(M, N, P, b, prec, d)
        par = info["nodes_parent"] * info["P_parent"] * info["bm"] * npc * 2
        out = info["nodes_out"] * info["P_out"] * info["bm"] * (4 if d == M - 1 else npc * 2)
        alg += par + out
    alg_bytes = alg / M
    roofline = {"bound": "tensor", "achieved": mma_tflops, "peak": peak, "unit": "TFLOP/s",
                "frac": mma_tflops / peak, "traffic": traffic,
                "traffic_per": "launch (DRAM read + write, mean of the m level launches of a step; ncu)",
                "algorithmic_bytes_per_launch": alg_bytes,
                "kernel": {"tma": "level_tma_kernel", "tc": "level_tc_kernel"}[kinds[0]] + " (all m levels)" if kinds else None,
                "achieved_counts": "useful flops x %d piece products per launch / CUDA-event duration" % nprod,
                "peak_source": peak_source,
                "frac_of_sustained_peak": mma_tflops / float(pk.get("bf16_tflops_sustained", 1700.0)),
                "useful_tflops": kern_flops / (kern_ms * 1e-3) / 1e12 if kern_ms > 0 else 0.0,
                "kernel_share_of_step": kern_ms / total_ms if total_ms > 0 else None,
                "levels": levels}

    e2e = fp64 = rel_err = cpu_base = packbw = r64 = C_r64 = None
    if not args.no_extras and args.prec == "bf16x6":
        # ---- the same step with the final C-block reduction in FP64 (BF16X6_R64)
        C_r64 = torch.empty_like(C)
        pr64 = st.STTSM_BF16X6_R64
        tot_r, _ = time_steps(torch, lambda: st.sttsm_bcss(A, dX, M, N, P, b, C_r64, pr64, ws), 10, 3)
        r64 = {"value": F / (tot_r / 10 * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": tot_r / 10,
               "cost_vs_bf16x6": (tot_r / 10) / ms,
               "what": "BF16X6 products, last level's FP32 group sums added in FP64 (C-writing tiles <= 128 columns)"}
    C64 = None
    if not args.no_extras:
        # ---- BCSS pack / unpack of the same tensor (HBM-bound copies)
        packbw = pack_bandwidth(st, torch, b, pk, pk_src)
        # ---- end to end through the host-buffer entry point
        e2e = end_to_end(st, torch, A, C, Xh, ws, b, F, prec, world, max(20, args.steps))
        # ---- plain FP64 GPU path on the same workload (rank 0)
        if rank == 0:
            fp64, C64 = fp64_path(st, torch, Xh, b, F, ms)
        # ---- accuracy against the oracle and the CPU baseline (rank 0; baseline at N = 1)
        if rank == 0 and not args.no_check:
            rel_err, cpu_base = check_and_baseline(args, C, C64, Xh, X32, b, F, world, C_r64)

    # ---- the other configurations, short forms (N = 1 only): m=4 n=128 p=64, the
    # 4096-instance batch, the serving stream
    configs = None
    a_mb = A.numel() * 4 / 1e6
    if world == 1 and not args.no_extras and not args.no_configs:
        del A, C, ws, C64, C_r64
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        configs = {}
        for name, fn in (("m4", lambda: run_m4(args, emit=False, short=True)),
                         ("batch", lambda: run_batch(args, emit=False, short=True)),
                         ("serve", lambda: run_serve(args, emit=False, seconds=args.configs_serve_seconds)),
                         ("serve_r64", lambda: run_serve(args, emit=False, seconds=args.configs_serve_seconds,
                                                         serve_prec="bf16x6_r64"))):
            t0 = time.perf_counter()
            configs[name] = fn()
            configs[name]["wall_seconds_of_leg"] = time.perf_counter() - t0
            torch.cuda.synchronize()
            torch.cuda.empty_cache()

    tts = None
    if sweep:
        ms_fast = times[b_fastest]
        tts = {"b": b_fastest, "ms_per_step": ms_fast, "tflops": st.sttsm_flops(M, N, P, b_fastest) / (ms_fast * 1e-3) / 1e12,
               "headline_b_ms_per_step": times.get(b), "source": "median of the autotuner's timed runs per b"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "p99_ms_per_step": float(np.percentile(per, 99)),
                "median_ms_per_step": float(np.median(per)),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
                "data": "synthetic",
                "config": {"workload": "sttsm m=3 n=p=768 b=%d %s" % (b, args.prec.upper()), "m": M, "n": N, "p": P,
                           "b": b, "precision": args.prec, "b_sweep_tflops": {str(k): v for k, v in sweep.items()},
                           "b_fastest_by_time": b_fastest,
                           "useful_flops_per_step": F, "l2": "inputs larger than L2 (A in BCSS FP32: %.0f MB)"
                           % a_mb, "parallelism": "replicas" if world > 1 else "single"},
                "roofline": roofline, "cpu_baseline": cpu_base, "e2e": e2e, "fp64_path": fp64, "rel_err": rel_err,
                "pack_unpack": packbw,
                "time_to_solution": tts, "configs": configs, "final_reduction_fp64": r64,
                "gpu_launches": args.steps * (M + (2 if "tma" in kinds else 1)), "clocks": clk}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
