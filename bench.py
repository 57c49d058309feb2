#!/usr/bin/env python
"""Benchmark: QTT solves/sec at relative residual 1e-8 on L = 12 plates.

One step = the whole hot path for one synthetic problem of the square-plate
family (left edge clamped, constant traction of amplitude amp at angle theta
on the top edge, n = 2^12 nodes per side, 33.5 M DOFs): assemble K and f on
the device from the host problem description (Algorithm 1), solve K u = f
with AMEn, and accept the solve when its FP64 relative residual
||f - K u|| / ||f|| (exact QTT matvec and sum in FP64, normed in full
format) is <= 1e-8.  value = accepted solves per second of CUDA-event time
over the timed steps (max over ranks).

Every timed step also gives the end-to-end figure: host wall time from the
host problem description to the solution cores and the solve record read
back into host memory (the e2e object), measured in the same loop.

Forms:
  --form fast   (default) mixed precision: FP64 interfaces and residuals,
                FP32 Krylov operators (tensor cores where the autotuner
                finds them faster), FP64 outer refinement; with
                --warm-start also the learned warm start (MLP inference;
                the network is trained before the timed region), with
                --superposition-start the start formed from stored method
                solutions interpolated in nu (solved before the timed
                region; the interpolation runs inside every timed step)
  --form plain  FP64 AMEn, cold start, one solve at a time
The fast-form line also carries a `plain` object: the plain form timed on
the first `--plain-solves` problems of the same workload after the timed
steps (the comparison the metric names).

--impl reference   the oracle (NumPy/SciPy FP64 on the host cores): each
                   step one complete oracle solve of a plate problem of the
                   same family at level --ref-L (an L = 12 oracle solve takes
                   minutes; the level is named in the line)

Multi-GPU: problems are independent; rank r solves every world-th problem
(weak scaling, no data-path collective; a barrier and a max reduction of the
timings only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QTT solves/sec at rel. residual 1e-8 (L=12); fast form vs plain FP64 GPU"
ACCEPT = 1e-8
MAX_SWEEPS = 24
KICK_RANK = 8
TENSOR_CORES = 0
LOCAL_DIRECT_MAX = 0
_T0 = time.perf_counter()
CLASSES = {0: "gemm_f64", 1: "gemm_f32", 2: "core_product", 3: "qr_panel", 4: "jacobi_svd", 5: "lu_panel",
           6: "permute", 7: "to_full", 8: "pcg_f32", 9: "jacobi_f32", 10: "tc_gemm_tf32x3"}


def log(msg: str):
    print(f"[bench {time.perf_counter() - _T0:8.1f}s] {msg}", file=sys.stderr, flush=True)


NU_GRID = (0.2, 0.283, 0.367, 0.45)


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="fast", choices=["fast", "plain"])
    ap.add_argument("--batch", type=int, default=1, help="problems per step per rank")
    ap.add_argument("--workers", type=int, default=1, help="concurrent solves when --batch > 1")
    ap.add_argument("--max-sweeps", type=int, default=24)
    ap.add_argument("--kick-rank", type=int, default=8, help="residual-proxy rank of the AMEn enrichment")
    ap.add_argument("--local-direct-max", type=int, default=0,
                    help="local systems up to this size use dense LU (0: the library default)")
    ap.add_argument("--tensor-cores", type=int, default=0,
                    help="FP32 local operator: 0 autotuned tcgen05/SIMT, 1 always tensor cores, -1 always SIMT")
    ap.add_argument("--L", type=int, default=12)
    ap.add_argument("--tol", type=float, default=ACCEPT)
    ap.add_argument("--plain-solves", type=int, default=1,
                    help="fast form: plain FP64 solves timed after the timed steps (0: none)")
    ap.add_argument("--plain-budget", type=float, default=1500.0,
                    help="start no plain solve once the run has taken this many seconds")
    ap.add_argument("--train-steps", type=int, default=400)
    ap.add_argument("--warm-start", action="store_true",
                    help="fast form with the learned warm start (8 basis solves + MLP training before timing)")
    ap.add_argument("--superposition-start", action="store_true",
                    help="fast form warm-started by superposing stored method solutions interpolated in nu "
                         "(basis solves before timing)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-L", type=int, default=6, help="level of the complete oracle solves (CPU legs)")
    ap.add_argument("--cpu-solves", type=int, default=3, help="timed oracle solves of the cpu_baseline leg")
    ap.add_argument("--no-profile", action="store_true",
                    help="do not bracket the timed launches with the per-class CUDA-event profiler")
    return ap.parse_args(argv)


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
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
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------
def workload(L: int, count: int, rank: int, world: int, seed: int = 2):
    """Held-out parameter rows (seed 2) of the plate family; rank r takes every
    world-th row.  Returns (params (n, 4), problems)."""
    import numpy as np
    import workloads as W
    P = W.plate_params(seed, count * world)[rank::world]
    probs = [W.plate_top_traction(L, float(E), float(nu), float(a), float(t)) for E, nu, a, t in P]
    return np.asarray(P), probs


def workload_name(L: int) -> str:
    return (f"plate L={L} ({2 * 4 ** L} DOFs), clamped left, constant top-edge traction; "
            f"(E, nu, amp, angle) from the held-out seed-2 set")


def combine_ranks(ms: float, accepted: int, total: int, dist=None, device: str = "cpu"):
    """Whole-job numbers over all ranks: the slowest rank's timed milliseconds
    and the sums of accepted and attempted solves; value = accepted solves
    per second of that time.  Returns (ms, accepted, total, value)."""
    import torch
    t_ms = torch.tensor([ms], dtype=torch.float64, device=device)
    t_n = torch.tensor([float(accepted), float(total)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t_ms, op=dist.ReduceOp.MAX)
        dist.all_reduce(t_n, op=dist.ReduceOp.SUM)
    ms_all, acc_all, tot_all = float(t_ms[0]), float(t_n[0]), float(t_n[1])
    value = acc_all / (ms_all / 1e3) if ms_all > 0 else 0.0
    return ms_all, acc_all, tot_all, value


def solve_kw(form: str, tol: float):
    import paper_2501_07778_gb300 as q
    prec = q.QTT_F64 if form == "plain" else q.QTT_MIXED
    return dict(tol=tol, precision=prec, kick_rank=KICK_RANK, max_sweeps=MAX_SWEEPS, tensor_cores=TENSOR_CORES,
                local_direct_max=LOCAL_DIRECT_MAX)


def problem_bytes(prob) -> int:
    """Bytes of the host problem description the library reads (the C
    struct and its arrays)."""
    q = prob.q
    return 2 * 4 + 2 * 8 + 2 * 8 + 2 * q * 4 + 4 * q * 4 + len(prob.body) * (3 * 4 + 8) + \
        len(prob.traction) * (2 * 4 + 2 * 8)


def run_step(form, params, probs, net, tol, workers):
    """The hot path over one batch: assembly, (warm start), solve with the
    FP64 residual check.  Returns (solutions, infos)."""
    import paper_2501_07778_gb300 as q
    KF = [q.qtt_assemble_stiffness(p) for p in probs]
    x0s = net.predict(params) if (net is not None and form == "fast") else [None] * len(probs)
    if len(probs) == 1:
        u, i = q.qtt_solve(KF[0][0], KF[0][1], x0=x0s[0], check=False, **solve_kw(form, tol))
        return [u], [i]
    if form == "plain":
        out = [q.qtt_solve(K, f, check=False, **solve_kw(form, tol)) for K, f in KF]
        return [u for u, _ in out], [i for _, i in out]
    return q.qtt_solve_batched([K for K, _ in KF], [f for _, f in KF], x0s, nworkers=workers,
                               **solve_kw(form, tol))


def train_warm_start(L: int, tol: float, steps: int):
    """Method solves at the nu grid, then the MLP on 2000 superposition
    targets.  Returns (net, info)."""
    import workloads as W
    from paper_2501_07778_gb300 import QTT_F32, QTT_MIXED
    from paper_2501_07778_gb300 import warmstart as ws
    t0 = time.perf_counter()
    log(f"warm start: {2 * len(NU_GRID)} basis solves at L={L}")
    basis64 = ws.basis_solutions(L, NU_GRID, tol=tol, precision=QTT_MIXED, kick_rank=KICK_RANK,
                                 max_sweeps=MAX_SWEEPS)
    basis = [b.copy(prec=QTT_F32) for b in basis64]
    t1 = time.perf_counter()
    log(f"warm start: basis solves took {t1 - t0:.1f} s; training {steps} steps")
    modes = W.qtt_modes(W.plate_top_traction(L, 1.0, 0.3, 1.0, 0.0))
    net = ws.WarmStartMLP(modes, r=16, H=256, seed=0)
    P, coef = ws.dataset(1, 2000, NU_GRID)
    losses = ws.train(net, basis, P, coef, steps=steps, batch=32, lr=3e-4)
    t2 = time.perf_counter()
    last = float(sum(losses[-10:]) / 10)
    used = last < 0.5
    return net if used else None, {"basis_solves": len(basis), "basis_s": round(t1 - t0, 2), "train_steps": steps,
                                   "train_s": round(t2 - t1, 2), "loss_first": round(float(losses[0]), 5),
                                   "loss_last": round(last, 5), "used": used}


# ----------------------------------------------------------------------------
# CPU: complete oracle solves
# ----------------------------------------------------------------------------
def oracle_solve(prob, tol: float):
    """One complete oracle solve (O-2 assembly of K and f in QTT + AMEn to
    tol, NumPy/SciPy FP64 on the host cores).  Returns (seconds, sweeps)."""
    import numpy as np
    import workloads as W
    from oracle import amen, assembly
    t0 = time.perf_counter()
    K, f = assembly.assemble(prob)
    modes = W.qtt_modes(prob)
    x0 = [np.ones((1, n, 1)) for n in modes]
    z0 = W.random_tt(1, modes, [1] + [8] * (len(modes) - 1) + [1])
    _, info = amen.amen_solve(K, f, x0, z0, tol, max_sweeps=40, local_direct_max=2048)
    return time.perf_counter() - t0, info.sweeps


def cpu_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return int(max((i.get("num_threads", 1) for i in info), default=os.cpu_count()))
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(L: int, tol: float, solves: int):
    """Median of `solves` complete oracle solves after one untimed warm-up
    solve, on held-out problems of the plate family at level L."""
    _, probs = workload(L, solves + 1, 0, 1)
    oracle_solve(probs[0], tol)
    times, sweeps = [], []
    for p in probs[1:]:
        t, s = oracle_solve(p, tol)
        times.append(t)
        sweeps.append(s)
    med = statistics.median(times)
    return {"value": 1.0 / med, "unit": "solves/s", "cores": cpu_threads(), "kind": "oracle",
            "sample": (f"{solves} complete oracle solves (QTT assembly + AMEn to {tol:g}) of L={L} plates of the same "
                       f"family, median {med:.2f} s after one warm-up solve (sweeps {sweeps}); an L=12 oracle solve "
                       f"takes minutes per problem, beyond the run's budget"),
            "L": L, "cpu": cpu_model()}


# ----------------------------------------------------------------------------
# reference arm: the oracle
# ----------------------------------------------------------------------------
def reference_main(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    _, probs = workload(args.ref_L, args.warmup + args.steps, 0, 1)
    times, sweeps = [], []
    for i, p in enumerate(probs):
        t, s = oracle_solve(p, args.tol)
        log(f"oracle solve {i}: {t:.2f} s, {s} sweeps")
        if i >= args.warmup:
            times.append(t)
            sweeps.append(s)
    total = sum(times)
    v = len(times) / total if total > 0 else 0.0
    desc = (f"each step one complete oracle solve (QTT assembly + AMEn to {args.tol:g}, NumPy/SciPy FP64) of an "
            f"L={args.ref_L} plate of the same family; {len(times)} solves in {total:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": len(times), "warmup": args.warmup, "ms_per_step": 1e3 * total / max(1, len(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.ref_L), "L": args.ref_L, "batch": 1,
                       "accept_rel_residual": args.tol,
                       "note": "oracle solves at L=12 take minutes each; the level is the largest whose "
                               "warm-up + timed solves fit a few minutes"},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": desc, "cpu": cpu_model()},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "solve_stats": {"sweeps": sweeps, "seconds": [round(t, 3) for t in times]}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def read_profile(lib):
    import ctypes as C
    out = {}
    for cid, nm in CLASSES.items():
        a, f_, b_, n_ = C.c_double(), C.c_double(), C.c_double(), C.c_longlong()
        lib.qtt_profile_read(cid, C.byref(a), C.byref(f_), C.byref(b_), C.byref(n_))
        out[nm] = [a.value, f_.value, b_.value, n_.value]
    return out


def measured_peaks(lib):
    """FP64 and FP32 FMA rates of this GPU measured by the library's own
    all-SM FMA-chain kernels (CUDA events), plus the measured HBM
    copy and BF16 GEMM rates."""
    import ctypes as C
    import torch
    peaks = {}
    try:
        peaks.update(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))))
    except Exception:
        pass
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for prec, key in ((0, "fp64_tflops"), (1, "fp32_tflops")):
        v = C.c_double()
        best = 0.0
        for _ in range(3):
            if lib.qtt_measure_fma_peak(prec, C.byref(v), s) == 0:
                best = max(best, v.value)
        peaks[key] = best
    return peaks


def roofline_of(prof, peaks, sms):
    dom = max(prof, key=lambda k: prof[k][0])
    ms, fl, by, n = prof[dom]
    sec = ms / 1e3
    if dom in ("gemm_f64", "qr_panel", "jacobi_svd", "lu_panel"):
        bound, unit, peak = "alu", "TFLOP/s", peaks.get("fp64_tflops")
        src = "FP64 FMA rate measured live by the library's all-SM FMA-chain kernel (qtt_measure_fma_peak)"
        achieved = fl / 1e12 / sec if sec > 0 else 0.0
    elif dom == "tc_gemm_tf32x3":
        bound, unit, peak = "tensor", "TFLOP/s", peaks.get("bf16_tflops", 1892.4) / 2.0 / 3.0
        src = ("3xTF32 on tcgen05: MEASURED_PEAKS bf16_tflops x 1/2 (TF32 vs BF16 dense rate) x 1/3 (three MMAs "
               "per product)")
        achieved = fl / 1e12 / sec if sec > 0 else 0.0
    elif dom in ("gemm_f32", "pcg_f32", "jacobi_f32"):
        bound, unit, peak = "alu", "TFLOP/s", peaks.get("fp32_tflops")
        src = "FP32 FMA rate measured live by the library's all-SM FMA-chain kernel (qtt_measure_fma_peak)"
        achieved = fl / 1e12 / sec if sec > 0 else 0.0
    else:
        bound, unit, peak = "hbm", "GB/s", peaks.get("hbm_gbs", 6800.0)
        src = "MEASURED_PEAKS.json hbm_gbs (driver-measured copy)"
        achieved = by / 1e9 / sec if sec > 0 else 0.0
    classes = {k: {"ms": round(v[0], 3), "gflop": round(v[1] / 1e9, 3), "gbytes": round(v[2] / 1e9, 3),
                   "launches": int(v[3])} for k, v in prof.items()}
    return {"bound": bound, "kernel": dom, "achieved": round(achieved, 4), "peak": round(peak, 3) if peak else None,
            "unit": unit, "frac": round(achieved / peak, 5) if peak else None, "traffic": None,
            "traffic_note": "null: the dominant kernels' operands are L2-resident and a solve's launches of them are "
                            "too many for an ncu capture; single-launch ncu captures in profiles/",
            "launches": int(n), "avg_launch_us": round(1e3 * ms / max(1, n), 2), "peak_source": src,
            "sms": sms, "classes": classes,
            "note": "per-class CUDA events bracket every launch of the timed steps on its own stream; "
                    "achieved = algorithmic work of those launches / their summed event time"}


def main(argv=None):
    args = parse(argv)
    if args.impl == "reference":
        return reference_main(args)
    import ctypes as C

    import numpy as np
    import torch

    import __graft_entry__
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    __graft_entry__.build()
    import paper_2501_07778_gb300 as q
    lib = q.lib()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    global MAX_SWEEPS, KICK_RANK, TENSOR_CORES, LOCAL_DIRECT_MAX
    MAX_SWEEPS = args.max_sweeps
    KICK_RANK = args.kick_rank
    TENSOR_CORES = args.tensor_cores
    LOCAL_DIRECT_MAX = args.local_direct_max
    batch = max(1, args.batch)
    nsteps = args.warmup + args.steps
    P, probs = workload(args.L, nsteps * batch, rank, world)
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    log(f"library ready; form {args.form}, L={args.L}, {batch} solve(s) per step, {nsteps} steps, {sms} SMs")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > 129 MB L2
    peaks = measured_peaks(lib)
    log(f"measured FMA peaks: FP64 {peaks.get('fp64_tflops', 0):.3f} TFLOP/s, "
        f"FP32 {peaks.get('fp32_tflops', 0):.2f} TFLOP/s")

    net, ws_info = None, None
    if args.form == "fast" and args.warm_start:
        net, ws_info = train_warm_start(args.L, args.tol, args.train_steps)
        log(f"warm start ready: {ws_info}")
    elif args.form == "fast" and args.superposition_start:
        from paper_2501_07778_gb300 import warmstart as ws
        t0 = time.perf_counter()
        nus = tuple(np.linspace(0.2, 0.45, 7))
        net = ws.SuperpositionStart(args.L, nus, order=3, tol=args.tol, precision=q.QTT_MIXED, kick_rank=KICK_RANK,
                                    max_sweeps=MAX_SWEEPS)
        ws_info = {"kind": "superposition of stored method solutions (2 unit tractions x 7 nu values), "
                           "Lagrange interpolation in nu over the 3 nearest", "basis_solves": 2 * len(nus),
                   "basis_s": round(time.perf_counter() - t0, 2), "used": True}
        log(f"superposition start ready: {ws_info}")

    def step_slice(st):
        return P[st * batch:(st + 1) * batch], probs[st * batch:(st + 1) * batch]

    for st in range(args.warmup):
        _, inf = run_step(args.form, *step_slice(st), net, args.tol, args.workers)
        log(f"warm-up step {st}: sweeps {[i['sweeps'] for i in inf]} res {[i['rel_residual'] for i in inf]}")
    barrier()

    sampler = ClockSampler(local)
    sampler.start()
    launches0 = lib.qtt_kernel_launches()
    accepted = total = 0
    ms = 0.0
    wall = 0.0
    h2d = d2h = 0
    infos = []
    prof = {k: [0.0, 0.0, 0.0, 0] for k in CLASSES.values()}
    read_profile(lib)                      # drop anything recorded before
    if not args.no_profile:
        lib.qtt_profile_enable(1)
    barrier()
    torch.cuda.nvtx.range_push("timed")
    timed_range = torch.cuda.nvtx.range_start("timed")
    for st in range(args.warmup, nsteps):
        flush.zero_()
        par, pr = step_slice(st)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0.record(stream)
        us, inf = run_step(args.form, par, pr, net, args.tol, args.workers)
        e1.record(stream)
        # end to end: the result (solution cores, host copies) read back
        for u in us:
            cores = u.cores()
            d2h += sum(c.nbytes for c in cores)
        e1.synchronize()
        wall += time.perf_counter() - t0
        h2d += sum(problem_bytes(p) for p in pr)
        step_ms = e0.elapsed_time(e1)
        ms += step_ms
        if not args.no_profile:
            for k, v in read_profile(lib).items():
                prof[k] = [a + b for a, b in zip(prof[k], v)]
        for i in inf:
            total += 1
            accepted += int(0 < i["rel_residual"] <= args.tol)
            infos.append(i)
        log(f"timed step {st - args.warmup}: {step_ms / 1e3:.2f} s, sweeps {[i['sweeps'] for i in inf]} "
            f"res {[i['rel_residual'] for i in inf]} checks {[i['checks'] for i in inf]} "
            f"check_ms {[round(i['check_ms']) for i in inf]} refine_ms {[round(i['refine_ms']) for i in inf]}")
    torch.cuda.nvtx.range_end(timed_range)
    torch.cuda.nvtx.range_pop()
    lib.qtt_profile_enable(0)
    barrier()
    launches = lib.qtt_kernel_launches() - launches0
    clocks = sampler.stop()
    ms_all, acc_all, tot_all, value = combine_ranks(ms, accepted, total, dist, device="cuda")
    wall_all, acc_e2e, _, e2e_value = combine_ranks(1e3 * wall, accepted, total, dist, device="cuda")
    log(f"timed: {ms_all:.1f} ms for {tot_all:.0f} solves ({acc_all:.0f} accepted); e2e wall {wall_all:.1f} ms")
    roofline = roofline_of(prof, peaks, sms) if not args.no_profile else None

    # ---- the plain FP64 form on the first problems of the timed set
    plain = None
    if args.form == "fast" and args.plain_solves > 0:
        pms, pacc, pinfo = 0.0, 0, []
        for j in range(args.plain_solves):
            if time.perf_counter() - _T0 > args.plain_budget:
                break
            par, pr = step_slice(args.warmup + j % max(1, args.steps))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            _, inf = run_step("plain", par[:1], pr[:1], None, args.tol, 1)
            e1.record(stream)
            e1.synchronize()
            pms += e0.elapsed_time(e1)
            pacc += int(0 < inf[0]["rel_residual"] <= args.tol)
            pinfo.append(inf[0])
            log(f"plain solve {j}: {e0.elapsed_time(e1) / 1e3:.2f} s, sweeps {inf[0]['sweeps']}, "
                f"refinements {inf[0]['refinements']}, res {inf[0]['rel_residual']:.3e}")
        if pinfo:
            pms_all, pacc_all, ptot_all, pvalue = combine_ranks(pms, pacc, len(pinfo), dist, device="cuda")
            plain = {"value": pvalue, "unit": "solves/s", "solves": int(ptot_all), "accepted": int(pacc_all),
                     "ms_per_solve": pms_all / max(1, len(pinfo)),
                     "form": "FP64 AMEn (FP64 local CG), cold start, one solve at a time, FP64 outer refinement",
                     "problems": "the first problem(s) of the timed set",
                     "rel_residual": [i["rel_residual"] for i in pinfo], "sweeps": [i["sweeps"] for i in pinfo],
                     "refinements": [i["refinements"] for i in pinfo],
                     "fast_over_plain": (value / pvalue) if pvalue > 0 else None}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(args.ref_L, args.tol, args.cpu_solves)
        log(f"cpu baseline: {cpu['value']:.4f} solves/s at L={args.ref_L}")

    e2e = {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d // max(1, args.steps),
           "d2h_bytes_per_step": d2h // max(1, args.steps),
           "what": "host wall time of each timed step: host problem description -> assembly, solve and FP64 "
                   "check through the C ABI -> solution cores copied to host memory"}
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.form == "fast" else "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args.L), "form": args.form, "L": args.L,
                       "batch_per_rank": batch, "workers": args.workers if batch > 1 else 1,
                       "learned_warm_start": bool(args.warm_start) and ws_info is not None and bool(ws_info.get("used")),
                       "superposition_start": bool(args.superposition_start),
                       "accept_rel_residual": args.tol, "kick_rank": args.kick_rank, "max_sweeps": args.max_sweeps,
                       "tensor_cores": {0: "autotuned", 1: "always"}.get(args.tensor_cores, "off"),
                       "l2": "flushed (256 MB write) before every timed step"},
            "accepted": int(acc_all), "solved": int(tot_all),
            "solve_stats": {"sweeps": [i["sweeps"] for i in infos], "max_rank": [i["max_rank"] for i in infos],
                            "rel_residual": [i["rel_residual"] for i in infos],
                            "refinements": [i["refinements"] for i in infos],
                            "local_iters": [i["local_iters"] for i in infos],
                            "checks": [i["checks"] for i in infos],
                            "check_ms": [round(i["check_ms"], 1) for i in infos],
                            "refine_ms": [round(i["refine_ms"], 1) for i in infos]},
            "autotune": q.autotune_table(),
            "plain": plain, "warm_start": ws_info, "gpu_launches": int(launches), "clocks": clocks,
            "roofline": roofline, "peaks": {k: peaks.get(k) for k in ("fp64_tflops", "fp32_tflops", "hbm_gbs",
                                                                       "bf16_tflops")},
            "cpu_baseline": cpu, "e2e": e2e}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
