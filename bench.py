"""Benchmark: eigensolves/s of the batched 3x3 symmetric eigensolver on GB300.

Workload (one "step"): the 2^24-matrix mixed-difficulty FP64 batch (60 %
iid N(0,1), 20 % clustered Q diag(1, 1+10^-k, -1) Q^T, 10 % near-diagonal,
10 % exact diagonals with repeats, each scaled by 10^U(-50,50)), solved for
eigenvalues and eigenvectors by one call of the C ABI.  Inputs (805 MB) and
outputs (1.6 GB) are far larger than the 129 MB L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank solves its own
2^24 batch (weak scaling, no collective on the data path); the time is the
max over ranks.  ``--impl reference`` times the CPU FP64 oracle on the host
cores instead (a bounded sample of the same workload).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "eigensolves/s at 2^24 batch (FP64 & FP32), % roofline; serving p50/p99 latency"
UNIT = "eigensolves/s"
N_MATRICES = 1 << 24
BYTES_PER_MATRIX_F64 = 48 + 24 + 72  # packed input + eigenvalues + eigenvectors
# Algorithmic FP64 operations per matrix of the mixed batch (add/sub + mul +
# div + sqrt of the paper's method as the oracle's counting scalar executes
# it, mean over the batch; tests/test_bench_constants.py re-derives it).
FLOPS_PER_MATRIX_F64 = 313.7
# FP64 peak from unit counts and clocks: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz.
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_JSON = os.path.join(ROOT, "profiles", "traffic.json")

# DRAM traffic per launch: measured by ncu on one launch of each kernel
# (--profile-case), stored per matrix in profiles/traffic.json together with
# a hash of the sources the kernel is built from, and reported only while
# that hash still matches (a changed kernel reports null).
_CSRC = os.path.join(ROOT, "paper_1806_06698_gb300", "csrc")
_COMMON = ["arith.cuh", "common.cuh", "internal.h", "../build.py"]
TRAFFIC_CASES = {
    # case: (kernel, sources, workload)
    "f64": ("k_syev3_f64", ["syev3_f64.cu", "solve_f64.cuh"] + _COMMON, "mixed FP64"),
    "f32": ("k_syev3_f32", ["syev3_f32.cu", "solve_f64.cuh"] + _COMMON, "mixed FP32, plain"),
    "f32c": ("k_syev3_f32", ["syev3_f32.cu", "solve_f64.cuh"] + _COMMON, "mixed FP32, compensated"),
    "f32ws": ("k_syev3_f32", ["syev3_f32.cu", "solve_f64.cuh", "syev3_api.cu"] + _COMMON,
              "mixed FP32, compensated through syev3_batched_ws (FP32 kernel; the refinement kernel is k_refine_f32)"),
    "bwd64": ("k_syev3_bwd", ["syev3_bwd.cu"] + _COMMON, "spectral FP64 backward"),
    "bwd32": ("k_syev3_bwd", ["syev3_bwd.cu"] + _COMMON, "spectral FP32 backward"),
}


def sources_hash(case: str) -> str:
    import hashlib

    h = hashlib.sha256()
    for f in TRAFFIC_CASES[case][1]:
        with open(os.path.normpath(os.path.join(_CSRC, f)), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_launch(case: str, n: int):
    """Measured DRAM bytes of one launch on n matrices, or None when no
    capture matches the current sources."""
    try:
        with open(TRAFFIC_JSON) as fh:
            rec = json.load(fh).get(case)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("sources") != sources_hash(case):
        return None
    return rec["bytes_per_matrix"] * n


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=60)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["native", "reference"], default="native")
    p.add_argument("--n", type=int, default=N_MATRICES, help=argparse.SUPPRESS)
    p.add_argument("--no-cpu-baseline", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--fp64-only", action="store_true", help="only the FP64 headline leg")
    p.add_argument("--serve-seconds", type=float, default=60.0,
                   help="length of the Poisson serving run (the configuration's 60 s by default)")
    p.add_argument("--profile-case", choices=sorted(TRAFFIC_CASES),
                   help="run exactly one launch of one kernel on its workload (for an ncu capture) and exit")
    p.add_argument("--record-traffic", metavar="NCU_CSV",
                   help="with --profile-case: read that case's ncu capture (dram__bytes_read.sum, "
                        "dram__bytes_write.sum) and store its bytes per matrix in profiles/traffic.json")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device="cpu") -> float:
    """The largest of every rank's x (all-reduce MAX); x itself when the
    process group is not initialised (one process)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_batch(n: int, rank: int) -> np.ndarray:
    """The batch rank `rank` solves: its own seeded 2^24 mixed batch (replicas,
    no exchange between ranks); rank 0's is the N=1 batch."""
    from paper_1806_06698_gb300 import inputs

    return inputs.mixed(n, seed=inputs.SEED_BASE + 1 + rank)[0]


def whole_job_rate(units_per_rank: int, world_size: int, steps: int, max_ms: float) -> float:
    """Units of all ranks per second over the slowest rank's time (weak
    scaling: every rank processes units_per_rank per step)."""
    return world_size * units_per_rank * steps / (max_ms * 1e-3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while active."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
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


_T0 = time.time()


def log(msg: str):
    """Progress of the legs on stderr (the JSON line stays alone on stdout)."""
    print(f"[bench {time.time() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


def load_peaks():
    try:
        with open(MEASURED_PEAKS) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform

    return platform.processor() or platform.machine()


def cpu_baseline(A: np.ndarray, sample: int, seconds_hint: float = 0.0) -> dict:
    """The CPU FP64 oracle (as it stands) over all host cores on a bounded
    sample of the workload, repeated up to about 10 core-seconds of work;
    also its single-thread rate on 2^20 matrices of the same batch."""
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    sub = np.ascontiguousarray(A[:sample])
    total, reps = 0.0, 0
    while reps < 6 and (reps == 0 or total * cores < 10.0):
        _, _, secs = oracle.syev3_timed(sub, cores)
        total += secs
        reps += 1
    one = np.ascontiguousarray(A[:min(sample, 1 << 20)])
    _, _, secs1 = oracle.syev3_timed(one, 1)
    return {"value": sample * reps / total, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {sample} matrices of the mixed FP64 batch x {reps}, std::thread over {cores} "
                      f"cores, {total:.2f} s wall ({total * cores:.1f} core-s)",
            "single_thread_value": one.shape[0] / secs1, "single_thread_sample": f"first {one.shape[0]} matrices",
            "cpu_model": _cpu_model()}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_1806_06698_gb300 import inputs

    A, _ = inputs.mixed(args.n)
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    sample = min(args.n, 1 << 21)
    times = []
    for i in range(args.warmup + args.steps):
        lo = (i * sample) % max(1, args.n - sample + 1)
        sub = np.ascontiguousarray(A[lo:lo + sample])
        _, _, secs = oracle.syev3_timed(sub, cores)
        if i >= args.warmup:
            times.append(secs)
    tot = sum(times)
    value = sample * len(times) / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "mixed FP64 batch (2^24 recipe), CPU oracle on a bounded sample",
                   "sample_per_step": sample, "threads": cores},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample} matrices of the 2^24 mixed FP64 batch per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measure_fp64_peak(dev, stream, repeats: int = 5) -> dict:
    """The FP64 operation rate of this GPU, measured: the library's DFMA probe
    (independent FP64 fused multiply-add chains on every resident thread)
    timed with CUDA events on ``stream``; best of ``repeats`` launches of
    about 20 ms, 2 flops per DFMA."""
    import torch

    from paper_1806_06698_gb300 import syev3

    sink = torch.zeros(1, dtype=torch.float64, device=dev)
    syev3.probe_dfma(1000, sink, stream=stream)
    best = 0.0
    iters = 200_000
    for _ in range(repeats):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        count = syev3.probe_dfma(iters, sink, stream=stream)
        t1.record(stream)
        t1.synchronize()
        best = max(best, count / (t0.elapsed_time(t1) * 1e-3))
    return {"dfma_per_s": best, "tflops": 2 * best / 1e12, "launches": repeats,
            "probe": "syev3_probe_dfma: 8 independent DFMA chains per thread, every resident thread, best of "
                     f"{repeats} launches"}


def _timed(step, steps: int, warmup: int, stream, barrier):
    """Run ``warmup`` untimed then ``steps`` timed calls of ``step`` on
    ``stream``; returns (total ms, per-launch ms) from CUDA events recorded on
    that stream."""
    import torch

    for _ in range(warmup):
        step()
    barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(steps):
        ev[2 * i].record(stream)
        step()
        ev[2 * i + 1].record(stream)
    t1.record(stream)
    barrier()
    return t0.elapsed_time(t1), [ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(steps)]


def _fp32_legs(args, dev, stream, barrier, A64_dev):
    """Precision form: the 2^24 mixed batch in FP32 (scale 10^U(-6,6)) and
    2^26 FP32 structure tensors, plain FP32 and compensated, each timed like
    the headline and checked against the FP64 kernel on a sample."""
    import torch

    from paper_1806_06698_gb300 import inputs, syev3

    hbm = load_peaks().get("hbm_gbs", 6686.1)
    out = {}
    A_mix, ids_mix = inputs.mixed_fp32(args.n)
    sets = [("mixed_fp32_2^24", A_mix, ids_mix),
            ("structure_tensors_fp32_2^26", inputs.structure_tensors(4 * args.n).astype(np.float32), None)]
    for name, A_np, ids in sets:
        n = A_np.shape[0]
        A = torch.from_numpy(A_np).to(dev)
        lam = torch.empty((n, 3), dtype=torch.float32, device=dev)
        U = torch.empty((n, 3, 3), dtype=torch.float32, device=dev)
        # FP64 solve of a sample of the same (upcast) matrices as the accuracy reference.
        idx = torch.arange(0, n, max(1, n // (1 << 18)), device=dev)
        A_ref = A[idx].double().contiguous()
        lam_ref, _ = syev3.syev3_batched(A_ref, stream=stream)
        lam_ref_h = lam_ref.cpu().numpy()
        nrm_h = np.linalg.norm(lam_ref_h, axis=1)
        # compensated: syev3_batched_ws (the FP64 refinement as a second
        # kernel over a list in a workspace); compensated_single_kernel:
        # syev3_batched (the refinement inside the FP32 kernel).
        ws = torch.empty(syev3.workspace_bytes(n, torch.float32, compensated=True), dtype=torch.uint8, device=dev)
        for mode in ("plain", "compensated", "compensated_single_kernel"):
            comp = mode != "plain"
            work = ws if mode == "compensated" else None
            ctr = torch.zeros(syev3.NUM_COUNTERS, dtype=torch.int64, device=dev)

            def step():
                syev3.syev3_batched(A, out=(lam, U), compensated=comp, workspace=work, stream=stream)

            total_ms, kms = _timed(step, args.steps, args.warmup, stream, barrier)
            log(f"  {name} {mode}: {total_ms / args.steps:.3f} ms per step")
            syev3.syev3_batched(A, out=(lam, U), compensated=comp, counters=ctr, workspace=work, stream=stream)
            barrier()
            # Accuracy on the host (no library GEMM in the bench's launch list).
            lam_s, U_s = lam[idx].double().cpu().numpy(), U[idx].double().cpu().numpy()
            dl_each = np.max(np.abs(lam_s - lam_ref_h), axis=1) / np.maximum(nrm_h, 1e-300)
            dl = float(np.max(dl_each))
            per_subset = None
            if ids is not None:
                sid = ids[idx.cpu().numpy()]
                per_subset = {inputs.SUBSET_NAMES[k]: float(np.max(dl_each[sid == k]) / 2.0 ** -23)
                              for k in inputs.SUBSET_NAMES if np.any(sid == k)}
            orth = float(np.max(np.linalg.norm(np.einsum("nki,nkj->nij", U_s, U_s) - np.eye(3), axis=(1, 2))))
            k = statistics.mean(kms)
            gbs = 72 * n / (k * 1e-3) / 1e9
            out[f"{name}_{mode}"] = {
                "value": n * args.steps / (total_ms * 1e-3), "unit": UNIT, "ms_per_step": total_ms / args.steps,
                "dtype": "f32", "n": n,
                "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                             "traffic": traffic_per_launch({"plain": "f32", "compensated": "f32ws"}.get(mode, "f32c"), n),
                             "kernel": "k_syev3_f32" + (" + k_refine_f32" if work is not None else ""),
                             "peak_source": "MEASURED_PEAKS hbm_gbs"},
                "fp64_refined_fraction": ctr[2].item() / n if comp else 0.0,
                "max_dlambda_vs_fp64_kernel_eps32": dl / 2.0 ** -23,
                "max_dlambda_vs_fp64_kernel_eps32_per_subset": per_subset,
                "max_orthogonality_eps32": orth / 2.0 ** -23,
                "accuracy_sample": int(idx.numel()),
            }
        # Eigenvalues only (plain FP32, U = NULL): 24 B in + 12 B out.
        lam_v = torch.empty((n, 3), dtype=torch.float32, device=dev)

        def vstep():
            syev3.syev3_batched(A, out=(lam_v, None), stream=stream)

        v_ms, v_kms = _timed(vstep, args.steps, args.warmup, stream, barrier)
        k = statistics.mean(v_kms)
        gbs = 36 * n / (k * 1e-3) / 1e9
        out[f"{name}_plain_eigenvalues_only"] = {
            "value": n * args.steps / (v_ms * 1e-3), "unit": UNIT, "ms_per_step": v_ms / args.steps, "dtype": "f32",
            "n": n, "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                                 "traffic": None, "kernel": "k_syev3_f32<plain, values only>",
                                 "peak_source": "MEASURED_PEAKS hbm_gbs"}}
        del A, lam, U, A_ref, ws, lam_v
        torch.cuda.empty_cache()
    return out


BWD_BYTES = {"f64": 240, "f32": 120}  # lambda, U, g_lambda, g_U in + packed gradient out
# Algorithmic operations of one backward: the antisymmetric part of U^T gU
# (36), ||A||_F and the gaps (9), the masked couplings (12), P = U sym(C)
# (45), the upper triangle of P U^T (33) and the doubling (3).
BWD_FLOPS = 138


def _bwd_legs(args, dev, stream, barrier, fp64_peak=None):
    """Differentiation form: 2^20 matrices Q diag(d) Q^T (95 % gaps >= 1e-3,
    5 % near-degenerate, masked with tau = 1e-6), loss sum w lambda + sum V o U,
    the backward kernel timed alone in FP64 and FP32."""
    import torch

    from paper_1806_06698_gb300 import inputs, syev3

    n = max(1, args.n // 16)
    A_np, _, _ = inputs.spectral(n, seed=inputs.SEED_BASE + 4)
    rng = np.random.default_rng(inputs.SEED_BASE + 6)
    wn, Vn = rng.standard_normal((n, 3)), rng.standard_normal((n, 3, 3))
    hbm = load_peaks().get("hbm_gbs", 6686.1)
    out = {}
    for dt, name in ((torch.float64, "f64"), (torch.float32, "f32")):
        A = torch.from_numpy(A_np).to(dev, dt)
        lam, U = syev3.syev3_batched(A, stream=stream)
        w, V = torch.from_numpy(wn).to(dev, dt), torch.from_numpy(Vn).to(dev, dt)
        gA = torch.empty((n, 6), dtype=dt, device=dev)

        def step():
            syev3.syev3_batched_bwd(lam, U, w, V, 1e-6, out=gA, stream=stream)

        # One call at a time from Python: at 2^20 matrices (about 20 us of
        # kernel per FP32 call) the host's per-call cost shows as GPU idle
        # time between the launches.
        api_ms, api_kms = _timed(step, args.steps, args.warmup, stream, barrier)
        # The kernel's throughput: the same K calls captured in one CUDA
        # graph (the library's launches are capture-safe) and replayed.
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(args.steps):
                syev3.syev3_batched_bwd(lam, U, w, V, 1e-6, out=gA)
        graph.replay()
        barrier()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        graph.replay()
        g1.record(stream)
        barrier()
        total_ms = g0.elapsed_time(g1)
        k = total_ms / args.steps
        rate = n / (k * 1e-3)
        del graph
        if name == "f64":
            roof = {"bound": "alu", "achieved": BWD_FLOPS * rate / 1e12, "peak": FP64_PEAK_GFLOPS / 1e3,
                    "unit": "TFLOP/s", "frac": BWD_FLOPS * rate / 1e9 / FP64_PEAK_GFLOPS,
                    "hbm_frac_of_measured": BWD_BYTES[name] * rate / 1e9 / hbm}
            if fp64_peak:
                roof["peak_measured"] = fp64_peak["tflops"]
                roof["frac_of_measured"] = BWD_FLOPS * rate / 1e12 / fp64_peak["tflops"]
        else:
            roof = {"bound": "hbm", "achieved": BWD_BYTES[name] * rate / 1e9, "peak": hbm, "unit": "GB/s",
                    "frac": BWD_BYTES[name] * rate / 1e9 / hbm}
        roof.update({"kernel": "k_syev3_bwd", "traffic": traffic_per_launch("bwd" + name[1:], n)})
        out[f"backward_{name}_2^20"] = {
            "value": n * args.steps / (total_ms * 1e-3), "unit": "gradients/s",
            "ms_per_step": total_ms / args.steps, "n": n, "roofline": roof,
            "timing": f"{args.steps} syev3_batched_bwd calls captured in one CUDA graph, replayed",
            "api_loop": {"value": n * args.steps / (api_ms * 1e-3), "ms_per_step": api_ms / args.steps,
                         "ms_per_step_events": statistics.mean(api_kms),
                         "what": "the same calls one at a time from Python (host-bound at this size)"}}
        del A, lam, U, w, V, gA
    return out


def _host_errors(A6: np.ndarray, lam: np.ndarray, U: np.ndarray):
    """Per matrix, on the host in FP64: ||A U - U Lambda||_F / ||A||_F and
    ||U^T U - I||_F."""
    from paper_1806_06698_gb300 import inputs

    M = inputs.unpack(A6)
    nrm = np.linalg.norm(M, axis=(1, 2))
    res = np.linalg.norm(M @ U - U * lam[:, None, :], axis=(1, 2)) / np.where(nrm > 0, nrm, 1.0)
    orth = np.linalg.norm(np.einsum("nki,nkj->nij", U, U) - np.eye(3), axis=(1, 2))
    return res, orth


def _method_study_leg(args, dev, stream, barrier):
    """The method variants (syev3_batched_method) on the mixed batch and its
    subsets: the production path, the FP64 Borges-Gragg iteration from
    Eq. (7) and Newton's method (Sec. 1.4.2); then the simplified against the
    EISPACK-style deflation test (Sec. 1.1)."""
    import torch

    from paper_1806_06698_gb300 import inputs, syev3

    n = max(1 << 12, args.n // 4)
    A_np, ids = inputs.mixed(n, seed=inputs.SEED_BASE + 1)
    names = {"production": syev3.ZF_PRODUCTION, "borges_gragg": syev3.ZF_BORGES_GRAGG, "newton": syev3.ZF_NEWTON}
    subsets = [("mixed", None)] + [(v, k) for k, v in inputs.SUBSET_NAMES.items()]
    sample = 1 << 14
    out = {"n": n, "zero_finder": {}, "deflation_test": {}}
    for sub, sid in subsets:
        Ah = A_np if sid is None else np.ascontiguousarray(A_np[ids == sid])
        m = Ah.shape[0]
        A = torch.from_numpy(Ah).to(dev)
        lam = torch.empty((m, 3), dtype=torch.float64, device=dev)
        U = torch.empty((m, 3, 3), dtype=torch.float64, device=dev)
        idx = np.linspace(0, m - 1, min(m, sample)).astype(np.int64)
        lam_bg = None
        rows = {}
        for name in ("borges_gragg", "production", "newton"):
            zf = names[name]
            stats = torch.zeros(len(syev3.METHOD_STATS), dtype=torch.int64, device=dev)

            def step():
                syev3.syev3_batched_method(A, zero_finder=zf, out=(lam, U), stream=stream)

            total_ms, _ = _timed(step, args.steps if args.steps < 10 else 10, 2, stream, barrier)
            reps = args.steps if args.steps < 10 else 10
            syev3.syev3_batched_method(A, zero_finder=zf, out=(lam, U), stats=stats, stream=stream)
            barrier()
            st = dict(zip(syev3.METHOD_STATS, stats.cpu().tolist()))
            lam_s, U_s = lam.cpu().numpy()[idx], U.cpu().numpy()[idx]
            res, orth = _host_errors(Ah[idx], lam_s, U_s)
            nrm = np.linalg.norm(inputs.unpack(Ah[idx]), axis=(1, 2))
            row = {"value": m * reps / (total_ms * 1e-3), "unit": UNIT,
                   "steps_per_root": st["steps"] / max(1, st["roots"]),
                   "simt_efficiency": st["steps"] / max(1, st["warp_slots"]),
                   "roots_full_iteration": st["roots"], "capped": st["capped"],
                   "max_residual_rel": float(res.max()), "max_orthogonality": float(orth.max())}
            if lam_bg is None:
                lam_bg = lam_s
            else:
                row["max_dlambda_vs_borges_gragg_rel"] = float(
                    np.max(np.max(np.abs(lam_s - lam_bg), axis=1) / np.where(nrm > 0, nrm, 1.0)))
            rows[name] = row
        out["zero_finder"][sub] = rows
        del A, lam, U
    # Deflation test: simplified (Sec. 1.1, adopted) vs EISPACK-style.
    for name, Ah in (("mixed", A_np), ("trace_free_spiked", inputs.trace_free_spiked(min(n, 1 << 20)))):
        m = Ah.shape[0]
        A = torch.from_numpy(Ah).to(dev)
        res_l = {}
        row = {}
        for defl, key in ((syev3.DEFLATION_SIMPLIFIED, "simplified"), (syev3.DEFLATION_EISPACK, "eispack")):
            stats = torch.zeros(len(syev3.METHOD_STATS), dtype=torch.int64, device=dev)
            lam, U = syev3.syev3_batched_method(A, deflation_test=defl, stats=stats, stream=stream)
            barrier()
            st = dict(zip(syev3.METHOD_STATS, stats.cpu().tolist()))
            idx = np.linspace(0, m - 1, min(m, sample)).astype(np.int64)
            res, orth = _host_errors(Ah[idx], lam.cpu().numpy()[idx], U.cpu().numpy()[idx])
            res_l[key] = lam.cpu().numpy()
            row[key] = {"deflated_fraction": st["deflated"] / m, "max_residual_rel": float(res.max()),
                        "max_orthogonality": float(orth.max())}
        nrm = np.linalg.norm(inputs.unpack(Ah), axis=(1, 2))
        row["max_dlambda_between_rel"] = float(np.max(np.max(np.abs(res_l["eispack"] - res_l["simplified"]), axis=1)
                                                     / np.where(nrm > 0, nrm, 1.0)))
        out["deflation_test"][name] = row
        del A
    torch.cuda.empty_cache()
    return out


def _accuracy_experiment(dev, stream, n: int = 100_000):
    """The test of Sec. 1.5 on this solver: n symmetric matrices with iid
    entries from U(0,1), N(0,1) and chi^2_1; ||I - V^T V||_F and
    ||T V - V Lambda||_F of the FP64 kernel and of LAPACK (numpy.linalg.eigh),
    differenced per matrix as LAPACK minus ours (positive where ours is more
    accurate) and summarised (the paper plots them sorted)."""
    import torch

    from paper_1806_06698_gb300 import inputs, syev3

    out = {"n": n, "reference": "numpy.linalg.eigh (LAPACK dsyevd) on the host"}
    for dist in ("uniform", "normal", "chisq"):
        T6 = inputs.paper_set(n, dist)
        lam, U = syev3.syev3_batched(torch.from_numpy(T6).to(dev), stream=stream)
        torch.cuda.synchronize(dev)
        lam, U = lam.cpu().numpy(), U.cpu().numpy()
        M = inputs.unpack(T6)
        lam_l, U_l = np.linalg.eigh(M)
        row = {}
        for meas, f in (("orthogonality", lambda L, V: np.linalg.norm(np.einsum("nki,nkj->nij", V, V) - np.eye(3),
                                                                         axis=(1, 2))),
                        ("residual", lambda L, V: np.linalg.norm(M @ V - V * L[:, None, :], axis=(1, 2)))):
            ours, ref = f(lam, U), f(lam_l, U_l)
            d = np.sort(ref - ours)
            row[meas] = {"ours_median": float(np.median(ours)), "lapack_median": float(np.median(ref)),
                         "ours_max": float(ours.max()), "lapack_max": float(ref.max()),
                         "frac_ours_better": float(np.mean(d > 0)), "frac_equal": float(np.mean(d == 0)),
                         "frac_lapack_better": float(np.mean(d < 0)),
                         "diff_quantiles_1_50_99": [float(np.quantile(d, q)) for q in (0.01, 0.5, 0.99)]}
        out[dist] = row
    return out


# Serving configuration: matrices of one request per round, matrices per
# round, rounds queued on the device.
SERVE_CHUNK, SERVE_ROUND, SERVE_INFLIGHT = 1 << 18, 1 << 21, 2


def _serving_leg(args, dev, A64):
    """Serving form: Poisson arrivals at 2000 requests/s for --serve-seconds,
    each request N = floor(exp(U(0, ln 2^22))) matrices, 70 % FP64 / 30 %
    FP32 (compensated), sliced from device-resident pools of the mixed
    batches, through a server with a 16 GiB budget.  Latency = the library's
    own submit -> done timestamps."""
    import threading

    import torch

    from paper_1806_06698_gb300 import inputs, syev3

    A32 = torch.from_numpy(inputs.mixed_fp32(A64.shape[0])[0]).to(dev)
    rng = np.random.default_rng(inputs.SEED_BASE + 7)
    rate, T = 2000.0, float(args.serve_seconds)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, int(rate * T * 1.2) + 16))
    arrivals = arrivals[arrivals < T]
    m = len(arrivals)
    sizes = np.floor(np.exp(rng.uniform(0.0, np.log(2.0 ** 22), m))).astype(np.int64)
    sizes = np.minimum(sizes, A64.shape[0])
    is64 = rng.uniform(0, 1, m) < 0.7
    offs = (rng.uniform(0, 1, m) * (A64.shape[0] - sizes + 1)).astype(np.int64)
    srv = syev3.Server(memory_budget_bytes=16 << 30, chunk=SERVE_CHUNK, round_matrices=SERVE_ROUND,
                       max_rounds_in_flight=SERVE_INFLIGHT)
    for k in range(8):  # warm-up requests (released: each holds a slot of the request ring)
        t = srv.submit(A64[: 1 << 16])
        srv.wait(t, 60.0)
        srv.release(t)
    tickets = [None] * m
    t_arrive = np.zeros(m, np.int64)
    retries = [0]
    failure = [None]
    ready = threading.Semaphore(0)

    def client():
        # Arrival = when the client issues the request (host monotonic clock,
        # the clock of the library's timestamps); a full request ring
        # (SYEV3_EAGAIN) is retried and the wait counts as latency.
        t0 = time.perf_counter()
        for i in range(m):
            dt = arrivals[i] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            pool = A64 if is64[i] else A32
            t_arrive[i] = time.monotonic_ns()
            try:
                while True:
                    try:
                        tickets[i] = srv.submit(pool[offs[i]:offs[i] + sizes[i]], compensated=not is64[i])
                        break
                    except syev3.Syev3Error as e:
                        if e.status != syev3.SYEV3_EAGAIN or time.monotonic_ns() - t_arrive[i] > 60e9:
                            raise
                        retries[0] += 1
                        time.sleep(0.0002)
            except Exception as e:  # hand the failure to the waiting thread instead of hanging it
                failure[0] = e
                ready.release()
                return
            ready.release()

    lat, queue, solve, t_first, t_last, waited = [], [], [], None, 0, 0
    th = threading.Thread(target=client, daemon=True)
    th.start()
    for i in range(m):
        ready.acquire()
        if failure[0] is not None:
            th.join()
            srv.close()
            raise RuntimeError(f"serving client failed at request {i}: {failure[0]}")
        if i % 20000 == 0:
            log(f"  serving: request {i} of {m}")
        info = srv.wait(tickets[i], 120.0)
        lat.append((info.t_done_ns - t_arrive[i]) * 1e-6)
        queue.append((info.t_admit_ns - info.t_submit_ns) * 1e-6)
        solve.append((info.t_done_ns - info.t_admit_ns) * 1e-6)
        t_first = info.t_submit_ns if t_first is None else min(t_first, info.t_submit_ns)
        t_last = max(t_last, info.t_done_ns)
        waited += info.t_admit_ns - info.t_submit_ns > 1_000_000
        srv.release(tickets[i])
    th.join()
    st = srv.stats()
    srv.close()
    lat, queue, solve = np.array(lat), np.array(queue), np.array(solve)
    total = int(sizes.sum())
    span = (t_last - t_first) * 1e-9
    return {"requests": m, "seconds": T, "arrival_rate_per_s": rate, "matrices": total,
            "offered_matrices_per_s": total / T, "value": total / span, "unit": UNIT,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "breakdown": {"queue_p50_ms": float(np.percentile(queue, 50)),
                          "queue_p99_ms": float(np.percentile(queue, 99)),
                          "solve_p50_ms": float(np.percentile(solve, 50)),
                          "solve_p99_ms": float(np.percentile(solve, 99)),
                          "what": "queue = submit to admission on the device; solve = admission to the end of "
                                  "the request's last round (device timer mapped to the host clock)"},
            "rounds": int(st.rounds), "launches": int(st.launches), "ring_full_retries": int(retries[0]),
            "latency": "request arrival (client, host monotonic clock) to the device's completion timestamp",
            "max_ms": float(lat.max()), "mean_ms": float(lat.mean()),
            "p99_ms_small_requests_le_4096": float(np.percentile(lat[sizes <= 4096], 99)),
            "arena_peak_bytes": int(st.arena_peak), "memory_budget_bytes": 16 << 30,
            "queued_over_1ms": int(waited), "chunks": int(st.chunks),
            "config": "Poisson 2000 req/s, N log-uniform [1, 2^22], 70% FP64 / 30% FP32 compensated, "
                      f"device-resident queues and admission, chunks of {SERVE_CHUNK} per request per round, "
                      f"{SERVE_ROUND} matrices per round, {SERVE_INFLIGHT} rounds in flight, 16 GiB budget"}


def run_native(args):
    import torch

    from paper_1806_06698_gb300 import build, inputs, syev3

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    build.build()
    n = args.n
    A_np = replica_batch(n, rank)
    A = torch.from_numpy(A_np).to(dev)
    lam = torch.empty((n, 3), dtype=torch.float64, device=dev)
    U = torch.empty((n, 3, 3), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    def step():
        syev3.syev3_batched(A, out=(lam, U), stream=stream)

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    total_ms, kernel_ms = _timed(step, args.steps, args.warmup, stream, barrier)
    clocks = sampler.stop()
    total_ms = max_over_ranks(total_ms, dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(n, ws, args.steps, total_ms)

    # End to end through the C ABI's host entry point: pinned host buffers in,
    # the pipelined H2D copy / solve / D2H copy of eigenvalues and
    # eigenvectors inside the timed region (the call returns when the host
    # outputs are written).
    A_host = torch.from_numpy(A_np).pin_memory()
    lam_host = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    U_host = torch.empty((n, 3, 3), dtype=torch.float64).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))

    def e2e_step():
        syev3.syev3_batched_host(A_host, lam_host, U_host, stream=stream)

    e2e_ms, e2e_each = _timed(e2e_step, e2e_steps, 1, stream, barrier)
    e2e_ms = max_over_ranks(e2e_ms, dev)
    e2e_value = whole_job_rate(n, ws, e2e_steps, e2e_ms)
    # The host link is shared with other jobs on the machine: the spread of
    # the steps shows whether a slow run was contention (a few slow steps)
    # or the pipeline (all steps alike).  The value stays the whole run.
    e2e_each = sorted(e2e_each)

    # Eigenvalues only (U = NULL): the same batch, no eigenvectors formed or
    # written (24 B out per matrix).
    lam_only = torch.empty((n, 3), dtype=torch.float64, device=dev)

    def values_step():
        syev3.syev3_batched(A, out=(lam_only, None), stream=stream)

    v_ms, v_kms = _timed(values_step, min(args.steps, 20), args.warmup, stream, barrier)
    v_rate = n * min(args.steps, 20) / (v_ms * 1e-3)
    values_only = {"value": v_rate, "unit": UNIT, "ms_per_step": v_ms / min(args.steps, 20),
                   "bytes_per_matrix": 72, "hbm_frac_of_measured": 72 * v_rate / 1e9 /
                   load_peaks().get("hbm_gbs", 6686.1), "kernel": "k_syev3_f64<bulk, production, values only>"}
    del lam_only

    log("headline, e2e and eigenvalues-only legs done")
    fp64_peak = measure_fp64_peak(dev, stream)
    log("FP64 peak probe done")
    fp32 = None if args.fp64_only else _fp32_legs(args, dev, stream, barrier, A)
    log("precision-form legs done")
    bwd = None if args.fp64_only else _bwd_legs(args, dev, stream, barrier, fp64_peak)
    log("differentiation-form legs done")
    serving = None if (args.fp64_only or args.serve_seconds <= 0) else _serving_leg(args, dev, A)
    log("serving leg done")
    study = None if args.fp64_only else _method_study_leg(args, dev, stream, barrier)
    log("method-study leg done")
    accuracy = None if args.fp64_only else _accuracy_experiment(dev, stream)
    log("accuracy-experiment leg done")

    if rank == 0:
        kms = statistics.mean(kernel_ms)
        achieved = FLOPS_PER_MATRIX_F64 * n / (kms * 1e-3) / 1e9  # GFLOP/s
        roofline = {"bound": "alu", "achieved": achieved / 1e3, "peak": FP64_PEAK_GFLOPS / 1e3,
                    "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_GFLOPS, "traffic": None,
                    "kernel": "k_syev3_f64", "peak_source": "152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz",
                    "peak_measured": fp64_peak["tflops"],
                    "frac_of_measured": achieved / 1e3 / fp64_peak["tflops"],
                    "peak_measured_source": fp64_peak["probe"],
                    "kernel_ms": kms,
                    "hbm_frac_of_measured": (BYTES_PER_MATRIX_F64 * n / (kms * 1e-3) / 1e9) /
                    load_peaks().get("hbm_gbs", 6686.1)}
        roofline["traffic"] = traffic_per_launch("f64", n)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "2^24 mixed-difficulty FP64 batch (60% N(0,1), 20% clustered, 10% "
                                   "near-diagonal, 10% exact diagonal w/ repeats, x10^U(-50,50))",
                       "n_per_gpu": n, "outputs": "eigenvalues + eigenvectors",
                       "l2": "inputs and outputs > L2 (805 MB in, 1.6 GB out); no flush needed",
                       "parallelism": f"replicas x{ws}"},
            "roofline": roofline,
            "gpu_launches": args.steps,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * 48,
                    "d2h_bytes_per_step": n * 96, "api": "syev3_batched_host (pinned host buffers, "
                    "3-stream copy/solve pipeline, chunks of 2^16 growing by a quarter to 2^20)",
                    "steps": e2e_steps, "ms_per_step": e2e_ms / e2e_steps,
                    "ms_per_step_min": e2e_each[0], "ms_per_step_median": e2e_each[len(e2e_each) // 2]},
            "clocks": clocks,
        }
        line["eigenvalues_only"] = values_only
        if fp32 is not None:
            line["precision_form"] = fp32
        if bwd is not None:
            line["differentiation_form"] = bwd
        if serving is not None:
            line["serving"] = serving
        if study is not None:
            line["method_study"] = study
        if accuracy is not None:
            line["accuracy_experiment"] = accuracy
        if not args.no_cpu_baseline and ws == 1:  # the host-core baseline: rank 0 at N = 1 only
            line["cpu_baseline"] = cpu_baseline(A_np, n)
            log("CPU baseline done")
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def _profile_inputs(case: str, n: int):
    from paper_1806_06698_gb300 import inputs

    if case == "f64":
        return inputs.mixed(n, seed=inputs.SEED_BASE + 1)[0]
    if case in ("f32", "f32c", "f32ws"):
        return inputs.mixed_fp32(n)[0]
    return inputs.spectral(n, seed=inputs.SEED_BASE + 4)[0]


def run_profile_case(args):
    """One launch of one kernel on its workload (n matrices): the command an
    ncu capture of that kernel runs.  The backward cases first run the
    forward solve they differentiate (a k_syev3_f64/f32 launch)."""
    import torch

    from paper_1806_06698_gb300 import build, syev3

    build.build()
    case, n = args.profile_case, args.n
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    dt = torch.float32 if case in ("f32", "f32c", "f32ws", "bwd32") else torch.float64
    A = torch.from_numpy(_profile_inputs(case, n)).to(dev, dt)
    lam = torch.empty((n, 3), dtype=dt, device=dev)
    U = torch.empty((n, 3, 3), dtype=dt, device=dev)
    ws = None
    if case == "f32ws":
        ws = torch.empty(syev3.workspace_bytes(n, dt, compensated=True), dtype=torch.uint8, device=dev)
    syev3.syev3_batched(A, out=(lam, U), compensated=case in ("f32c", "f32ws"), workspace=ws, stream=stream)
    if case.startswith("bwd"):
        rng = np.random.default_rng(1806066986)
        w = torch.from_numpy(rng.standard_normal((n, 3))).to(dev, dt)
        V = torch.from_numpy(rng.standard_normal((n, 3, 3))).to(dev, dt)
        gA = torch.empty((n, 6), dtype=dt, device=dev)
        syev3.syev3_batched_bwd(lam, U, w, V, 1e-6, out=gA, stream=stream)
    torch.cuda.synchronize(dev)
    print(json.dumps({"profile_case": case, "n": n, "kernel": TRAFFIC_CASES[case][0]}), flush=True)


_BYTE_UNITS = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}


def record_traffic(args):
    """Store DRAM bytes per matrix of --profile-case from its ncu CSV
    (the first launch of the case's kernel in the capture)."""
    import csv

    case, n = args.profile_case, args.n
    kernel = TRAFFIC_CASES[case][0]
    with open(args.record_traffic) as fh:
        rows = list(csv.reader(line for line in fh if line.startswith('"')))
    hdr = rows[0]
    ki, mi, ui, vi, ii = (hdr.index(k) for k in ("Kernel Name", "Metric Name", "Metric Unit", "Metric Value", "ID"))
    # Every launch of the case's kernel in the capture, summed: the
    # pipelined compensated path launches the FP32 kernel once per run.
    launches, got = set(), {"dram__bytes_read.sum": 0.0, "dram__bytes_write.sum": 0.0}
    for r in rows[1:]:
        if kernel not in r[ki]:
            continue
        launches.add(r[ii])
        if r[mi] in got:
            got[r[mi]] += float(r[vi].replace(",", "")) * _BYTE_UNITS[r[ui]]
    rd, wr = got["dram__bytes_read.sum"], got["dram__bytes_write.sum"]
    try:
        with open(TRAFFIC_JSON) as fh:
            table = json.load(fh)
    except (OSError, ValueError):
        table = {}
    table[case] = {"kernel": kernel, "workload": TRAFFIC_CASES[case][2], "n": n, "sources": sources_hash(case),
                   "launches": len(launches),
                   "dram_read_bytes": rd, "dram_write_bytes": wr, "bytes_per_matrix": (rd + wr) / n,
                   "command": f"ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
                              f"--clock-control none -k regex:{kernel} -c {len(launches)} --csv "
                              f"python bench.py --profile-case {case} --n {n}"}
    with open(TRAFFIC_JSON, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)
        fh.write("\n")
    print(json.dumps(table[case]))


def main():
    args = parse()
    if args.profile_case and args.record_traffic:
        record_traffic(args)
        return
    if args.profile_case:
        run_profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
