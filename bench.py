"""Throughput of the local SDDMM + SpMM step on GB300.

A step is one pass of the hot path over one batch of input: out = SDDMM(S, A, B)
(Eq. 1) followed by C = SpMM(S, B) (Eq. 2) on the power-law workload (R-MAT
scale 20, edge factor 16, K = 64, FP32), inputs resident in HBM, L2 flushed
between steps.  Metric: GFLOP/s = 2 * (2 * nnz * K) / step time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload rmat20|tiny|rec|gnn] [--dtype f32|bf16]

Prints one JSON line (rank 0).  With torchrun, every rank runs an independent
replica on its own GPU (the step has no data exchange) and the line reports
the aggregate over ranks, timed by the slowest rank.

--impl reference times the FP64 CPU oracle (the reference implementation) on a
bounded row sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "SDDMM+SpMM GFLOP/s (2*nnz*K per op)"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------
def load_workload(name: str):
    if name == "rmat20":
        P = synth.rmat_problem(20, 16, 64, seed=0)
        desc = ("rmat20: R-MAT scale 20 (1,048,576 x 1,048,576), edge factor 16, (a,b,c,d)=(0.57,0.19,0.19,0.05), "
                "duplicates removed, values U[-1,1]; A, B 2^20 x 64 N(0,1)")
    elif name == "tiny":
        P = synth.tiny(seed=0)
        desc = "tiny: 4096 x 4096, 16 distinct uniform columns per row, values U[-1,1]; A, B 4096 x 32 U[-1,1]"
    elif name == "rec":
        P = synth.rec(seed=0)
        desc = ("rec: 2,000,000 x 500,000 Chung-Lu, Zipf(1.1) weights clipped to [1,20000], 50,000,000 nnz, "
                "values U{1..5}; A 2M x 128, B 500K x 128 N(0,1)")
    elif name == "gnn":
        P = synth.gnn(seed=0)
        P.vals = None
        desc = "gnn: R-MAT scale 22, edge factor 8, unit values; A = B = H 2^22 x 64 N(0,0.1)"
    else:
        raise SystemExit(f"unknown workload {name}")
    return P, desc


def algorithmic_bytes(P, elt: int) -> dict:
    """Compulsory HBM bytes per launch: every input read once, every output
    written once (index arrays int32, values FP32, factors `elt` bytes)."""
    M, N, K, nnz = P.M, P.N, P.K, P.nnz
    sddmm = 4 * (M + 1) + 4 * nnz + 4 * nnz + M * K * elt + N * K * elt + 4 * nnz
    spmm = 4 * (M + 1) + 8 * nnz + N * K * elt + M * K * 4
    return {"sddmm": sddmm, "spmm": spmm}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d.get("bf16_tflops", 0))}, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


# The files the step kernels (k_sddmm_ring, k_spmm_ring and their register
# and row-split siblings) compile from: a change elsewhere in csrc/ (FusedMM,
# batch, tensor-core tiles, plans) leaves their ncu traffic valid.
STEP_KERNEL_SOURCES = ("common.cuh", "tiles.cuh", "lean.cuh", "ring.cuh", "sddmm_impl.cuh", "spmm_impl.cuh",
                       "sddmm_f32.cu", "sddmm_bf16.cu", "sddmm_f16.cu", "sddmm_e4m3.cu",
                       "spmm_f32.cu", "spmm_bf16.cu", "spmm_f16.cu", "spmm_e4m3.cu")


def kernel_sources_sha() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2404_19638_gb300", "csrc")
    for f in STEP_KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, dtype: str):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"sddmm_spmm_{workload}_{dtype}.md")
    if not os.path.exists(path):
        return None
    m = re.search(r"^traffic_per_launch:\s*(\{.*\})\s*$", open(path).read(), flags=re.M)
    if not m:
        return None
    d = json.loads(m.group(1))
    if d.get("source_sha") != kernel_sources_sha():
        return None
    return d


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class _Nvml:
    """Minimal ctypes access to NVML (read-only queries: clocks and the active
    clock-event reasons); None where the library is absent."""
    SM = 1                                   # NVML_CLOCK_SM
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, gpu_index: int):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(gpu_index), ctypes.byref(self.h)) != 0:
            raise OSError("no NVML handle")
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        m = ctypes.c_uint()
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.SM, ctypes.byref(m))
        self.max_mhz = float(m.value)

    def sample(self):
        c, r = self.ct.c_uint(), self.ct.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, self.SM, self.ct.byref(c)) != 0:
            return None
        self.reasons_fn(self.h, self.ct.byref(r))
        return float(c.value), self.max_mhz, [n for b, n in self.REASONS.items() if r.value & b]


class ClockSampler:
    """SM clock and clock-event reasons sampled during the timed region: NVML
    every millisecond where the library loads (a 20-step region of ~20 ms still
    gets tens of samples), else nvidia-smi every 100 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_s: float = 0.001):
        self.gpu = gpu_index
        self.period = period_s
        self.proc = None
        self.nvml = None
        self.stop = False
        self.rows = []                        # (host time, sm_mhz, max_mhz, [reasons])
        self.window = None
        self.source = None

    def __enter__(self):
        try:
            self.nvml = _Nvml(self.gpu)
            self.source = "nvml, every 1 ms"
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()
            return self
        except Exception:
            self.nvml = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi, every 100 ms"
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.perf_counter()
            while not self.rows and time.perf_counter() - t0 < 5.0:     # sampler running before timing
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def _poll(self):
        while not self.stop:
            r = self.nvml.sample()
            if r is not None:
                self.rows.append((time.perf_counter(),) + r)
            time.sleep(self.period)

    def _read(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.proc.stdout:
            p = [x.strip() for x in line.strip().split(",")]
            if len(p) < 9:
                continue
            try:
                self.rows.append((time.perf_counter(), float(p[1]), float(p[2]),
                                  [names[k] for k in range(4) if p[5 + k].lower() == "active"]))
            except ValueError:
                continue

    def mark(self, t_start: float, t_end: float) -> None:
        """Host-clock bounds of the timed region; samples outside are ignored
        (plus one sample after the end, which covers its last interval)."""
        self.window = (t_start, t_end)

    def __exit__(self, *exc):
        self.stop = True
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = list(self.rows)
        if self.window is not None:
            t0, t1 = self.window
            rows = [r for r in rows if t0 <= r[0] <= t1] + [r for r in rows if r[0] > t1][:1]
        if not rows:
            return None
        reasons = sorted({n for r in rows for n in r[3]})
        return {"sm_mhz": statistics.median(r[1] for r in rows), "sm_max_mhz": max(r[2] for r in rows),
                "sm_mhz_min": min(r[1] for r in rows), "reasons": reasons, "samples": len(rows),
                "source": self.source}


# ----------------------------------------------------------------------------
# oracle timing (CPU baseline and the reference arm)
# ----------------------------------------------------------------------------
def oracle_sample_rows(P, step: int, target_nnz: int):
    """Every stride-th row starting at `step % stride`: a bounded, stratified
    sample over the whole matrix (heavy rows at the top included in turn)."""
    stride = max(1, int(round(P.nnz / max(target_nnz, 1))))
    rows = np.arange(step % stride, P.M, stride, dtype=np.int64)
    nnz = int(np.diff(P.rowptr.astype(np.int64))[rows].sum())
    return rows, nnz, stride


def time_oracle_step(P, rows, keep=False):
    """Seconds of one oracle SDDMM + SpMM over `rows`; with keep, also its
    outputs (the SDDMM values, NaN outside the rows, and the SpMM rows)."""
    import oracle
    t0 = time.perf_counter()
    o = oracle.sddmm(P.rowptr, P.colidx, P.A, P.B, P.vals, rows=rows)
    c = oracle.spmm(P.rowptr, P.colidx, P.B, P.vals, rows=rows)
    t = time.perf_counter() - t0
    return (t, o, c) if keep else t


def comp_err(got, ref, den) -> float:
    """Componentwise error |got - ref| / (sum of the magnitudes of the terms);
    outputs with a zero denominator must match exactly (inf otherwise)."""
    got = np.asarray(got, np.float64)
    d = np.abs(got - ref)
    zero = den == 0
    if np.any(zero) and np.any(d[zero] != 0):
        return float("inf")
    return float(np.max(np.where(zero, 0.0, d / np.where(zero, 1.0, den)), initial=0.0))


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle_step_threads(P, rows, threads: int):
    """The same oracle calls on `threads` host threads, each on an interleaved
    share of the rows (the oracle's C routines run without the interpreter
    lock, so the shares run in parallel; each call still allocates and fills
    its own nnz-long SDDMM output, as the oracle does)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    shares = [rows[t::threads] for t in range(threads)]

    def run(share):
        oracle.sddmm(P.rowptr, P.colidx, P.A, P.B, P.vals, rows=share)
        oracle.spmm(P.rowptr, P.colidx, P.B, P.vals, rows=share)

    oracle.lib()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        t0 = time.perf_counter()
        list(ex.map(run, shares))
        return time.perf_counter() - t0


def reference_arm_batch(args):
    """Reference arm of the batched workload: the oracle on a bounded sample
    (every 16th matrix from an offset that moves each step, about 2000 rows
    of each), one host core."""
    import oracle
    oracle.build()
    probs = synth.batch(seed=0)
    for p in probs:                 # FP64 values for the oracle (exact from FP32), converted once, untimed
        if p.vals is not None:
            p.vals = p.vals.astype(np.float64)
    times, flops = [], []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        fl = 0.0
        for p in probs[s % 16::16]:
            rows = np.arange(0, p.M, max(1, p.M // 2000), dtype=np.int64)
            nz = int(np.diff(p.rowptr.astype(np.int64))[rows].sum())
            oracle.sddmm(p.rowptr, p.colidx, p.A, p.B, p.vals, rows=rows)
            oracle.spmm(p.rowptr, p.colidx, p.B, p.vals, rows=rows)
            fl += 4.0 * nz * p.K
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
            flops.append(fl)
    T = sum(times)
    value = sum(flops) / T / 1e9
    sample = "per step: every 16th matrix (offset = step mod 16), about 2000 evenly spaced rows each, FP64 oracle, single thread"
    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * T / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": BATCH_DESC}, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload == "batch":
        return reference_arm_batch(args)
    # the relabelling and dense-tile workloads compute the rmat20 step and a
    # plain SDDMM: the oracle's reference for them is that of rmat20
    P, desc = load_workload("rmat20" if args.workload in ("reorder", "blocks") else args.workload)
    import oracle
    oracle.build()
    if P.vals is not None:          # the oracle takes values in FP64 (exact from FP32): convert once, untimed
        P.vals = P.vals.astype(np.float64)
    target = args.ref_nnz
    times, flops = [], []
    for s in range(args.warmup + args.steps):
        rows, nnz, stride = oracle_sample_rows(P, s, target)
        t = time_oracle_step(P, rows)
        if s >= args.warmup:
            times.append(t)
            flops.append(2.0 * 2.0 * nnz * P.K)
    T = sum(times)
    value = sum(flops) / T / 1e9
    sample = (f"per step: rows i = s mod {stride} (every {stride}-th row, ~{target:,} of {P.nnz:,} nonzeros), "
              f"SDDMM + SpMM in the FP64 oracle, single thread")
    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * T / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "M": P.M, "N": P.N, "K": P.K, "nnz": P.nnz},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# replicas: every rank times its own copy of the step; the job's time is the
# slowest rank's
# ----------------------------------------------------------------------------
def max_over_ranks(x: float, device) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def event_ms(fn, stream, flush, reps=5):
    """Median CUDA-event time of fn on `stream`, L2 flushed before each rep."""
    import torch
    fn()
    fn()
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def aux_measurements(spk, S, P, A32, A, B, dt, elt, flush, stream, args):
    """The other steps of the path on the same pattern, outside the timed step:
    setup (schedule, transpose plan; wall clock, includes their host work),
    S^T Y through the plan, and the precision conversions."""
    import torch
    dev = A32.device

    def wall_ms(fn, reps=3):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize(dev)
            ts.append(1e3 * (time.perf_counter() - t0))
        return statistics.median(ts)

    S2 = spk.CSR(P.rowptr, P.colidx, (P.M, P.N), device=dev, schedule=False)
    out = {"schedule_build_ms": wall_ms(lambda: S2.build_schedule(args.chunk_work)),
           "transpose_plan_build_ms": wall_ms(lambda: spk.TransposePlan(S, args.chunk_work))}
    del S2
    plan = S.transpose_plan(args.chunk_work)
    X = torch.empty((P.N, P.K), dtype=torch.float32, device=dev)
    t = event_ms(lambda: spk.spmm_t(S, A, out=X, plan=plan), stream, flush)
    # colptr, CSC rows, COO rows of S^T, slot permutation, permuted values; Y once, X written once
    bytes_t = 4 * (P.N + 1) + 16 * P.nnz + P.M * P.K * elt + P.N * P.K * 4
    out["spmm_t_ms"] = t
    out["spmm_t_algo_gbs"] = bytes_t / (t / 1e3) / 1e9
    n = A32.numel()
    t = event_ms(lambda: spk.cast(A32, torch.bfloat16), stream, flush)
    out["cast_bf16_ms"] = t
    out["cast_bf16_algo_gbs"] = 6 * n / (t / 1e3) / 1e9
    t = event_ms(lambda: spk.quantize_e4m3_rows(A32), stream, flush)
    out["quantize_e4m3_ms"] = t
    out["quantize_e4m3_algo_gbs"] = (5 * n + 4 * A32.size(0)) / (t / 1e3) / 1e9
    # the GNN-layer cascade: scores e = SDDMM(S, A, B) become the values of SpMM(S_e, B)
    Bd = B
    e_buf = torch.empty(P.nnz, dtype=torch.float32, device=dev)
    Yl = torch.empty((P.M, P.K), dtype=torch.float32, device=dev)

    def layer_separate():
        spk.sddmm(S, A, Bd, out=e_buf)
        spk.spmm(S, Bd, e_buf, out=Yl)
    out["layer_separate_ms"] = event_ms(layer_separate, stream, flush)
    fb = 4 * (P.M + 1) + 12 * P.nnz + P.M * P.K * elt + P.N * P.K * elt + P.M * P.K * 4
    for name, kw in (("fusedmm_ms", {}), ("fusedmm_softmax_ms", {"softmax": True}),
                     ("fusedmm_softmax_4heads_ms", {"softmax": True, "heads": 4})):
        if P.K % (4 * (16 // elt)) and "heads" in kw:
            continue
        t = event_ms(lambda: spk.fusedmm(S, A, Bd, out=Yl, **kw), stream, flush)
        out[name] = t
        out[name.replace("_ms", "_algo_gbs")] = fb / (t / 1e3) / 1e9
    if "fusedmm_softmax_4heads_ms" in out:
        # forward + backward of the differentiable layer (dA and dB, 4 heads, softmax)
        Ag = A.detach().clone().requires_grad_()
        Bg = Bd.detach().clone().requires_grad_()
        dY = torch.ones((P.M, P.K), dtype=torch.float32, device=dev)

        def fwd_bwd():
            Ag.grad = None
            Bg.grad = None
            spk.autograd.fusedmm(S, Ag, Bg, S.vals, heads=4, softmax=True).backward(dY)
        out["fusedmm_softmax_4heads_fwd_bwd_ms"] = event_ms(fwd_bwd, stream, flush)
        del Ag, Bg, dY
    if P.M == P.N:
        # the attention-style graph layer Y = SpMM(S_e, H), e = SDDMM(S, H, H),
        # differentiated: forward, then dH through SDDMM, SpMM and two SpMM^T
        try:
            Hg = A.detach().clone().requires_grad_()
            dYl = torch.ones((P.M, P.K), dtype=torch.float32, device=dev)

            def gnn_fwd_bwd():
                Hg.grad = None
                spk.autograd.gnn_layer(S, Hg).backward(dYl)
            out["gnn_layer_fwd_bwd_ms"] = event_ms(gnn_fwd_bwd, stream, flush)
            del Hg, dYl
        except Exception as exc:                    # keep the line if this extra figure fails
            out["gnn_layer_fwd_bwd_error"] = str(exc)[:200]
    out["note"] = ("measured after the timed step on the same pattern; builds by wall clock, kernels by CUDA "
                   "events with the L2 flushed; layer_separate = SDDMM then SpMM on its scores, fusedmm = the "
                   "same layer in one kernel; fwd_bwd = that layer differentiated (forward, then dA and dB); "
                   "gnn_layer_fwd_bwd = the separate-kernel layer with H as both factors, forward then dH")
    return out



def other_workloads(spk, dev, flush, stream, pk, args):
    """SDDMM and SpMM of the other power-law configurations, timed like the
    line's step (CUDA events on the launching stream, L2 flushed before each
    launch): rec (2M x 500K, 50M nnz, K = 128) with FP32 and BF16 factors, and
    gnn (R-MAT scale 22, K = 64) with BF16 H as both factors."""
    import torch
    out = {}
    for name, dtypes in (("rec", ("f32", "bf16")), ("gnn", ("bf16",))):
        t0 = time.perf_counter()
        P, desc = load_workload(name)
        gen_s = time.perf_counter() - t0
        vals = None if P.vals is None else torch.from_numpy(P.vals).to(dev)
        S = spk.CSR(P.rowptr, P.colidx, (P.M, P.N), vals, device=dev, chunk_work=args.chunk_work)
        A32 = torch.from_numpy(P.A).to(dev)
        B32 = A32 if P.B is P.A else torch.from_numpy(P.B).to(dev)
        res = {"workload": desc, "M": P.M, "N": P.N, "K": P.K, "nnz": P.nnz, "generation_s": round(gen_s, 1)}
        o = torch.empty(P.nnz, dtype=torch.float32, device=dev)
        C = torch.empty((P.M, P.K), dtype=torch.float32, device=dev)
        for dt in dtypes:
            if dt == "f32":
                A, B, elt = A32, B32, 4
            else:
                A = spk.cast(A32, torch.bfloat16)
                B = A if P.B is P.A else spk.cast(B32, torch.bfloat16)
                elt = 2
            sd = event_ms(lambda: spk.sddmm(S, A, B, out=o), stream, flush, reps=10)
            sp = event_ms(lambda: spk.spmm(S, B, out=C), stream, flush, reps=10)
            ab = algorithmic_bytes(P, elt)
            res[dt] = {"sddmm_ms": sd, "spmm_ms": sp,
                       "sddmm_gflops": 2.0 * P.nnz * P.K / (sd / 1e3) / 1e9,
                       "spmm_gflops": 2.0 * P.nnz * P.K / (sp / 1e3) / 1e9,
                       "sddmm_algo_gbs": ab["sddmm"] / (sd / 1e3) / 1e9,
                       "spmm_algo_gbs": ab["spmm"] / (sp / 1e3) / 1e9,
                       "sddmm_frac": ab["sddmm"] / (sd / 1e3) / 1e9 / pk["hbm_gbs"],
                       "spmm_frac": ab["spmm"] / (sp / 1e3) / 1e9 / pk["hbm_gbs"]}
            del A, B
        out[name] = res
        del S, A32, B32, o, C, vals, P
        torch.cuda.empty_cache()
    out["note"] = ("median of 10 CUDA-event timings per kernel, L2 flushed before each; algorithmic bytes as for "
                   "the line's roofline (factors once, indices, values, outputs); frac of the measured copy peak")
    return out


def main(args):
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "batch":
        return main_batch(args)
    if args.workload == "reorder":
        return main_reorder(args)
    if args.workload == "blocks":
        return main_blocks(args)

    import torch
    import torch.distributed as dist
    import paper_2404_19638_gb300 as spk

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", torch.cuda.current_device())

    P, desc = load_workload(args.workload)
    K = P.K
    dt = torch.float32 if args.dtype == "f32" else torch.bfloat16
    elt = 4 if args.dtype == "f32" else 2
    vals = None if P.vals is None else torch.from_numpy(P.vals).to(dev)
    S = spk.CSR(P.rowptr, P.colidx, (P.M, P.N), vals, device=dev, chunk_work=args.chunk_work)
    A32 = torch.from_numpy(P.A).to(dev)
    B32 = A32 if P.B is P.A else torch.from_numpy(P.B).to(dev)
    A = A32 if dt == torch.float32 else spk.cast(A32, dt)
    B = B32 if dt == torch.float32 else (A if P.B is P.A else spk.cast(B32, dt))
    out = torch.empty(P.nnz, dtype=torch.float32, device=dev)
    C = torch.empty((P.M, K), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)      # > 129 MB L2
    tune_sd = json.loads(args.tune_sddmm) if args.tune_sddmm else None
    tune_sp = json.loads(args.tune_spmm) if args.tune_spmm else None
    stream = torch.cuda.current_stream(dev)

    def step():
        spk.sddmm(S, A, B, out=out, tune=tune_sd)
        ev[1].record(stream)
        spk.spmm(S, B, out=C, tune=tune_sp)

    for _ in range(args.warmup):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        step()
    torch.cuda.synchronize(dev)

    events = []
    with ClockSampler(dev.index if world == 1 else local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            step()
            ev[2].record(stream)
            events.append(ev)
        torch.cuda.synchronize(dev)
        clk.mark(wall0, time.perf_counter())
        time.sleep(0.05)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    clocks = clk.summary()
    t_sd = [e[0].elapsed_time(e[1]) for e in events]
    t_sp = [e[1].elapsed_time(e[2]) for e in events]

    # the same step with BF16 factors (RNE casts of the same A, B, made once,
    # untimed), FP32 accumulation and outputs: the precision comparison
    bf = None
    if dt == torch.float32 and not args.no_bf16:
        Ab = spk.cast(A32, torch.bfloat16)
        Bb = Ab if P.B is P.A else spk.cast(B32, torch.bfloat16)
        out_b = torch.empty_like(out)
        C_b = torch.empty_like(C)

        def step_b():
            spk.sddmm(S, Ab, Bb, out=out_b)
            evb[1].record(stream)
            spk.spmm(S, Bb, out=C_b)

        for _ in range(args.warmup):
            flush.zero_()
            evb = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            step_b()
        torch.cuda.synchronize(dev)
        events_b = []
        with ClockSampler(dev.index if world == 1 else local) as clk_b:
            torch.cuda.synchronize(dev)
            w0 = time.perf_counter()
            for _ in range(args.steps):
                flush.zero_()
                evb = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                evb[0].record(stream)
                step_b()
                evb[2].record(stream)
                events_b.append(evb)
            torch.cuda.synchronize(dev)
            clk_b.mark(w0, time.perf_counter())
            time.sleep(0.05)
        tb_sd = [e[0].elapsed_time(e[1]) for e in events_b]
        tb_sp = [e[1].elapsed_time(e[2]) for e in events_b]
        Tb = max_over_ranks((sum(tb_sd) + sum(tb_sp)) / 1e3, dev)
        bf = {"t_sd": tb_sd, "t_sp": tb_sp, "T": Tb, "clocks": clk_b.summary(), "out": out_b, "C": C_b}
    T = (sum(t_sd) + sum(t_sp)) / 1e3                      # seconds, this rank
    T = max_over_ranks(T, dev)
    flops_step = 2.0 * 2.0 * P.nnz * K
    value = world * flops_step * args.steps / T / 1e9

    # end to end through the public API: every step copies its inputs in from
    # pinned host memory and its results back out.  Steps are pipelined over
    # three streams (inputs of step s+1 travel in while step s computes and
    # the results of step s-1 travel out), with two device buffer sets.
    hA = torch.from_numpy(P.A).pin_memory()
    hB = hA if P.B is P.A else torch.from_numpy(P.B).pin_memory()
    hv = None if P.vals is None else torch.from_numpy(P.vals).pin_memory()
    hout = torch.empty(P.nnz, dtype=torch.float32).pin_memory()
    hC = torch.empty((P.M, K), dtype=torch.float32).pin_memory()
    sets = []
    for _ in range(2):
        dA_ = torch.empty_like(A32)
        dB_ = dA_ if P.B is P.A else torch.empty_like(B32)
        dv_ = None if hv is None else torch.empty_like(vals)
        sets.append((dA_, dB_, dv_, torch.empty_like(out), torch.empty_like(C)))
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_comp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    started = [False, False]

    def e2e_step(k):
        dA_, dB_, dv_, o_, C_ = sets[k % 2]
        with torch.cuda.stream(s_in):
            if started[k % 2]:
                s_in.wait_event(ev_comp[k % 2])          # step k-2 has read this set
            dA_.copy_(hA, non_blocking=True)
            if dB_ is not dA_:
                dB_.copy_(hB, non_blocking=True)
            if dv_ is not None:
                dv_.copy_(hv, non_blocking=True)
            ev_in[k % 2].record(s_in)
        stream.wait_event(ev_in[k % 2])
        if started[k % 2]:
            stream.wait_event(ev_out[k % 2])             # step k-2's results are out
        a = dA_ if dt == torch.float32 else spk.cast(dA_, dt)
        b = dB_ if dt == torch.float32 else (a if dB_ is dA_ else spk.cast(dB_, dt))
        spk.sddmm(S, a, b, dv_, out=o_, tune=tune_sd)
        spk.spmm(S, b, dv_, out=C_, tune=tune_sp)
        ev_comp[k % 2].record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_comp[k % 2])
            hout.copy_(o_, non_blocking=True)
            hC.copy_(C_, non_blocking=True)
            ev_out[k % 2].record(s_out)
        started[k % 2] = True

    for k in range(2):
        e2e_step(k)
    torch.cuda.synchronize(dev)
    e2e_steps = max(4, args.steps // 2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    for k in range(e2e_steps):
        e2e_step(k)
    s_out.wait_stream(stream)
    e1.record(s_out)
    torch.cuda.synchronize(dev)
    Te = e0.elapsed_time(e1) / 1e3
    Te = max_over_ranks(Te, dev)
    h2d = (hA.numel() * 4 + (0 if hB is hA else hB.numel() * 4) + (0 if hv is None else hv.numel() * 4))
    d2h = hout.numel() * 4 + hC.numel() * 4

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    aux = None if args.no_aux else aux_measurements(spk, S, P, A32, A, B, dt, elt, flush, stream, args)

    pk, pk_kind = peaks()
    ab = algorithmic_bytes(P, elt)
    ms_sd, ms_sp = statistics.mean(t_sd), statistics.mean(t_sp)
    dom = "sddmm" if ms_sd >= ms_sp else "spmm"
    ms_dom = ms_sd if dom == "sddmm" else ms_sp
    achieved = ab[dom] / (ms_dom / 1e3) / 1e9
    traffic = profiled_traffic(args.workload, args.dtype)
    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": desc, "M": P.M, "N": P.N, "K": K, "nnz": P.nnz, "op": "SDDMM then SpMM",
                   "l2": "flushed between steps (256 MB write outside the timed events)",
                   "chunk_work": args.chunk_work, "parallelism": "replicas" if world > 1 else "single GPU"},
        "kernels": {"sddmm_ms": ms_sd, "spmm_ms": ms_sp,
                    "sddmm_gflops": 2.0 * P.nnz * K / (ms_sd / 1e3) / 1e9,
                    "spmm_gflops": 2.0 * P.nnz * K / (ms_sp / 1e3) / 1e9,
                    "sddmm_algo_gbs": ab["sddmm"] / (ms_sd / 1e3) / 1e9,
                    "spmm_algo_gbs": ab["spmm"] / (ms_sp / 1e3) / 1e9},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "peak_kind": pk_kind,
                     "algorithmic_bytes": ab[dom],
                     "traffic": None if traffic is None else traffic.get(dom)},
        "e2e": {"value": world * flops_step * e2e_steps / Te / 1e9, "unit": "GFLOP/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": 2 * args.steps,
        "wall_s": wall,
    }
    if args.warmup != args.warmup_requested:
        line["config"]["warmup_note"] = f"--warmup {args.warmup_requested} raised to {args.warmup} (at least 3)"
    if bf is not None:
        ab16 = algorithmic_bytes(P, 2)
        bsd, bsp = statistics.mean(bf["t_sd"]), statistics.mean(bf["t_sp"])
        line["kernels_bf16"] = {
            "step_ms": 1e3 * bf["T"] / args.steps, "value": world * flops_step * args.steps / bf["T"] / 1e9,
            "sddmm_ms": bsd, "spmm_ms": bsp,
            "sddmm_gflops": 2.0 * P.nnz * K / (bsd / 1e3) / 1e9, "spmm_gflops": 2.0 * P.nnz * K / (bsp / 1e3) / 1e9,
            "sddmm_algo_gbs": ab16["sddmm"] / (bsd / 1e3) / 1e9, "spmm_algo_gbs": ab16["spmm"] / (bsp / 1e3) / 1e9,
            "clocks": bf["clocks"],
            "note": "A, B cast to BF16 (round to nearest even) once, untimed; FP32 accumulation and outputs; "
                    "same pattern, values, steps and L2 flushes as the FP32 line"}
        line["bf16_over_f32"] = {"step": (T / args.steps) / (bf["T"] / args.steps), "sddmm": ms_sd / bsd,
                                 "spmm": ms_sp / bsp, "note": "FP32 time / BF16 time (> 1: BF16 faster)"}
    if aux is not None:
        line["aux"] = aux
    line["clocks"] = clocks
    if world == 1 and not args.no_extra and args.workload == "rmat20":
        try:
            line["other_workloads"] = other_workloads(spk, dev, flush, stream, pk, args)
        except Exception as exc:                    # keep the line if this extra measurement fails
            line["other_workloads"] = {"error": str(exc)[:200]}
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        if P.vals is not None:      # FP64 values for the oracle (exact from FP32), converted once, untimed
            P.vals = P.vals.astype(np.float64)
        rows, nnz, stride = oracle_sample_rows(P, 0, args.cpu_nnz)
        t, o_ref, c_ref = time_oracle_step(P, rows, keep=True)
        cores = min(host_cores(), 64)               # each thread holds an nnz-long output while it runs
        tc = time_oracle_step_threads(P, rows, cores) if cores > 1 else t
        line["cpu_baseline"] = {"value": 2.0 * 2.0 * nnz * K / tc / 1e9, "unit": "GFLOP/s", "cores": cores,
                                "kind": "oracle",
                                "single_core_value": 2.0 * 2.0 * nnz * K / t / 1e9,
                                "sample": (("all rows" if stride == 1 else f"every {stride}-th row")
                                           + f" ({nnz:,} of {P.nnz:,} nonzeros), SDDMM + SpMM in the FP64 "
                                           f"oracle: {t:.1f} s on one host core, {tc:.2f} s on {cores} host "
                                           "threads (rows interleaved over the threads)")}
        # what the timed oracle outputs say about the GPU's: componentwise
        # error of the FP32 and BF16 steps against the FP64 oracle on the
        # original FP32 inputs, on every 16th row of the sample (the
        # denominators, sums of term magnitudes, come from the oracle too)
        import oracle
        er = rows[::16]
        ent = np.concatenate([np.arange(P.rowptr[r], P.rowptr[r + 1]) for r in er]).astype(np.int64)
        o_den = oracle.sddmm(P.rowptr, P.colidx, P.A, P.B, P.vals, rows=er, absmode=True)[ent]
        c_den = oracle.spmm(P.rowptr, P.colidx, P.B, P.vals, rows=er, absmode=True)
        pos = np.searchsorted(rows, er)
        par = {"rows": int(er.size), "nonzeros": int(ent.size),
               "metric": "max |gpu - oracle| / sum of |terms| (oracle in FP64 on the FP32 inputs)",
               "gates": {"f32": 1e-5, "bf16": 2e-2},
               "f32": {"sddmm": comp_err(out.cpu().numpy()[ent], o_ref[ent], o_den),
                       "spmm": comp_err(C.cpu().numpy()[er], c_ref[pos], c_den)}}
        if bf is not None:
            par["bf16"] = {"sddmm": comp_err(bf["out"].cpu().numpy()[ent], o_ref[ent], o_den),
                           "spmm": comp_err(bf["C"].cpu().numpy()[er], c_ref[pos], c_den)}
        line["cpu_baseline"]["parity"] = par
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


BATCH_DESC = ("batch: 256 independent matrices, n log-uniform in [1e3, 2e5] (9,570,975 rows, 147,971,228 nonzeros); "
              "128 Erdos-Renyi with exactly d ~ U{4..32} columns per row, 128 R-MAT edge factor 16; K ~ U{16,32,64}; "
              "values, A, B U[-1,1]; every matrix runs SDDMM and SpMM")


def main_batch(args):
    """The batched work list: SDDMM and SpMM of all 256 matrices (512 work
    items) in one persistent launch, replayed from a CUDA graph each step."""
    import torch
    import torch.distributed as dist
    import paper_2404_19638_gb300 as spk

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", torch.cuda.current_device())
    dt = torch.float32 if args.dtype == "f32" else torch.bfloat16
    elt = 4 if args.dtype == "f32" else 2
    probs = synth.batch(seed=0)
    items, keep = [], []
    flops_step, algo = 0.0, 0
    h2d = d2h = 0
    for p in probs:
        S = spk.CSR(p.rowptr, p.colidx, (p.M, p.N), torch.from_numpy(p.vals), device=dev, chunk_work=args.chunk_work)
        A = torch.from_numpy(p.A).to(dev).to(dt)
        B = torch.from_numpy(p.B).to(dev).to(dt)
        out = torch.empty(p.nnz, dtype=torch.float32, device=dev)
        C = torch.empty((p.M, p.K), dtype=torch.float32, device=dev)
        items.append(spk.Item(spk.OP_SDDMM, S, B, out, A=A))
        items.append(spk.Item(spk.OP_SPMM, S, B, C))
        keep.append((S, A, B, out, C, p))
        flops_step += 2.0 * 2.0 * p.nnz * p.K
        ab = algorithmic_bytes(p, elt)
        algo += ab["sddmm"] + ab["spmm"]
        h2d += p.A.nbytes + p.B.nbytes + p.vals.nbytes
        d2h += out.numel() * 4 + C.numel() * 4
    batch = spk.Batch(items)
    t0 = time.perf_counter()
    tuned = batch.autotune((64, 128, 256, 512), per_item=True)     # schedules, shapes, registers, by timing
    tune_s = time.perf_counter() - t0
    batch.capture()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        flush.zero_()
        batch.replay()
    torch.cuda.synchronize(dev)
    events = []
    with ClockSampler(dev.index if world == 1 else local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch.replay()
            e1.record(stream)
            events.append((e0, e1))
        torch.cuda.synchronize(dev)
        clk.mark(wall0, time.perf_counter())
        time.sleep(0.15)
    if world > 1:
        dist.barrier()
    T = sum(a.elapsed_time(b) for a, b in events) / 1e3
    T = max_over_ranks(T, dev)
    ms = 1e3 * T / args.steps

    # the same work as one launch per (matrix, op), for comparison
    def per_matrix():
        for S, A, B, out, C, p in keep:
            spk.sddmm(S, A, B, out=out)
            spk.spmm(S, B, out=C)
    per_ms = event_ms(per_matrix, stream, flush, reps=3)

    # end to end: inputs from pinned host memory, outputs back, one persistent launch
    hosts = [(torch.from_numpy(p.A).pin_memory(), torch.from_numpy(p.B).pin_memory(),
              torch.from_numpy(p.vals).pin_memory(), torch.empty(p.nnz).pin_memory(),
              torch.empty((p.M, p.K)).pin_memory()) for (_, _, _, _, _, p) in keep]
    stage = [(torch.empty(p.A.shape, device=dev), torch.empty(p.B.shape, device=dev)) for (_, _, _, _, _, p) in keep]

    def e2e_step():
        for (S, A, B, out, C, p), (hA, hB, hv, ho, hC), (sA, sB) in zip(keep, hosts, stage):
            if dt == torch.float32:
                A.copy_(hA, non_blocking=True)
                B.copy_(hB, non_blocking=True)
            else:
                sA.copy_(hA, non_blocking=True)
                sB.copy_(hB, non_blocking=True)
                A.copy_(spk.cast(sA, dt))
                B.copy_(spk.cast(sB, dt))
            S.vals.copy_(hv, non_blocking=True)
        batch.replay()
        for (S, A, B, out, C, p), (hA, hB, hv, ho, hC), _ in zip(keep, hosts, stage):
            ho.copy_(out, non_blocking=True)
            hC.copy_(C, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize(dev)
    e2e_steps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    Te = e0.elapsed_time(e1) / 1e3
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    pk, pk_kind = peaks()
    achieved = algo / (ms / 1e3) / 1e9
    info = batch.info()
    line = {
        "metric": METRIC, "value": world * flops_step * args.steps / T / 1e9, "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": BATCH_DESC, "matrices": len(keep), "work_items": len(items),
                   "nnz": int(sum(p.nnz for *_, p in keep)), "rows": int(sum(p.M for *_, p in keep)),
                   "l2": "flushed between steps (256 MB write outside the timed events)",
                   "launch": "one persistent kernel per step, replayed from a CUDA graph",
                   "chunk_work": tuned["chunk_work"],
                   "autotune_ms": {str(k): round(v, 4) for k, v in tuned["ms"].items()},
                   "autotune": {"chunk_work_by_nnz": tuned["chunk_work_by_nnz"],
                                "shapes": {k: v for k, v in tuned["shapes"].items()},
                                "registers": tuned["registers"], "ms_final": round(tuned["ms_final"], 4),
                                "trials": tuned["trials"], "seconds": round(tune_s, 1),
                                "note": "per-item choices by whole-launch timing; shape null = default by K"},
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "kernels": {"batch_ms": ms, "per_matrix_launches_ms": per_ms, "per_matrix_launches": 2 * len(keep),
                    "work_units": info["work_units"], "ctas": info["ctas"],
                    # tuning (4 chunk sizes + trials, reps 3 + 1 each), graph capture's warm-up run, warm-up replays
                    "k_batch_launches_before_timed": 4 * 4 + 4 * tuned["trials"] + 1 + args.warmup},
        "roofline": {"bound": "hbm", "kernel": "batch", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "peak_kind": pk_kind, "algorithmic_bytes": algo,
                     "traffic": None},
        "e2e": {"value": world * flops_step * e2e_steps / Te / 1e9, "unit": "GFLOP/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
    }
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        for *_, p in keep[::2]:        # FP64 values for the oracle (exact from FP32), converted once, untimed
            if p.vals is not None:
                p.vals = p.vals.astype(np.float64)
        t0 = time.perf_counter()
        fl = 0.0
        used = 0
        for S, A, B, out, C, p in keep[::2]:
            rows = np.arange(0, p.M, 2, dtype=np.int64)
            nz = int(np.diff(p.rowptr.astype(np.int64))[rows].sum())
            oracle.sddmm(p.rowptr, p.colidx, p.A, p.B, p.vals, rows=rows)
            oracle.spmm(p.rowptr, p.colidx, p.B, p.vals, rows=rows)
            fl += 4.0 * nz * p.K
            used += 1
        t = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": fl / t / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                                "sample": f"every 2nd matrix ({used}), every 2nd row of each, "
                                          f"SDDMM + SpMM in the FP64 oracle on one host core, {t:.1f} s"}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


REORDER_DESC = {
    "rmat20": ("reorder: rmat20 (R-MAT scale 20, edge factor 16, values U[-1,1], A, B 2^20 x 64 N(0,1) FP32) "
               "with its rows relabelled ({orders}) vs the original order"),
    "gnn": ("reorder: gnn (R-MAT scale 22, edge factor 8, unit values, A = B = H 2^22 x 64 N(0,0.1) in BF16) "
            "with its rows relabelled ({orders}) vs the original order"),
}
BLOCKS_DESC = ("blocks: 131,072 x 131,072, 1500 fully dense 128 x 64 blocks at aligned positions over 2 uniform "
               "columns per row, values U[-1,1]; A, B N(0,1) in BF16")


def _single_gpu_line(args, metric_value, ms, desc, extra, dtype):
    import torch
    return {"metric": METRIC, "value": metric_value, "unit": "GFLOP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": desc, "l2": "flushed before every timed launch (256 MB write)",
                       "parallelism": "single GPU"}, **extra}


def main_reorder(args):
    """Step time of rmat20 (FP32) or gnn (BF16) in each row order (the
    relabelled pattern keeps the original column ids; A is gathered into the
    new row order once).  Per order: SDDMM 1 + reps launches, then SpMM
    1 + reps, original order first."""
    import torch
    import paper_2404_19638_gb300 as spk
    dev = torch.device("cuda", torch.cuda.current_device())
    P, _ = load_workload(args.reorder_pattern)
    vals = None if P.vals is None else torch.from_numpy(P.vals).to(dev)
    S = spk.CSR(P.rowptr, P.colidx, (P.M, P.N), vals, device=dev)
    dt = torch.float32 if args.reorder_pattern == "rmat20" else torch.bfloat16
    A32 = torch.from_numpy(P.A).to(dev)
    A = A32 if dt == torch.float32 else spk.cast(A32, dt)
    B = A if P.B is P.A else (torch.from_numpy(P.B).to(dev) if dt == torch.float32
                              else spk.cast(torch.from_numpy(P.B).to(dev), dt))
    del A32
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    reps = max(args.steps, 5)
    orders = [o for o in args.orders.split(",") if o]
    res = {"original": {"sddmm_ms": event_ms(lambda: spk.sddmm(S, A, B), stream, flush, reps),
                        "spmm_ms": event_ms(lambda: spk.spmm(S, B), stream, flush, reps)}}
    for order in orders:
        t0 = time.perf_counter()
        R = spk.Reordering(S, order)
        torch.cuda.synchronize(dev)
        build = time.perf_counter() - t0
        Ar = R.gather_rows(A)
        res[order] = {"plan_build_s": build, "sddmm_ms": event_ms(lambda: spk.sddmm(R.S, Ar, B), stream, flush, reps),
                      "spmm_ms": event_ms(lambda: spk.spmm(R.S, B), stream, flush, reps),
                      "gather_rows_ms": event_ms(lambda: R.gather_rows(A), stream, flush, reps)}
        if vals is not None:
            res[order]["scatter_values_ms"] = event_ms(lambda: R.scatter_values(vals), stream, flush, reps)
        del R, Ar
    best = min(orders, key=lambda o: res[o]["sddmm_ms"] + res[o]["spmm_ms"])
    ms = res[best]["sddmm_ms"] + res[best]["spmm_ms"]
    desc = REORDER_DESC[args.reorder_pattern].format(orders=", ".join(orders))
    line = _single_gpu_line(args, 2.0 * 2.0 * P.nnz * P.K / (ms / 1e3) / 1e9, ms, desc,
                            {"reorder": res, "best_order": best, "gpu_launches": 2 * reps},
                            "f32" if dt == torch.float32 else "bf16")
    print(json.dumps(line), flush=True)
    return 0


def main_blocks(args):
    """SDDMM of a pattern with dense blocks: the tensor-core tiles plus the
    gather kernels on the rest, against the gather kernels on everything."""
    import torch
    import paper_2404_19638_gb300 as spk
    dev = torch.device("cuda", torch.cuda.current_device())
    n = 1 << 17
    rp, ci = synth.dense_blocks(n, n, 1500, 1.0, 2, seed=3)
    vals = torch.from_numpy(synth.uniform(ci.size, -1.0, 1.0, 3, 9)).to(dev)
    S = spk.CSR(rp, ci, (n, n), vals, device=dev)
    t0 = time.perf_counter()
    plan = spk.TensorCorePlan(S, 1024)
    torch.cuda.synchronize(dev)
    build = time.perf_counter() - t0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    reps = max(args.steps, 5)
    res = {"plan": plan.info(), "plan_build_s": build}
    for K in (64, 128, 256):
        A = torch.from_numpy(synth.normal((n, K), 1.0, 3, 2)).to(dev).to(torch.bfloat16)
        B = torch.from_numpy(synth.normal((n, K), 1.0, 3, 3)).to(dev).to(torch.bfloat16)
        g = event_ms(lambda: spk.sddmm(S, A, B), stream, flush, reps)
        t = event_ms(lambda: spk.tc_sddmm(plan, A, B), stream, flush, reps)
        res[f"K{K}"] = {"gather_sddmm_ms": g, "tc_sddmm_ms": t, "speedup": g / t,
                        "tc_gflops": 2.0 * ci.size * K / (t / 1e3) / 1e9}
    ms = res["K128"]["tc_sddmm_ms"]
    line = _single_gpu_line(args, res["K128"]["tc_gflops"], ms, BLOCKS_DESC,
                            {"tc": res, "op": "SDDMM (K = 128 for the value)", "gpu_launches": 3 * reps}, "bf16")
    print(json.dumps(line), flush=True)
    return 0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat20", choices=["rmat20", "tiny", "rec", "gnn", "batch", "reorder", "blocks"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16"])
    ap.add_argument("--chunk-work", type=int, default=None,
                    help="balanced-schedule chunk size (default 512; 128 for the batched workload)")
    ap.add_argument("--tune-sddmm", default=None, help='JSON spk_tune fields, e.g. {"group_lanes": 8}')
    ap.add_argument("--tune-spmm", default=None)
    ap.add_argument("--cpu-nnz", type=int, default=16_000_000,
                    help="nonzeros in the CPU-baseline sample (every k-th row; about 10 s of oracle work by default)")
    ap.add_argument("--ref-nnz", type=int, default=100_000, help="nonzeros per reference-arm step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-aux", action="store_true", help="skip the setup / SpMM^T / conversion measurements")
    ap.add_argument("--no-bf16", action="store_true", help="skip the BF16-factor timing of the FP32 line")
    ap.add_argument("--no-extra", action="store_true", help="skip the rec and gnn kernel timings")
    ap.add_argument("--reorder-pattern", default="rmat20", choices=["rmat20", "gnn"],
                    help="pattern of --workload reorder (rmat20 in FP32, gnn in BF16)")
    ap.add_argument("--orders", default="degree,leading,rcm", help="row orders of --workload reorder")
    a = ap.parse_args()
    a.warmup_requested = a.warmup
    if a.warmup < 3:                # the timing rules ask for at least 3 warm-up steps; the line says so
        print(f"bench.py: --warmup {a.warmup} raised to 3", file=sys.stderr)
        a.warmup = 3
    if a.chunk_work is None:
        # many small matrices with short rows: smaller chunks keep more warps busy
        a.chunk_work = 128 if a.workload == "batch" else 512
    return a


if __name__ == "__main__":
    sys.exit(main(parse()))
