#!/usr/bin/env python
"""Benchmark of the block-orthogonalization hot path on one GB300 (or N replicas).

Workload (one "step" = one pass of the whole path over one block):
  V: 4,000,000 x 64 FP64 orthonormal basis, Y: 4,000,000 x 16 FP64 with
  singular values log-spaced 1 .. 1e-10 (seeded, synthetic; see synth.py).
  step = eo_gram          (C = V^T Y, compensated; tcgen05 digit engine)
       + eo_project_apply (Y~ = Y - V C, compensated)
       + eo_gram          (M = Y~^T Y~, compensated; tcgen05 digit engine)
       + eo_cholqr        (compensated, first pass from M, automatic second pass).
The inputs (2.6 GB per step) are larger than L2 (129 MB), so no flush is
needed between steps.

Prints ONE JSON line.  `value` is algorithmic HBM bytes / device time (GB/s)
over all ranks; `e2e` is the same metric through the C-ABI with the inputs in
pinned host memory and the host<->device copies inside the timed region.
`--impl reference` times the binary128 CPU oracle on a bounded row sample of
the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gram/CholQR HBM GB/s and blocks/s at ||Q^TQ-I||<=1e-14, DD vs plain FP64; p50/p99"
WORKLOAD = ("projection plus orthogonalization: V {n:,}x{kv} orthonormal FP64, Y {n:,}x{k} FP64 (sigma 1..1/{kappa:g}); "
            "V^T Y, Y - V(V^T Y), DD-Gram CholQR")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["eo", "reference"], default="eo")
    ap.add_argument("--n", type=int, default=4_000_000)
    ap.add_argument("--kv", type=int, default=64)
    ap.add_argument("--k", type=int, default=16)
    ap.add_argument("--kappa", type=float, default=1e10)
    ap.add_argument("--cpu-rows", type=int, default=0, help="rows of the CPU-oracle sample (0 = auto)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="skip the runs of the other workloads that the default line summarises")
    ap.add_argument("--no-comparators", action="store_true",
                    help="skip the FP64, DD-EFT, same-accuracy and single-block comparisons (profiling runs)")
    ap.add_argument("--workload", choices=["project", "iterated", "batched", "serve", "sweep", "single", "update"],
                    default="project",
                    help="project: the default line; iterated: the iterated two-phase algorithm on the "
                         "runtime-figure shapes (n = 8e6 unless --n is given); batched: many SVQB blocks of "
                         "uneven n and k in one graph launch; serve: the request server under Poisson arrivals; "
                         "sweep: the Gram precision sweep (n = 32e6, k 1..64); single: one 100,000 x 8 CholQR; "
                         "update: the compensated update Q = X R^-1 alone (one CholQR pass, M given) for --ks")
    ap.add_argument("--ks", default="4,8,16,32", help="column counts of the update workload")
    ap.add_argument("--blocks", type=int, default=512, help="blocks of the batched workload")
    ap.add_argument("--clients", type=int, default=256, help="resident bases of the serving workload")
    ap.add_argument("--requests", type=int, default=2000, help="requests of the serving trace")
    ap.add_argument("--rate", type=float, default=2000.0, help="offered requests/s of the serving trace")
    ap.add_argument("--slots", type=int, default=16, help="concurrent slots of the server")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="device-memory budget of the server")
    ap.add_argument("--branches", type=int, default=0, help="graph branches of the batched workload (0 = auto)")
    return ap.parse_args()


class _Skip(Exception):
    """A comparison left out on request."""


def max_over_ranks(x, device):
    """Largest value of x over all ranks (x itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world_size, bytes_per_rank, max_ms):
    """Whole-job GB/s: every rank processed bytes_per_rank in at most max_ms."""
    return world_size * bytes_per_rank / (max_ms * 1e-3) / 1e9


def alu_peak_tflops(sm_mhz=2070.0, sms=152):
    """Peak of the compensated (EO_DD) engine in algorithmic TFLOP/s: 64
    integer multiply-add lanes per SM per clock, ten 32x32->64-bit limb
    products per exact multiply-add, two flops per multiply-add."""
    return 64 * sms * sm_mhz * 1e6 / 10 * 2 / 1e12


def step_bytes(n, kv, k, two_passes):
    """Algorithmic HBM bytes of one step: what the method must read and write.

    V^T Y reads V and Y; the fused pass reads V and Y and writes Y~; the first
    CholQR update reads and writes Y~; a second pass reads Q for its Gram
    matrix and reads and writes it in its update."""
    b = 8 * n * (kv + k) + 8 * n * (kv + 2 * k) + 16 * n * k
    if two_passes:
        b += 8 * n * k + 16 * n * k
    return b


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------ CPU oracle

def cpu_sample(v, y, rows, mode, passes=2):
    """Time one step of the oracle's CPU arithmetic (mode: oracle.DD = Dot2
    double-double, oracle.FP64 = plain) -- projection, Gram of the result,
    CholQR with `passes` passes -- on the first `rows` rows.  Returns
    (seconds, algorithmic bytes, Q, Cholesky info)."""
    import oracle
    vs = v[:rows] if v.flags.f_contiguous and rows == v.shape[0] else np.asfortranarray(v[:rows])
    ys = np.asfortranarray(y[:rows])
    t0 = time.perf_counter()
    yt, _, m = oracle.fp64_project(vs, ys, mode=mode)
    q, _, info = oracle.fp64_cholqr(yt, passes=passes, mode=mode, m=m)
    dt = time.perf_counter() - t0
    return dt, step_bytes(rows, v.shape[1], y.shape[1], passes == 2), q, info


def cpu_baseline(v, y, rows):
    """The paper's CPU arithmetic on the host's cores: the double-double
    (Dot2) step on all cores (the line's value), the plain FP64 CholQR2 step,
    and the double-double step on one core, each on the first `rows` rows of
    the same V and Y (0 = all rows)."""
    import oracle
    n = v.shape[0]
    rows = n if rows <= 0 else min(rows, n)
    cores = oracle.threads()
    dt, nbytes, q, info = cpu_sample(v, y, rows, oracle.DD)
    orth = None
    if info == 0:  # ||Q^T Q - I||_2 from the Dot2 Gram of the result
        gh, gl = oracle.fp64_gram(q, mode=oracle.DD)
        orth = float(np.linalg.norm((gh - np.eye(q.shape[1])) + gl, 2))
    del q
    dt64, nb64, _, info64 = cpu_sample(v, y, rows, oracle.FP64)
    one_rows = min(rows, 250_000)
    oracle.set_threads(1)
    try:
        dt1, nb1, _, _ = cpu_sample(v, y, one_rows, oracle.DD)
    finally:
        oracle.set_threads(cores)
    return {"value": nbytes / dt / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"first {rows:,} rows of the same V and Y: the paper's CPU arithmetic, projection + Gram + "
                      f"2-pass CholQR with Dot2 double-double sums (OpenMP over output entries and rows), "
                      f"{dt:.1f} s",
            "ms_per_step": dt * 1e3, "blocks_per_s": 1.0 / dt if rows == n else None,
            "fp64_cholqr2": {"value": nb64 / dt64 / 1e9, "unit": "GB/s", "ms_per_step": dt64 * 1e3,
                             "cholesky_info": info64},
            "one_core_dd": {"value": nb1 / dt1 / 1e9, "unit": "GB/s", "rows": one_rows},
            "orth_err": orth}


# -------------------------------------------------------------- clocks

def clocks_path(name):
    """Where the clock samples of a run go: $EO_CLOCKS_DIR/<name> when that
    variable names a folder, else a file in the temporary directory."""
    d = os.environ.get("EO_CLOCKS_DIR")
    if d and os.path.isdir(d):
        return os.path.join(d, name)
    return os.path.join(tempfile.gettempdir(), f"eo_{os.getpid()}_{name}")


class Clocks:
    def __init__(self, path, index):
        self.path = path
        self.proc = None
        self.index = index

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            # the timed region starts once the sampler writes (a short region
            # would otherwise end before nvidia-smi's first sample)
            t0 = time.time()
            while time.time() - t0 < 5.0 and self.proc.poll() is None:
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [s.strip() for s in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


DIGIT_PAIRS = 120  # FP16 digit-pair products per multiply-add of the compensated tensor-core kernels


def gram_traffic(n, kv, k):
    """DRAM bytes of one V^T Y launch of the tensor-core Gram kernel, from one
    ncu capture of the full-size launch (4e6 rows, kv = 64, k = 16:
    dram__bytes_read.sum 2,560.20 MB, dram__bytes_write.sum 3.08 MB of
    row-chunk partials); reads scale with the rows, the partials do not.
    None for other shapes."""
    if (kv, k) != (64, 16):
        return None
    return 2560.195328e6 * n / 4e6 + 3.078656e6


def apply_traffic(n, kv, k):
    """DRAM bytes of one projection launch (umma_rowprod_kernel<16>) at
    kv = 64, k = 16, from one ncu capture of the full-size launch (4e6 rows:
    dram__bytes_read.sum 2,560.24 MB, dram__bytes_write.sum 497.86 MB; the
    rest of the 512 MB of Y~ was still in L2 when the kernel ended); None for
    other shapes."""
    if (n, kv, k) != (4_000_000, 64, 16):
        return None
    return 2560.240384e6 + 497.863680e6


def peak_tensor():
    """Sustained dense BF16 (= FP16) tensor peak in TFLOP/s: the kernels run inside a long step."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["bf16_tflops_sustained"]), "measured"
    except Exception:
        return 1700.0, "fallback"


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------- GPU arm

def run_eo(a):
    import torch
    import torch.distributed as dist
    import paper_1806_01036_gb300 as eo
    import synth

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    n, kv, k = a.n, a.kv, a.k
    v_np, y_np = synth.project_block(seed=synth.SEED_BASE + 1 + 1000 * rank, n=n, kv=kv, k=k, kappa=a.kappa)

    def to_dev(x):
        return torch.from_numpy(np.ascontiguousarray(x.T)).to(dev).t()

    V, Y = to_dev(v_np), to_dev(y_np)
    Yt = torch.empty((k, n), dtype=torch.float64, device=dev).t()
    ctx = eo.Context(local)
    stream = torch.cuda.current_stream(dev)

    def step(prec=eo.DD, out=None, passes=0):
        out = Yt if out is None else out
        c = eo.gram(ctx, V, Y, prec=prec)
        eo.project_apply(ctx, V, Y, c, Yout=out, prec=prec, want_m=False)
        m = eo.gram(ctx, out, prec=prec)
        return eo.cholqr(ctx, out, passes=passes, prec=prec, M=m)

    for _ in range(max(3, a.warmup)):
        rh, rl, info = step()
    torch.cuda.synchronize()
    info0 = int(info.item())
    rd = torch.diagonal(rh).abs()
    two_passes = bool((rd.max() / rd.min()).item() > 1e7)
    # orthogonality of the result, measured with the library's own DD Gram
    gh, gl = eo.gram(ctx, Yt, prec=eo.DD)
    e = (gh.cpu().numpy() - np.eye(k)) + gl.cpu().numpy()  # k-by-k: its 2-norm on the host
    orth = float(np.linalg.norm(e, 2))
    cross = eo.gram(ctx, V, Yt, prec=eo.DD)
    cross_err = float(np.linalg.norm(cross[0].cpu().numpy() + cross[1].cpu().numpy(), 2))

    nbytes = step_bytes(n, kv, k, two_passes)
    ev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(5)) for _ in range(a.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = ctx.launches()
    clk = Clocks(clocks_path(f"clocks_rank{rank}.csv"), local)
    with clk:
        torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed launches
        t_all0 = torch.cuda.Event(enable_timing=True)
        t_all1 = torch.cuda.Event(enable_timing=True)
        t_all0.record(stream)
        for i in range(a.steps):
            ev[i][0].record(stream)
            c = eo.gram(ctx, V, Y, prec=eo.DD)
            ev[i][1].record(stream)
            eo.project_apply(ctx, V, Y, c, Yout=Yt, prec=eo.DD, want_m=False)
            ev[i][2].record(stream)
            m = eo.gram(ctx, Yt, prec=eo.DD)
            ev[i][3].record(stream)
            eo.cholqr(ctx, Yt, passes=0, prec=eo.DD, M=m)
            ev[i][4].record(stream)
        t_all1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    launches = ctx.launches() - l0
    if ws > 1:
        dist.barrier()
    total_ms = max_over_ranks(t_all0.elapsed_time(t_all1), dev)
    per = [e[0].elapsed_time(e[4]) for e in ev]
    gram_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    apply_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
    gram_m_ms = statistics.mean(e[2].elapsed_time(e[3]) for e in ev)
    chol_ms = statistics.mean(e[3].elapsed_time(e[4]) for e in ev)
    ms = total_ms / a.steps
    value = weak_scaling_value(ws, nbytes, ms)

    # roofline of the dominant kernel: the projection umma_rowprod_kernel<16>
    # (compensated Y - V C; the largest launch of the step, ahead of the
    # V^T Y Gram umma_gram_partial_kernel<16>, whose roofline is kept beside
    # it).  The path streams its operands from HBM, so the bound is the
    # measured copy bandwidth and `achieved` counts the algorithmic bytes
    # (V and Y read once, Y~ written once; V^T Y: V and Y read once) over the
    # launch's CUDA-event time.  The tensor-core view of the Gram
    # (algorithmic flops against the FP16 dense peak / 120 digit pairs per
    # multiply-add) is kept beside it.
    hbm_peak, peak_kind = peak_hbm()
    tc_peak, tc_kind = peak_tensor()
    gram_bytes = 8 * n * (kv + k)
    apply_bytes = 8 * n * (kv + 2 * k)
    gram_flops = 2.0 * n * kv * k
    gram_gbs = gram_bytes / (gram_ms * 1e-3) / 1e9
    apply_gbs = apply_bytes / (apply_ms * 1e-3) / 1e9
    tc_achieved = gram_flops / (gram_ms * 1e-3) / 1e12
    roof = {"bound": "hbm", "achieved": apply_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": apply_gbs / hbm_peak,
            "traffic": apply_traffic(n, kv, k),
            "kernel": f"umma_rowprod_kernel<16> (compensated Y - V C, {n:,} x {kv} x {k})",
            "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
            "algorithmic_bytes_per_launch": apply_bytes, "launch_ms": apply_ms,
            "gram_vty": {"kernel": f"umma_gram_partial_kernel<16> (compensated V^T Y, {n:,} x {kv} x {k})",
                         "ms": gram_ms, "algorithmic_bytes_per_launch": gram_bytes, "achieved": gram_gbs,
                         "frac": gram_gbs / hbm_peak, "traffic": gram_traffic(n, kv, k),
                         "tensor_digit_pairs": {"achieved_tflops": tc_achieved, "peak_tflops": tc_peak / DIGIT_PAIRS,
                                                "frac": tc_achieved / (tc_peak / DIGIT_PAIRS),
                                                "peak_source": f"{tc_kind} FP16/BF16 dense sustained {tc_peak:.1f} "
                                                               f"TFLOP/s / {DIGIT_PAIRS} digit pairs per multiply-add"}},
            "phases_ms": {"gram_vty": gram_ms, "apply": apply_ms, "gram_m": gram_m_ms, "cholqr": chol_ms},
            "phases_gbs": {"gram_vty": gram_gbs, "apply": apply_gbs,
                           "gram_m": 8 * n * k / (gram_m_ms * 1e-3) / 1e9,
                           "cholqr": (nbytes - gram_bytes - apply_bytes) / (chol_ms * 1e-3) / 1e9}}

    def timed_steps(fn, reps, warm=3):
        """Warm-up, then `reps` CUDA-event timings of fn(); returns (times, last result)."""
        res = None
        for _ in range(warm):
            res = fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return ts, res

    def dd_orth(q):
        gh, gl = eo.gram(ctx, q, prec=eo.DD)
        return float(np.linalg.norm((gh.cpu().numpy() - np.eye(q.shape[1])) + gl.cpu().numpy(), 2))

    def summary(ts, nb):
        p50 = float(np.percentile(ts, 50))
        return {"p50_ms": p50, "p99_ms": float(np.percentile(ts, 99)), "reps": len(ts),
                "value": nb / (p50 * 1e-3) / 1e9, "unit": "GB/s", "blocks_per_s": 1e3 / p50}

    reps = max(20, a.steps)
    # plain FP64 CholQR2 and the paper's FP64-pipe compensated kernels on the same input
    Yp = torch.empty_like(Yt.t()).t()
    comp, eft, same, single = {}, {}, {}, {}
    try:
        if a.no_comparators:
            raise _Skip()
        ts, (_, _, infop) = timed_steps(lambda: step(prec=eo.FP64, out=Yp, passes=2), reps)
        comp = dict(summary(ts, step_bytes(n, kv, k, True)), prec="fp64 CholQR2", cholesky_info=int(infop.item()),
                    orth_err=dd_orth(Yp))
    except _Skip:
        comp = {"skipped": "--no-comparators"}
    except Exception as ex:  # pragma: no cover - reporting only
        comp = {"error": str(ex)}
    try:
        if a.no_comparators:
            raise _Skip()
        ts, (_, _, infoe) = timed_steps(lambda: step(prec=eo.DD_EFT, out=Yp, passes=0), max(5, reps // 4), warm=1)
        eft = dict(summary(ts, nbytes), prec="dd_eft (FP64-pipe TwoProd/TwoSum)", cholesky_info=int(infoe.item()),
                   orth_err=dd_orth(Yp))
    except _Skip:
        eft = {"skipped": "--no-comparators"}
    except Exception as ex:  # pragma: no cover - reporting only
        eft = {"error": str(ex)}

    # same accuracy, more blocks/s: where plain FP64 CholQR2 succeeds (kappa = 1e6) the compensated step
    # needs one CholQR pass; both are timed on the same V and a Y with kappa(Y) = 1e6
    try:
        if a.no_comparators:
            raise _Skip()
        y6 = synth.conditioned(n, k, 1e6, synth.SEED_BASE + 2 + 1000 * rank)
        Ys6 = Y
        Y = to_dev(y6)
        del y6
        Y6t = torch.empty_like(Yt.t()).t()
        ts_dd, (rh6, _, info6) = timed_steps(lambda: step(prec=eo.DD, out=Y6t, passes=0), reps)
        rd6 = torch.diagonal(rh6).abs()
        passes6 = 2 if (rd6.max() / rd6.min()).item() > 1e7 else 1
        orth_dd6 = dd_orth(Y6t)
        del Y6t
        ts_64, (_, _, info64) = timed_steps(lambda: step(prec=eo.FP64, out=Yp, passes=2), reps)
        orth_646 = dd_orth(Yp)
        same = {"kappa": 1e6,
                "dd": dict(summary(ts_dd, step_bytes(n, kv, k, passes6 == 2)), passes=passes6,
                           cholesky_info=int(info6.item()), orth_err=orth_dd6),
                "fp64_cholqr2": dict(summary(ts_64, step_bytes(n, kv, k, True)), cholesky_info=int(info64.item()),
                                     orth_err=orth_646)}
        same["dd_speedup_blocks_per_s"] = same["dd"]["blocks_per_s"] / same["fp64_cholqr2"]["blocks_per_s"]
        Y = Ys6
    except _Skip:
        same = {"skipped": "--no-comparators"}
    except Exception as ex:  # pragma: no cover - reporting only
        same = {"error": str(ex)}
    # the single-block configuration (100,000 x 8, sigma 1 .. 1e-6, L2-resident): CholQR alone
    try:
        if a.no_comparators:
            raise _Skip()
        xs = synth.single_cholqr()
        X0s = to_dev(xs)
        Xs = torch.empty_like(X0s.t()).t()

        def one(prec, passes):
            Xs.copy_(X0s)
            return eo.cholqr(ctx, Xs, passes=passes, prec=prec)

        res = {}
        for prec, passes, name in ((eo.FP64, 2, "fp64_cholqr2"), (eo.DD, 0, "dd")):
            ts, _ = timed_steps(lambda: one(prec, passes), max(50, reps))
            res[name] = {"p50_ms": float(np.percentile(ts, 50)), "p99_ms": float(np.percentile(ts, 99)),
                         "blocks_per_s": 1e3 / float(np.percentile(ts, 50)), "orth_err": dd_orth(Xs),
                         "note": "includes the device copy restoring X (0.8 MB)"}
            # the same call captured once in a CUDA graph and replayed: one launch per block
            one(prec, passes)
            torch.cuda.synchronize()
            gr = torch.cuda.CUDAGraph()
            cap = torch.cuda.Stream(dev)
            cap.wait_stream(stream)
            with torch.cuda.stream(cap):
                with torch.cuda.graph(gr, stream=cap):
                    one(prec, passes)  # the binding runs the call on the capturing stream
            torch.cuda.synchronize()
            tsg, _ = timed_steps(gr.replay, max(50, reps))
            res[name + "_graph"] = {"p50_ms": float(np.percentile(tsg, 50)), "p99_ms": float(np.percentile(tsg, 99)),
                                    "blocks_per_s": 1e3 / float(np.percentile(tsg, 50)), "orth_err": dd_orth(Xs),
                                    "note": "one CUDA-graph replay of the copy restoring X and the call"}
            del gr
        single = {"workload": "single CholQR, X 100,000 x 8, sigma 1 .. 1e-6 (L2-resident)", **res}
        del X0s, Xs
    except _Skip:
        single = {"skipped": "--no-comparators"}
    except Exception as ex:  # pragma: no cover - reporting only
        single = {"error": str(ex)}
    del Yp

    # end to end through the C-ABI with pinned host buffers: every step copies
    # its V and Y from the host and reads Q and R back.  Consecutive steps
    # are independent blocks, so the copies overlap the compute of the
    # neighbouring steps: the inputs of step i + 1 go up on one copy stream
    # (into the second of two device buffer sets) while step i runs, and Q
    # of step i comes back on another copy stream; events order each buffer's
    # reuse.  The timed region holds every copy of every step.
    e2e = None
    if not a.no_e2e:
        Vh = torch.from_numpy(np.ascontiguousarray(v_np.T)).pin_memory()
        Yh = torch.from_numpy(np.ascontiguousarray(y_np.T)).pin_memory()
        Qh = [torch.empty((k, n), dtype=torch.float64).pin_memory() for _ in range(2)]
        Rh = [torch.empty((k, k), dtype=torch.float64).pin_memory() for _ in range(2)]
        Vd = [torch.empty((kv, n), dtype=torch.float64, device=dev) for _ in range(2)]
        Yd = [torch.empty((k, n), dtype=torch.float64, device=dev) for _ in range(2)]
        Qd = [torch.empty((k, n), dtype=torch.float64, device=dev) for _ in range(2)]
        Rd = [None, None]
        up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        ev_in = [torch.cuda.Event() for _ in range(2)]     # inputs of buffer b are on the device
        ev_used = [torch.cuda.Event() for _ in range(2)]   # compute on buffer b's inputs is done
        ev_out = [torch.cuda.Event() for _ in range(2)]    # Q of buffer b is computed
        ev_back = [torch.cuda.Event() for _ in range(2)]   # Q of buffer b is back on the host
        for b in range(2):
            ev_used[b].record(stream)
            ev_back[b].record(stream)

        def upload(b):
            with torch.cuda.stream(up):
                up.wait_event(ev_used[b])
                Vd[b].copy_(Vh, non_blocking=True)
                Yd[b].copy_(Yh, non_blocking=True)
                ev_in[b].record(up)

        def compute(b):
            stream.wait_event(ev_in[b])
            stream.wait_event(ev_back[b])  # Q buffer b is free again
            c = eo.gram(ctx, Vd[b].t(), Yd[b].t(), prec=eo.DD)
            eo.project_apply(ctx, Vd[b].t(), Yd[b].t(), c, Yout=Qd[b].t(), prec=eo.DD, want_m=False)
            m = eo.gram(ctx, Qd[b].t(), prec=eo.DD)
            Rd[b], _, _ = eo.cholqr(ctx, Qd[b].t(), passes=0, prec=eo.DD, M=m)
            ev_used[b].record(stream)
            ev_out[b].record(stream)

        def download(b):
            with torch.cuda.stream(down):
                down.wait_event(ev_out[b])
                Qh[b].copy_(Qd[b], non_blocking=True)
                Rh[b].copy_(Rd[b].t(), non_blocking=True)
                ev_back[b].record(down)

        done = []  # per step: its read-back finished (timing events on the copy-back stream)

        def run_steps(count, mark=False):
            upload(0)
            for i in range(count):
                b = i & 1
                if i + 1 < count:
                    upload(b ^ 1)
                compute(b)
                download(b)
                if mark:
                    done.append(torch.cuda.Event(enable_timing=True))
                    done[-1].record(down)
            stream.wait_stream(down)

        run_steps(2)
        torch.cuda.synchronize()
        ke = max(2, a.steps)  # the same K steps as the device-timed region (fill and drain included)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        s0.record(stream)
        run_steps(ke, mark=True)
        s1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(s0.elapsed_time(s1) / ke, dev)
        gaps = [s0.elapsed_time(done[0])] + [done[i - 1].elapsed_time(done[i]) for i in range(1, len(done))]
        q_ok = bool(np.array_equal(Qh[(ke - 1) & 1].numpy()[:, :1024], Yt.t()[:, :1024].cpu().numpy()))
        # the copies of one step alone, both directions at once (after the
        # timed region): the least time a step can take on this host link,
        # which varies from box to box and run to run
        fl = []
        for _ in range(3):
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            f0.record(stream)
            up.wait_stream(stream)
            down.wait_stream(stream)
            with torch.cuda.stream(up):
                Vd[0].copy_(Vh, non_blocking=True)
                Yd[0].copy_(Yh, non_blocking=True)
            with torch.cuda.stream(down):
                Qh[0].copy_(Qd[0], non_blocking=True)
            stream.wait_stream(up)
            stream.wait_stream(down)
            f1.record(stream)
            torch.cuda.synchronize()
            fl.append(f0.elapsed_time(f1))
        e2e = {"value": weak_scaling_value(ws, nbytes, ems), "unit": "GB/s", "ms_per_step": ems,
               "h2d_bytes_per_step": 8 * n * (kv + k), "d2h_bytes_per_step": 8 * n * k + 8 * k * k,
               "steps": ke, "overlap": "inputs of step i+1 uploaded and Q of step i-1 read back while step i runs",
               "copy_floor_ms": float(np.median(fl)),
               "step_gaps_ms": [round(g, 3) for g in gaps],  # start -> first read-back done, then between read-backs
               "result_matches_device_run": q_ok}
        del Vd, Yd, Qd

    cpu = None
    if rank == 0 and not a.no_cpu:
        cpu = cpu_baseline(v_np, y_np, a.cpu_rows)
    others = None
    if rank == 0 and ws == 1 and not a.no_comparators and not a.no_other_configs:
        others = other_configs()

    out = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded; V Haar-orthonormal, Y = U diag(sigma) W^T, sigma 1..1e-10)",
        "config": {"workload": WORKLOAD.format(n=n, kv=kv, k=k, kappa=a.kappa), "n": n, "kv": kv, "k": k, "kappa": a.kappa, "prec": "dd",
                   "passes": 2 if two_passes else 1, "parallelism": f"replicas x{ws}",
                   "l2": "inputs (2.6 GB/step) larger than L2; no flush"},
        "blocks_per_s": ws * 1000.0 / ms, "p50_ms": float(np.percentile(per, 50)),
        "p99_ms": float(np.percentile(per, 99)),
        "orth_err": orth, "cross_err": cross_err, "cholesky_info": info0,
        "bytes_per_step": nbytes, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        "clocks": clk.summary(), "gpu_launches": launches, "fp64_comparator": comp, "dd_eft_comparator": eft,
        "same_accuracy": same, "single_block": single, "other_configs": others,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def other_configs():
    """The other workloads, each in its own process after the step's
    measurements (outside its timed region), summarised: the precision sweep,
    the batched SVQB graph, serving at 2,000 requests/s offered and at 0.8x
    the capacity that run measured, the iterated two-phase algorithm and the
    compensated update alone per k.  A workload that fails or runs out of
    time is reported as such."""
    def run(args, timeout=420):
        t0 = time.time()
        try:
            r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True,
                               text=True, timeout=timeout, cwd=ROOT)
            lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
            if r.returncode != 0 or not lines:
                return None, {"error": f"exit {r.returncode}", "stderr_tail": r.stderr[-300:]}
            return json.loads(lines[-1]), {"seconds": round(time.time() - t0, 1)}
        except Exception as e:  # reported, never fatal to the main line
            return None, {"error": repr(e)[:300]}

    def summarise(info, f):
        try:
            info.update(f())
        except Exception as e:  # a workload whose line lacks a field: reported, never fatal
            info["error"] = "summary: " + repr(e)[:200]
        return info

    out = {}
    d, info = run(["--workload", "sweep"])
    if d:
        def sweep():
            res = {}
            for r in d["results"]:
                res.setdefault(str(r["k"]), {})[r["mode"]] = [round(r["xtx_gbs"], 1), round(r["xty_gbs"], 1)]
            return {"command": "python bench.py --workload sweep", "unit": "GB/s [X^T X, X^T Y]",
                    "config": d["config"]["workload"], "results": res}
        summarise(info, sweep)
    out["sweep"] = info
    d, info = run(["--workload", "batched", "--steps", "5", "--warmup", "3"])
    if d:
        summarise(info, lambda: {
            "command": "python bench.py --workload batched --steps 5 --warmup 3", "config": d["config"]["workload"],
            "ms_per_step": d["ms_per_step"], "blocks_per_s": d["blocks_per_s"], "gbs": d["value"],
            "p50_ms": d["p50_ms"], "p99_ms": d["p99_ms"], "orth_err_max": d["orth_err_max"],
            "hbm_frac": d["roofline"]["frac"], "fp64_graph_ms": d["comparators"]["fp64_graph_ms"],
            "clocks": d["clocks"]})
    out["batched"] = info
    d, info = run(["--workload", "serve"])
    cap = None
    if d:
        summarise(info, lambda: {
            "command": "python bench.py --workload serve", "config": d["config"]["workload"],
            "requests_per_s": d["value"], "gbs": d["gbs"], "p50_ms": d["p50_ms"], "p99_ms": d["p99_ms"],
            "queue_p50_ms": d["queue_p50_ms"], "queue_p99_ms": d["queue_p99_ms"],
            "orth_err_max": d["orth_err_max"], "cross_err_max": d["cross_err_max"]})
        cap = d.get("value")
    out["serve_offered_2000"] = info
    if cap:
        rate = round(0.8 * cap, 1)
        d, info = run(["--workload", "serve", "--rate", str(rate), "--requests", "1500"])
        if d:
            summarise(info, lambda: {
                "command": f"python bench.py --workload serve --rate {rate} --requests 1500",
                "offered_per_s": rate, "requests_per_s": d["value"], "p50_ms": d["p50_ms"], "p99_ms": d["p99_ms"],
                "queue_p99_ms": d["queue_p99_ms"]})
        out["serve_at_0.8_capacity"] = info
    d, info = run(["--workload", "iterated"])
    if d:
        summarise(info, lambda: {
            "command": "python bench.py --workload iterated", "config": d["config"]["workload"],
            "ms_per_block [kv, k, fp64, dd, dd iterations]": [
                [r["kv"], r["k"], round(r["fp64"]["ms"], 2), round(r["dd"]["ms"], 2), r["dd"]["iterations"]]
                for r in d["results"]]})
    out["iterated"] = info
    d, info = run(["--workload", "update"])
    if d:
        summarise(info, lambda: {
            "command": "python bench.py --workload update", "config": d["config"]["workload"],
            "p50_ms_and_gbs_per_k": {k: [round(r["p50_ms"], 3), round(r["gbs"], 1)] for k, r in d["results"].items()}})
    out["update"] = info
    return out


# --------------------------------------------------------- reference arm

def run_reference(a):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import synth
    n, kv, k = a.n, a.kv, a.k
    rows = min(n, a.cpu_rows if a.cpu_rows > 0 else 1_000_000)
    v_np = synth.orthonormal_basis(rows, kv, synth.SEED_BASE + 1)
    y_np = synth.conditioned(rows, k, a.kappa, synth.SEED_BASE + 1 + 1000)
    for _ in range(a.warmup):
        cpu_sample(v_np, y_np, rows, oracle.DD)
    times = []
    nbytes = 0
    for _ in range(a.steps):
        dt, nbytes, _, _ = cpu_sample(v_np, y_np, rows, oracle.DD)
        times.append(dt)
    ms = 1000 * statistics.mean(times)
    value = nbytes / (ms * 1e-3) / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64 (double-double sums)", "data": "synthetic (seeded, same recipe)",
           "p50_ms": float(np.percentile(times, 50)) * 1e3, "p99_ms": float(np.percentile(times, 99)) * 1e3,
           "config": {"workload": WORKLOAD.format(n=n, kv=kv, k=k, kappa=a.kappa), "n": n, "kv": kv, "k": k,
                      "kappa": a.kappa, "sample_rows": rows},
           "cpu_baseline": {"value": value, "unit": "GB/s", "cores": oracle.threads(), "kind": "oracle",
                            "sample": f"{rows:,} rows per step of the same workload recipe: the paper's CPU "
                                      "arithmetic (Dot2 double-double sums), projection + Gram + 2-pass CholQR"},
           "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------ iterated orthogonalization

ITER_METRIC = "iterated two-phase orthogonalization: ms per block and iterations to eps = 1e-10, FP64 vs DD"


def run_iterated(a):
    """The runtime figure's setting (Sec. 4.2): W n x kv orthonormal, X n x k
    with kappa(X) = 1e6 and kappa(X, W) = 1e12, orthogonalized by repeated
    phase I + SVQB until max(||W^T X||_2, ||X^T X - I||_2) <= 1e-10, in plain
    FP64 and in the compensated mode.  Inputs are generated on the GPU from a
    seeded Gaussian (W and the factors of X: torch's QR; X = W A + U diag(s)
    V^T / kappa(X, W) with s log-spaced 1 .. 1e-6)."""
    import torch
    import paper_1806_01036_gb300 as eo

    ws, rank, local = dist_env()
    dev = torch.device("cuda", local)
    n = a.n if a.n != 4_000_000 else 8_000_000
    ctx = eo.Context(local)
    stream = torch.cuda.current_stream(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(20180604 + 7 + 1000 * rank)
    f64 = torch.float64

    def colmajor(t):
        return t.t().contiguous().t()

    def haar(rows, cols):
        q, r = torch.linalg.qr(torch.randn(rows, cols, dtype=f64, device=dev, generator=g))
        return q * torch.sign(torch.diagonal(r))[None, :]

    results = []
    for kv in (10, 20, 40):
        W = colmajor(haar(n, kv))
        for k in (1, 2, 4):
            A = torch.randn(kv, k, dtype=f64, device=dev, generator=g)
            s = torch.logspace(0.0, -6.0, k, dtype=f64, device=dev) if k > 1 else torch.ones(1, dtype=f64, device=dev)
            X0 = colmajor(W @ A + (haar(n, k) * s[None, :]) @ haar(k, k).t() / 1e12)
            X = torch.empty_like(X0)
            row = {"n": n, "kv": kv, "k": k}
            for prec, name in ((eo.FP64, "fp64"), (eo.DD, "dd")):
                for _ in range(max(1, a.warmup)):
                    X.copy_(X0)
                    eo.orthogonalize(ctx, W, X, eps=1e-10, max_iter=12, prec=prec)
                times, its = [], None
                for _ in range(a.steps):
                    X.copy_(X0)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    its, rk = eo.orthogonalize(ctx, W, X, eps=1e-10, max_iter=12, prec=prec)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1))
                ch, cl = eo.gram(ctx, W, X, prec=eo.DD)
                gh, gl = eo.gram(ctx, X, prec=eo.DD)
                cross = float(torch.linalg.matrix_norm((ch + cl).cpu(), ord=2))
                orth = float(torch.linalg.matrix_norm((gh - torch.eye(k, dtype=f64, device=dev) + gl).cpu(), ord=2))
                row[name] = {"ms": statistics.median(times), "iterations": int(its.item()), "rank": int(rk.item()),
                             "cross_err": cross, "orth_err": orth}
            results.append(row)
            del X0, X
        del W
    out = {"metric": ITER_METRIC, "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
           "data": "synthetic (seeded on the GPU; torch QR factors)", "dtype": "f64",
           "config": {"workload": f"iterated two-phase orthogonalization, n = {n:,}, kv in 10/20/40, k in 1/2/4, "
                                  "kappa(X) = 1e6, kappa(X, W) = 1e12, eps = 1e-10"},
           "results": results}
    if rank == 0:
        print(json.dumps(out), flush=True)


# ------------------------------------------------------- batched SVQB

BATCH_METRIC = "batched SVQB: HBM GB/s and blocks/s of one CUDA-graph launch, DD vs plain FP64; p50/p99"


def run_batched(a):
    """Many blocks of uneven n and k in one graph launch (eo_batch_*): 512
    blocks with n log-uniform in [1e4, 2e6], k uniform in {4, 8, 16, 32},
    kappa log-uniform in [1e2, 1e10]; SVQB in the compensated mode with the
    automatic second pass, launch shapes from the autotuner.  Blocks are
    X = G diag(sigma) Q^T with G Gaussian / sqrt(n) (its condition number is
    within (1 + sqrt(k/n)) / (1 - sqrt(k/n)) <= 1.13 of 1; seeded, on the GPU),
    sigma log-spaced 1 .. 1/kappa and Q a Haar k x k rotation (seeded numpy
    QR on the host).  A step restores the blocks from a pristine copy
    (untimed) and runs the graph once (timed with CUDA events)."""
    import torch
    import paper_1806_01036_gb300 as eo

    ws, rank, local = dist_env()
    dev = torch.device("cuda", local)
    nblk = a.blocks
    rng = np.random.default_rng(20180604 + 3 + 1000 * rank)
    ns = np.exp(rng.uniform(np.log(1e4), np.log(2e6), nblk)).astype(np.int64)
    ks = rng.choice([4, 8, 16, 32], nblk)
    kappas = np.exp(rng.uniform(np.log(1e2), np.log(1e10), nblk))
    g = torch.Generator(device=dev)
    g.manual_seed(20180604 + 3 + 1000 * rank)
    f64 = torch.float64
    X, X0 = [], []
    for n, k, kap in zip(ns, ks, kappas):
        n, k = int(n), int(k)
        qn, rn = np.linalg.qr(rng.standard_normal((k, k)))  # Haar k x k rotation (host: k is small)
        q = torch.from_numpy(qn * np.sign(np.diag(rn))[None, :]).to(dev)
        s = torch.logspace(0.0, -float(np.log10(kap)), k, dtype=f64, device=dev)
        x0 = (torch.randn(n, k, dtype=f64, device=dev, generator=g) * (s / float(np.sqrt(n)))[None, :]) @ q.t()
        x0 = x0.t().contiguous().t()
        X0.append(x0)
        X.append(torch.empty_like(x0.t()).t())
    ctx = eo.Context(local)
    stream = torch.cuda.current_stream(dev)

    def restore():
        for x, x0 in zip(X, X0):
            x.copy_(x0)

    def make(prec, tune, branches=0):
        t0 = time.perf_counter()
        b = eo.Batch(ctx, X, method=eo.BATCH_SVQB, passes=0, prec=prec, tune=tune, branches=branches)
        return b, time.perf_counter() - t0

    def timed(run, steps):
        times = []
        for _ in range(steps):
            restore()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return times

    bt, create_s = make(eo.DD, True, a.branches)
    for _ in range(max(3, a.warmup)):
        restore()
        bt.run()
    torch.cuda.synchronize()
    passes = bt.passes()
    nbytes = int(sum(24 * int(n) * int(k) * p for n, k, p in zip(ns, ks, passes)))
    # accuracy of the last run: max over blocks of ||Q^T Q - I||_2 (library DD Gram)
    orth = 0.0
    for x, k in zip(X, ks):
        gh, gl = eo.gram(ctx, x, prec=eo.DD)
        e = (gh.cpu().numpy() - np.eye(int(k))) + gl.cpu().numpy()
        orth = max(orth, float(np.linalg.norm(e, 2)))
    ranks = bt.out.cpu().numpy()
    sweeps = bt.sweeps()  # Jacobi sweeps of each block's last eigensolve
    sweep_stats = {}
    for kk in (4, 8, 16, 32):
        sel = [sw for sw, kb, pb in zip(sweeps, ks, passes) if int(kb) == kk]
        if sel:
            sweep_stats[f"k{kk}"] = {"blocks": len(sel), "mean": float(np.mean(sel)), "max": int(np.max(sel))}

    torch.cuda.synchronize()
    l0 = ctx.launches()
    clk = Clocks(clocks_path(f"clocks_batched_rank{rank}.csv"), local)
    with clk:
        torch.cuda.nvtx.range_push("timed")
        times = timed(bt.run, a.steps)
        torch.cuda.nvtx.range_pop()
    launches = (ctx.launches() - l0)
    ms = statistics.mean(times)
    value = weak_scaling_value(ws, nbytes, max_over_ranks(ms, dev))

    # comparators on the same blocks: untuned shapes, one call per block on
    # one stream (no graph), and plain FP64 in the same graph form
    bu, _ = make(eo.DD, False, a.branches)
    untuned = statistics.mean(timed(bu.run, max(1, a.steps // 2)))
    bu.close()

    def sequential():
        for x in X:
            eo.svqb(ctx, x, passes=0, prec=eo.DD)

    seq = statistics.mean(timed(sequential, max(1, a.steps // 2)))
    bf, _ = make(eo.FP64, False, a.branches)
    fp64 = statistics.mean(timed(bf.run, max(1, a.steps // 2)))
    orth_fp64 = 0.0
    for x, k in zip(X, ks):
        gh, gl = eo.gram(ctx, x, prec=eo.DD)
        e = (gh.cpu().numpy() - np.eye(int(k))) + gl.cpu().numpy()
        orth_fp64 = max(orth_fp64, float(np.linalg.norm(e, 2))) if np.all(np.isfinite(e)) else float("inf")
    bf.close()
    hbm_peak, peak_kind = peak_hbm()
    tiles = {}
    for i in range(nblk):
        key = f"k{int(ks[i])}_n2^{int(np.log2(ns[i]))}"
        tiles[key] = bt.tile(i)
    out = {
        "metric": BATCH_METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded on the GPU: Gaussian x diag(sigma) x Haar rotation)",
        "config": {"workload": f"batched SVQB: {nblk} blocks, n log-uniform [1e4, 2e6], k in 4/8/16/32, "
                               "kappa log-uniform [1e2, 1e10], DD with automatic second pass, one graph launch",
                   "blocks": nblk, "rows_total": int(ns.sum()), "branches": bt.branches(),
                   "two_pass_blocks": int(sum(p == 2 for p in passes)),
                   "l2": "blocks total %.1f GB, larger than L2; no flush" % (8 * float(np.sum(ns * ks)) / 1e9)},
        "blocks_per_s": ws * nblk / (ms * 1e-3), "p50_ms": float(np.percentile(times, 50)),
        "p99_ms": float(np.percentile(times, 99)), "orth_err_max": orth, "min_rank_over_k": float(np.min(ranks / ks)),
        "bytes_per_step": nbytes,
        "roofline": {"bound": "hbm", "achieved": nbytes / (ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                     "frac": nbytes / (ms * 1e-3) / 1e9 / hbm_peak, "traffic": None,
                     "peak_source": peak_kind, "kernel": "whole graph (Gram + eigensolve + update per block)"},
        "gpu_launches": launches, "graph_kernels": bt.kernels(), "create_s": create_s,
        "comparators": {"untuned_ms": untuned, "sequential_calls_ms": seq, "fp64_graph_ms": fp64,
                        "fp64_orth_err_max": orth_fp64},
        "tiles": tiles, "clocks": clk.summary(), "last_pass_jacobi_sweeps": sweep_stats,
    }
    bt.close()
    if rank == 0:
        print(json.dumps(out), flush=True)


# ------------------------------------------------------------- serving

SERVE_METRIC = "serving: requests/s with p50/p99 latency, projection + compensated CholQR against resident bases"


def run_serve(a):
    """Request server under Poisson arrivals (eo_server_*): 256 simulated
    eigensolves, each with a resident orthonormal basis V (n log-uniform in
    [5e4, 8e6], kv uniform in {8, 16, 32, 64}), submit blocks Y of kv/4
    columns (kappa log-uniform in [1e2, 1e12]) at 2,000 requests/s in total
    (seeded exponential gaps, client uniform); each request is
    Y - V (V^T Y) and a compensated CholQR with the automatic second pass,
    admitted under a 150 GB device-memory budget.  Bases are seeded
    Gaussians made orthonormal by the library's own two-pass compensated
    CholQR; blocks are Gaussian x diag(sigma), generated on the GPU."""
    import torch
    import paper_1806_01036_gb300 as eo

    ws, rank, local = dist_env()
    dev = torch.device("cuda", local)
    rng = np.random.default_rng(20180604 + 4 + 1000 * rank)
    nc = a.clients
    ns = np.exp(rng.uniform(np.log(5e4), np.log(8e6), nc)).astype(np.int64)
    kvs = rng.choice([8, 16, 32, 64], nc)
    kappas = np.exp(rng.uniform(np.log(1e2), np.log(1e12), nc))
    g = torch.Generator(device=dev)
    g.manual_seed(20180604 + 4 + 1000 * rank)
    f64 = torch.float64
    ctx = eo.Context(local)

    def colmajor_randn(n, k):
        return torch.randn(k, n, dtype=f64, device=dev, generator=g).t()

    V, Y, Yo = [], [], []
    for n, kv, kap in zip(ns, kvs, kappas):
        n, kv = int(n), int(kv)
        v = colmajor_randn(n, kv)
        eo.cholqr(ctx, v, passes=2, prec=eo.DD)
        k = max(1, kv // 4)
        s = torch.logspace(0.0, -float(np.log10(kap)), k, dtype=f64, device=dev)
        y = colmajor_randn(n, k) * (s / float(np.sqrt(n)))[None, :]
        V.append(v)
        Y.append(y)
        Yo.append(torch.empty_like(y.t()).t())
    torch.cuda.synchronize()
    srv = eo.Server(ctx, budget=int(a.budget_gb * 1e9), slots=a.slots)
    ids = [srv.add_basis(v) for v in V]
    # warm-up: one request per client
    for i in range(nc):
        srv.submit(ids[i], Y[i], Yout=Yo[i])
    while True:
        st = srv.stats()
        if st["queued"] == 0 and st["running"] == 0:
            break
        time.sleep(0.001)
    srv.poll(1 << 16)
    # the timed trace
    nreq = a.requests
    gaps = rng.exponential(1.0 / a.rate, nreq)
    arrival = np.cumsum(gaps)
    who = rng.integers(0, nc, nreq)
    nbytes = 0
    for i in who:
        n, kv = int(ns[i]), int(kvs[i])
        k = max(1, kv // 4)
        nbytes += 8 * n * (2 * kv + 5 * k)
    clk = Clocks(clocks_path(f"clocks_serve_rank{rank}.csv"), local)
    l0 = srv.stats()["kernels"]
    with clk:
        t0 = time.perf_counter()
        rids = []
        for t, i in zip(arrival, who):
            while time.perf_counter() - t0 < t:
                pass
            rids.append(srv.submit(ids[i], Y[i], Yout=Yo[i]))
        lat = []
        for r in rids:
            st, l = srv.wait(r, timeout=600.0)
            if st != eo.OK:
                raise RuntimeError("request failed")
            lat.append(l)
        t1 = time.perf_counter()
    done = srv.poll(1 << 16)
    qms = [q for _, _, q, _ in done]
    stats = srv.stats()
    launches = stats["kernels"] - l0
    # accuracy of the last result of every client
    orth, cross = 0.0, 0.0
    for i in sorted(set(int(x) for x in who)):
        k = Yo[i].shape[1]
        gh, gl = eo.gram(ctx, Yo[i], prec=eo.DD)
        e = (gh.cpu().numpy() - np.eye(k)) + gl.cpu().numpy()
        orth = max(orth, float(np.linalg.norm(e, 2)))
        ch, cl = eo.gram(ctx, V[i], Yo[i], prec=eo.DD)
        cross = max(cross, float(np.linalg.norm(ch.cpu().numpy() + cl.cpu().numpy(), 2)))
    srv.close()
    span = t1 - t0
    hbm_peak, peak_kind = peak_hbm()
    out = {
        "metric": SERVE_METRIC, "value": nreq / span, "unit": "requests/s", "n_gpus": ws, "steps": nreq,
        "warmup": nc, "ms_per_step": 1e3 * span / nreq, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded on the GPU: bases made orthonormal by the library's DD CholQR2)",
        "config": {"workload": f"serving: {nc} resident bases (n log-uniform [5e4, 8e6], kv in 8/16/32/64), "
                               f"blocks of kv/4 columns (kappa log-uniform [1e2, 1e12]), Poisson arrivals at "
                               f"{a.rate:g} requests/s, {a.budget_gb:g} GB budget, {a.slots} slots",
                   "resident_gb": stats["resident"] / 1e9, "offered_rate": a.rate, "requests": nreq,
                   "l2": "bases and blocks far larger than L2; no flush"},
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(np.mean(lat)), "queue_p50_ms": float(np.percentile(qms, 50)) if qms else None,
        "queue_p99_ms": float(np.percentile(qms, 99)) if qms else None,
        "gbs": nbytes / span / 1e9, "hbm_frac": nbytes / span / 1e9 / hbm_peak, "hbm_peak_source": peak_kind,
        "peak_running": stats["peak_running"], "peak_inflight_gb": stats["peak_inflight"] / 1e9,
        "orth_err_max": orth, "cross_err_max": cross, "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(out), flush=True)


# --------------------------------------------------- precision sweep, single

SWEEP_METRIC = "Gram X^T X and X^T Y: HBM GB/s per mode (FP64, DD, FP32-in, DD-EFT) and k"


def run_sweep(a):
    """The precision sweep of the Gram products: n rows (32e6 unless --n is
    given), k in {1, 2, 4, 8, 16, 32, 64}, X built with kappa = 1e8 (seeded
    Gaussian / sqrt(n) times sigma log-spaced 1 .. 1e-8 on the GPU; an FP32
    copy for the FP32-input mode), Y a second such block; modes FP64, DD
    (compensated), FP32 inputs with FP64 accumulation, and the paper's FP64
    error-free transformations (DD-EFT, k <= 16).  Each entry: median of
    --steps launches after --warmup, CUDA events; bytes 8nk (X^T X) or 16nk
    (X^T Y), 4nk / 8nk for FP32 inputs.  Accuracy: max |G - G_DD| / max |G_DD|."""
    import torch
    import paper_1806_01036_gb300 as eo

    ws, rank, local = dist_env()
    dev = torch.device("cuda", local)
    n = a.n if a.n != 4_000_000 else 32_000_000
    ctx = eo.Context(local)
    stream = torch.cuda.current_stream(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(20180604 + 2 + 1000 * rank)

    def block(k):
        s = torch.logspace(0.0, -8.0, k, dtype=torch.float64, device=dev) if k > 1 else torch.ones(
            1, dtype=torch.float64, device=dev)
        return (torch.randn(k, n, dtype=torch.float64, device=dev, generator=g) * (s / n ** 0.5)[:, None]).t()

    def timed(f):
        for _ in range(max(1, a.warmup)):
            f()
        ts = []
        for _ in range(max(1, a.steps)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            f()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    hbm_peak, peak_kind = peak_hbm()
    rows = []
    for k in (1, 2, 4, 8, 16, 32, 64):
        X, Y = block(k), block(k)
        X32, Y32 = X.float().t().contiguous().t(), Y.float().t().contiguous().t()
        ref = eo.gram(ctx, X, prec=eo.DD)
        refxy = eo.gram(ctx, X, Y, prec=eo.DD)
        scale = float(ref[0].abs().max())
        scalexy = float(refxy[0].abs().max())
        for prec, name in ((eo.FP64, "fp64"), (eo.DD, "dd"), (eo.F32, "f32"), (eo.DD_EFT, "dd_eft")):
            if prec == eo.DD_EFT and k > 16:
                continue
            A, B, w = (X32, Y32, 4) if prec == eo.F32 else (X, Y, 8)
            ms = timed(lambda: eo.gram(ctx, A, prec=prec))
            msxy = timed(lambda: eo.gram(ctx, A, B, prec=prec))
            gh, gl = eo.gram(ctx, A, prec=prec)
            ghxy, glxy = eo.gram(ctx, A, B, prec=prec)
            err = float(((gh - ref[0]) + (gl - ref[1])).abs().max()) / scale
            errxy = float(((ghxy - refxy[0]) + (glxy - refxy[1])).abs().max()) / scalexy
            rows.append({"k": k, "mode": name, "xtx_ms": ms, "xtx_gbs": w * n * k / (ms * 1e-3) / 1e9,
                         "xty_ms": msxy, "xty_gbs": 2 * w * n * k / (msxy * 1e-3) / 1e9,
                         "xtx_err_vs_dd": err, "xty_err_vs_dd": errxy})
        del X, Y, X32, Y32
        torch.cuda.empty_cache()
    out = {"metric": SWEEP_METRIC, "n_gpus": ws, "steps": a.steps, "warmup": a.warmup, "dtype": "f64",
           "data": "synthetic (seeded on the GPU)", "hbm_peak_gbs": hbm_peak, "hbm_peak_source": peak_kind,
           "config": {"workload": f"precision sweep: n = {n:,}, k in 1..64, kappa = 1e8, X^T X and X^T Y",
                      "l2": "inputs of k >= 1 are 256 MB or more, larger than L2; no flush"},
           "results": rows}
    if rank == 0:
        print(json.dumps(out), flush=True)


SINGLE_METRIC = "single CholQR of 100,000 x 8: blocks/s, FP64 CholQR2 vs DD one pass (L2-resident)"


def run_single(a):
    """A small block that fits in L2 (6.4 MB): X 100,000 x 8 with sigma
    log-spaced 1 .. 1e-6 (synth.single_cholqr), orthogonalized in place from
    a device copy each call: plain FP64 CholQR2 against compensated CholQR
    (automatic pass count).  Reported L2-warm, as the block stays resident."""
    import torch
    import paper_1806_01036_gb300 as eo
    import synth

    ws, rank, local = dist_env()
    dev = torch.device("cuda", local)
    x = synth.single_cholqr()
    X0 = torch.from_numpy(np.ascontiguousarray(x.T)).to(dev).t()
    X = torch.empty_like(X0.t()).t()
    ctx = eo.Context(local)
    stream = torch.cuda.current_stream(dev)
    res = {}
    for prec, passes, name in ((eo.FP64, 2, "fp64_cholqr2"), (eo.DD, 0, "dd_auto")):
        for _ in range(max(3, a.warmup)):
            X.copy_(X0)
            eo.cholqr(ctx, X, passes=passes, prec=prec)
        ts = []
        for _ in range(max(50, a.steps)):
            X.copy_(X0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            eo.cholqr(ctx, X, passes=passes, prec=prec)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        gh, gl = eo.gram(ctx, X, prec=eo.DD)
        orth = float(np.linalg.norm((gh.cpu().numpy() - np.eye(8)) + gl.cpu().numpy(), 2))
        res[name] = {"p50_ms": float(np.percentile(ts, 50)), "p99_ms": float(np.percentile(ts, 99)),
                     "blocks_per_s": 1e3 / float(np.percentile(ts, 50)), "orth_err": orth}
        # the copy and the call captured once in a CUDA graph, replayed per block
        gr = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(dev)
        cap.wait_stream(stream)
        torch.cuda.synchronize()
        with torch.cuda.stream(cap):
            with torch.cuda.graph(gr, stream=cap):
                X.copy_(X0)
                eo.cholqr(ctx, X, passes=passes, prec=prec)
        torch.cuda.synchronize()
        for _ in range(3):
            gr.replay()
        ts = []
        for _ in range(max(50, a.steps)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gr.replay()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        res[name + "_graph"] = {"p50_ms": float(np.percentile(ts, 50)), "p99_ms": float(np.percentile(ts, 99)),
                                "blocks_per_s": 1e3 / float(np.percentile(ts, 50))}
    out = {"metric": SINGLE_METRIC, "n_gpus": ws, "dtype": "f64", "data": "synthetic (synth.single_cholqr)",
           "config": {"workload": "single CholQR, X 100,000 x 8, sigma 1 .. 1e-6", "l2": "L2-warm (6.4 MB)"},
           "results": res}
    if rank == 0:
        print(json.dumps(out), flush=True)


UPDATE_METRIC = "compensated update Q = X R^-1 (one CholQR pass with M given): HBM GB/s per k; p50/p99"


def run_update(a):
    """The row engines alone: one compensated CholQR pass of X (n x k, seeded
    Gaussian on the device) with its Gram matrix given, i.e. the k x k
    factorization and the update Q = X R^-1, which reads and writes X once
    (16 n k algorithmic bytes), restored from a device copy before each
    call (outside the timed region)."""
    import torch
    import paper_1806_01036_gb300 as eo

    ws, rank, local = dist_env()
    dev = torch.device("cuda", local)
    ctx = eo.Context(local)
    stream = torch.cuda.current_stream(dev)
    n = a.n
    res = {}
    for k in [int(t) for t in a.ks.split(",") if t]:
        g = torch.Generator(device=dev).manual_seed(20180604 + 31 * k + rank)
        X0 = torch.randn((k, n), device=dev, dtype=torch.float64, generator=g).t()
        X = torch.empty_like(X0.t()).t()
        mh, ml = eo.gram(ctx, X0, prec=eo.DD)
        ts = []
        for it in range(max(1, a.warmup) + max(3, a.steps)):
            X.copy_(X0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, info = eo.cholqr(ctx, X, passes=1, prec=eo.DD, M=(mh, ml))
            e1.record(stream)
            torch.cuda.synchronize()
            if it >= max(1, a.warmup):
                ts.append(e0.elapsed_time(e1))
        p50 = float(np.percentile(ts, 50))
        res[str(k)] = {"p50_ms": p50, "p99_ms": float(np.percentile(ts, 99)), "gbs": 16 * n * k / p50 / 1e6,
                       "cholesky_info": int(info.item())}
        del X0, X
    out = {"metric": UPDATE_METRIC, "n_gpus": ws, "dtype": "f64", "data": "synthetic (seeded Gaussian on the GPU)",
           "config": {"workload": f"compensated update alone: X {n:,} x k, k in {a.ks}", "n": n},
           "results": res}
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "iterated":
        run_iterated(a)
    elif a.workload == "batched":
        run_batched(a)
    elif a.workload == "serve":
        run_serve(a)
    elif a.workload == "sweep":
        run_sweep(a)
    elif a.workload == "single":
        run_single(a)
    elif a.workload == "update":
        run_update(a)
    else:
        run_eo(a)


if __name__ == "__main__":
    main()
