#!/usr/bin/env python3
"""Benchmark of the overlapping-fragments-method hot path on GB300.

Workload (default): the large lattice, 384x192x192 grid (spacing 0.5 bohr),
~20000 Gaussian wells on 64 self-avoiding chains, 1024 boxes of 40^3 points
on a 16x8x8 lattice of stride 24, 96 states per fragment -- the largest
configuration that runs on one GPU.

Set-up (untimed): V copied in, pair list planned (a2), the fragment states
computed by the library's own batched eigensolver (a0), the assembly
schedule chosen by the library's measuring autotuner.

One step = the assembly of Sec. II from the resident states: H phi on every
dilated box and the operands (a1), every pair block [S_ab | H_ab] on the
tensor cores (a3/a4), the symmetrised FP64 blocks (a5) -- ofm_assemble_HS.
The metric is the pair-block rate: algorithmic pair flops of one assembly
(sum over pairs a<=b of 2 n_a n_b (|B_a∩B_b| + |B_a∩B_b+|)) times the steps
over the device time of the steps (L2 flushed before each step).

e2e: the same metric through the C ABI with host buffers: per step a new
potential from pinned host memory (ofm_set_potential), the assembly, and
every block read back into pinned host memory (ofm_get_blocks).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (pair blocks of seeded states, the rate extrapolated by flops).
Under torchrun every rank runs an independent replica (the method's units
are independent workloads; no collective on the data path).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLUSH_BYTES = 512 << 20   # larger than the 129 MB L2


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="large")
    p.add_argument("--precision", default="bf16x3",
                   help="pair-contraction arithmetic: tf32 bf16 bf16x3 fp32")
    p.add_argument("--no-extras", action="store_true", help="skip e2e, sweeps and the alkane run")
    p.add_argument("--step", default="assembly", choices=["assembly", "full"],
                   help="assembly: a1-a5 from resident states (the headline); full: the whole "
                        "method per step (a2 build, a0 eigensolve, a1-a5, a6 window), for "
                        "workloads whose basis the dense window solver takes")
    return p.parse_args()


HBM_CLASSES = {"apply", "convert", "eig_export", "eig_init", "finalize", "scatter", "filter"}
FP64_CLASSES = {"cholesky", "reduce", "tridiag", "bisect"}


def peaks(measured=None):
    """Roofline denominators: MEASURED_PEAKS.json (driver-written: HBM copy
    bandwidth, cuBLAS BF16 burst and sustained), else the fallback figures;
    FP64 / FP32 / TF32 from this run's own GEMM probes when given."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        pk = {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
              "bf16_tflops_sustained": d.get("bf16_tflops_sustained"), "source": "measured"}
    except Exception:
        pk = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
              "source": "fallback"}
    if measured:
        pk.update(measured)
    return pk


def tensor_peak(pk, precision):
    """Peak of ALGORITHMIC flops for a tensor-core precision: BF16 takes the
    BF16 burst; the hi+lo split issues three BF16 products per credited
    product; TF32 takes this run's measured TF32 GEMM rate when there is one,
    else the BF16 burst times the nominal ratio 1.1/2.25."""
    bf16 = pk["bf16_tflops"]
    if precision == "bf16":
        return bf16, "bf16 burst (measured)" if pk["source"] == "measured" else "bf16 fallback"
    if precision == "bf16x3":
        return bf16 / 3.0, "bf16 burst / 3 (three bf16 products per credited product)"
    if precision == "tf32":
        if pk.get("tf32_tflops"):
            return pk["tf32_tflops"], "tf32 cuBLAS GEMM measured in this run"
        return bf16 * 1.1 / 2.25, "bf16 burst x nominal tf32/bf16 ratio 1.1/2.25"
    if precision == "fp32":
        if pk.get("fp32_tflops"):
            return pk["fp32_tflops"], "fp32 SGEMM measured in this run"
        return None, "fp32 peak not measured"
    if pk.get("fp64_tflops"):
        return pk["fp64_tflops"], "fp64 DGEMM measured in this run"
    return None, "fp64 peak not measured"


def roofline_for(name, s, pk, precision):
    """Roofline of one kernel class: algorithmic bytes or flops per launch
    over its event-timed duration, against the class's bound."""
    ms = s["ms"] / max(1, s["launches"])
    r = {"kernel": name, "row": s["row"], "launches": s["launches"], "ms_per_launch": ms}
    if name == "contract" and precision in ("tf32", "bf16", "bf16x3"):
        per = s["flops"] / max(1, s["launches"])
        per_b = s["bytes"] / max(1, s["launches"])
        tpeak, src = tensor_peak(pk, precision)
        r.update(bound="tensor", unit="TFLOP/s", achieved=per / (ms * 1e-3) / 1e12, peak=tpeak,
                 peak_source=src, algorithmic_flops_per_launch=per,
                 operand_bytes_per_launch=per_b,
                 intensity_flop_per_byte=per / per_b if per_b else None,
                 operand_gbs=per_b / (ms * 1e-3) / 1e9)
    elif name in FP64_CLASSES:
        per = s["flops"] / max(1, s["launches"])
        tpeak, src = tensor_peak(pk, "fp64")
        r.update(bound="alu", unit="TFLOP/s", achieved=per / (ms * 1e-3) / 1e12, peak=tpeak,
                 peak_source=src, algorithmic_flops_per_launch=per)
    elif name in HBM_CLASSES or (s["flops"] == 0 and s["bytes"] > 0):
        per = s["bytes"] / max(1, s["launches"])
        r.update(bound="hbm", unit="GB/s", achieved=per / (ms * 1e-3) / 1e9, peak=pk["hbm_gbs"],
                 peak_source=pk["source"] + " copy bandwidth", algorithmic_bytes_per_launch=per)
    else:
        per = s["flops"] / max(1, s["launches"])
        tpeak, src = tensor_peak(pk, "fp32")
        r.update(bound="alu", unit="TFLOP/s", achieved=per / (ms * 1e-3) / 1e12, peak=tpeak,
                 peak_source=src, algorithmic_flops_per_launch=per)
    r["frac"] = r["achieved"] / r["peak"] if r["peak"] else None
    return r


def profiled_traffic(kernel_class, workload):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    summary is absent, was taken on another workload, or on a different
    version of the kernel."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(path))[kernel_class]
    except Exception:
        return None
    if d.get("workload") != workload:
        return None
    import hashlib
    src = os.path.join(ROOT, "paper_1011_4764_gb300", "csrc", d["source"])
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if sha != d.get("source_sha"):
        return None
    return d.get("dram_bytes_per_launch")


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
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
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------ oracle legs --

def _sample_pairs(wl, count, seed=0):
    """A seeded sample of the workload's pairs (self and neighbour pairs)."""
    import numpy as np
    from paper_1011_4764_gb300 import ofm
    pairs, cnt, _ = ofm.plan_pairs(wl.grid, wl.frags)
    rng = np.random.default_rng(seed)
    pick = sorted(rng.choice(len(pairs), size=min(count, len(pairs)), replace=False).tolist())
    return [pairs[i] for i in pick], [tuple(cnt[i]) for i in pick]


def _oracle_pairs(args):
    """Worker: the oracle's pair blocks for `pairs` of the workload on seeded
    random states, `reps` times; returns the seconds of each repetition."""
    grid, frags, vpath, pairs, reps = args
    import numpy as np
    from ofm_inputs import random_states
    from oracle import ofm_oracle as O
    H = O.hamiltonian(grid, np.load(vpath, mmap_mode="r"))
    states = {}
    for a, b in pairs:
        for f in (a, b):
            if f not in states:
                states[f] = random_states(grid, frags[f], seed=1000 + f)
    out = []
    for _ in range(reps):
        t0 = time.perf_counter()
        for a, b in pairs:
            O.pair_block(H, grid, frags[a], states[a], frags[b], states[b])
        out.append(time.perf_counter() - t0)
    return out


def oracle_sample(name, npairs, workers, reps=1):
    """The FP64 oracle, as it stands, on `npairs` seeded sampled pair blocks
    of the workload, spread over `workers` single-threaded processes
    (spawned; each builds the sparse H once, untimed).  Returns (sampled pair
    flops, per repetition the seconds of the slowest worker, workers)."""
    import multiprocessing as mp
    import numpy as np
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    from ofm_inputs import make_workload
    wl = make_workload(name)
    pairs, cnt = _sample_pairs(wl, npairs)
    F = sum(2 * wl.frags[a].n_states * wl.frags[b].n_states * (ks + kh)
            for (a, b), (ks, kh) in zip(pairs, cnt))
    w = max(1, min(workers, len(pairs)))
    chunks = [pairs[i::w] for i in range(w)]
    with tempfile.TemporaryDirectory() as tmp:
        vpath = os.path.join(tmp, "V.npy")
        np.save(vpath, np.ascontiguousarray(wl.V))
        with mp.get_context("spawn").Pool(w) as pool:
            secs = pool.map(_oracle_pairs, [(wl.grid, wl.frags, vpath, c, reps) for c in chunks])
    per_rep = [max(s[r] for s in secs) for r in range(reps)]
    return F, per_rep, w


def cpu_baseline_leg(name, npairs=64):
    cores = os.cpu_count() or 1
    F, per_rep, w = oracle_sample(name, npairs, cores)
    dt = per_rep[0]
    return {"value": F / dt / 1e12, "unit": "TFLOP/s", "cores": w, "kind": "oracle",
            "sample": f"{npairs} seeded sampled pair blocks of {name} on seeded random states, "
                      f"{w} single-threaded processes; {F:.3e} pair flops in {dt:.1f} s (the slowest "
                      f"process, pair blocks only, the sparse H built beforehand); extrapolated: "
                      f"the rate is carried by flops to the whole workload"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    npairs = max(1, min(cores, 16))
    F, per_rep, w = oracle_sample(args.workload, npairs, cores, reps=args.warmup + args.steps)
    times = per_rep[args.warmup:] or per_rep
    t = sum(times) / len(times)
    val = F / t / 1e12
    name = _workload_name(args.workload)
    out = {
        "impl": "reference", "metric": "H/S pair-block TFLOP/s", "value": val, "unit": "TFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "sample_pairs": npairs},
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": w, "kind": "oracle",
                         "sample": f"{npairs} seeded sampled pair blocks of {name} per step on "
                                   f"seeded random states, {w} processes, rate extrapolated by flops"},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def _workload_name(key):
    return {"large": "large_lattice_384x192x192", "alkane": "alkane_chain_256x32x32",
            "polymer": "amorphous_polymer_128c", "scaled": "chains_scaled_192c",
            "tiny": "tiny_32x12x12"}.get(key, key)


# ---------------------------------------------------------------- our arm --

def job_time_ms(t_ms, dist, device):
    """The slowest rank's timed-region milliseconds (every rank calls this;
    dist None: one process)."""
    if dist is None:
        return float(t_ms)
    import torch
    t = torch.tensor([float(t_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, flops_per_step, steps, t_ms):
    """Whole-job TFLOP/s: the pair flops every rank's replica computed in its
    K steps over the slowest rank's time."""
    return world * flops_per_step * steps / (t_ms * 1e-3) / 1e12


def gemm_peaks(dev):
    """FP64, FP32 (no TF32) and TF32 dense GEMM rates of this GPU (cuBLAS via
    torch), the denominators of the FP64 / FP32 / TF32 fractions."""
    import torch
    out = {}
    for key, dtype, tf32, n in (("fp64_tflops", torch.float64, False, 4096),
                                ("fp32_tflops", torch.float32, False, 8192),
                                ("tf32_tflops", torch.float32, True, 8192)):
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = tf32
        try:
            a = torch.randn(n, n, device=dev, dtype=dtype)
            b = torch.randn(n, n, device=dev, dtype=dtype)
            for _ in range(2):
                a @ b
            torch.cuda.synchronize(dev)
            reps = 5
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                a @ b
            e1.record()
            e1.synchronize()
            out[key] = 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12
        finally:
            torch.backends.cuda.matmul.allow_tf32 = prev
        del a, b
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else torch.cuda.current_device())

    from ofm_inputs import make_workload
    from paper_1011_4764_gb300 import build
    build.build()
    from paper_1011_4764_gb300 import ofm

    wl = make_workload(args.workload)
    grid, frags = wl.grid, wl.frags
    prec = args.precision
    stream = torch.cuda.Stream(device=dev)
    ctx = ofm.Context(stream)
    V_dev = torch.from_numpy(np.ascontiguousarray(wl.V)).to(dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # ---- set-up: pairs, the fragment states from the library's eigensolver,
    # the assembly schedule from its autotuner
    t_setup = time.perf_counter()
    ctx.build_fragments(grid, V_dev, frags, storage="fp32")
    info = ctx.plan_info()
    F = info["pair_flops"]
    eps, res, eig_status = ctx.fragment_eigs(allow_not_converged=True)
    eig_s = time.perf_counter() - t_setup
    t_chunk, t_form, t_ms, t_times = ctx.autotune_assembly(prec, reps=3)
    schedule = {"schedule": ctx.tuned["schedule"], "region_ms": ctx.tuned["region_ms"],
                "pair_best_ms": float(np.min(t_times[t_times > 0])) if np.any(t_times > 0) else None,
                "pair_chunk_points": t_chunk,
                "pair_stencil_form": ["register", "staged"][t_form - 1]}
    setup_s = time.perf_counter() - t_setup

    if args.step == "full":
        rule = wl.window
        if rule is None or rule.kind != "above_gap" or info["basis_size"] > 12800:
            raise SystemExit("--step full needs an above-gap window and a basis of at most 12800")

        def step():
            ctx.build_fragments(grid, V_dev, frags, storage="fp32")
            ctx.fragment_eigs()
            ctx.assemble(prec)
            ctx.window_from_index(rule.n_occ, rule.width)
    else:
        def step():
            ctx.assemble(prec)

    for _ in range(args.warmup):
        step()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed_steps(profile):
        """K steps, L2 flushed before each (untimed), timed with CUDA events
        on the library stream; with profile=True the library also brackets
        every kernel class with events (per-class durations)."""
        ctx.set_profiling(profile)
        launches0 = sum(v["launches"] for v in ctx.kernel_stats().values())
        ms = []
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        launches = sum(v["launches"] for v in ctx.kernel_stats().values()) - launches0
        st = ctx.kernel_stats() if profile else None
        ctx.set_profiling(False)
        return ms, launches, st

    # ---- timed region
    clocks = ClockSampler(local if world > 1 else dev.index or 0)
    barrier()
    clocks.start()
    t_wall0 = time.perf_counter()
    step_ms, timed_launches, _ = timed_steps(False)
    barrier()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    # ---- the same K steps with per-class CUDA events: rows and rooflines
    barrier()
    prof_ms, _, stats = timed_steps(True)
    barrier()
    t_ms = job_time_ms(sum(step_ms), dist, dev)
    K = args.steps
    value = job_value(world, F, K, t_ms)

    measured = gemm_peaks(dev) if rank == 0 else {}
    pk = peaks(measured)
    dom_name, dom = max(stats.items(), key=lambda kv: kv[1]["ms"])
    roof = roofline_for(dom_name, dom, pk, prec)
    roof["traffic"] = profiled_traffic(dom_name, wl.name)
    others = {k: roofline_for(k, s, pk, prec) for k, s in stats.items() if k != dom_name}
    for k in others:
        others[k]["traffic"] = profiled_traffic(k, wl.name)
    rows = {}
    for name, s in stats.items():
        rows[s["row"]] = rows.get(s["row"], 0.0) + s["ms"] / K

    out = {
        "metric": "H/S pair-block TFLOP/s", "value": value, "unit": "TFLOP/s",
        "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": t_ms / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32", "tf32": "tf32", "bf16": "bf16",
                  "bf16x3": "bf16x3"}[prec],
        "data": "synthetic",
        "config": {"workload": wl.name, "grid": list(grid.n), "h": grid.h,
                   "fragments": len(frags), "states": sorted({f.n_states for f in frags}),
                   "pairs": info["n_pairs"], "basis": info["basis_size"], "pair_flops": F,
                   "contraction": prec, "storage": "fp32",
                   "step": ("a1 H apply + operands, a3/a4 pair contraction, a5 FP64 blocks "
                            "(ofm_assemble_HS) from resident states") if args.step == "assembly" else
                           ("a2 build + a0 eigensolve + a1-a5 assembly + a6 window above the gap "
                            "(the whole method)"),
                   "states_from": "the library's batched fragment eigensolver, run once untimed "
                                  f"({eig_s:.1f} s with the pair planning; status "
                                  f"{ofm.status_name(eig_status)}, max residual {float(res.max()):.2e})",
                   "schedule": schedule["schedule"],
                   "l2": "flushed by a 512 MiB device write before every step (untimed)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "value_profiled": job_value(world, F, K, sum(prof_ms)),
        "profile_pass": "rows_ms, kernels, roofline and rooflines come from a second pass of the same "
                        "K steps with per-class CUDA events (value_profiled is its throughput); value "
                        "and gpu_launches come from the unprofiled timed pass",
        "rows_ms": {k: round(v, 4) for k, v in sorted(rows.items())},
        "kernels": {k: {"row": s["row"], "launches": s["launches"] // K, "ms": s["ms"] / K}
                    for k, s in sorted(stats.items())},
        "assembly_schedule": schedule,
        "setup_s": setup_s,
        "wall_s": wall,
        "gpu_launches": timed_launches,
        "roofline": roof,
        "rooflines": others,
        "peaks": {k: v for k, v in pk.items()},
        "clocks": clk,
    }
    if not args.no_extras and rank == 0:
        out.update(extras(args, ctx, ofm, wl, stream, F, dev, prec))
    ctx.close()
    del ctx
    torch.cuda.empty_cache()
    if not args.no_extras and rank == 0:
        try:
            out["alkane_chain"] = alkane_extra(ofm, stream, dev)
        except Exception as e:  # an extra must not hide the headline line
            out["alkane_chain"] = {"error": str(e)}
        try:
            out["amorphous_polymer"] = polymer_extra(ofm, stream, dev)
        except Exception as e:
            out["amorphous_polymer"] = {"error": str(e)}
    if rank == 0:
        if world == 1 and not args.no_extras:
            try:
                out["cpu_baseline"] = cpu_baseline_leg(args.workload)
            except Exception as e:
                out["cpu_baseline"] = {"value": None, "unit": "TFLOP/s", "cores": 0,
                                       "kind": "oracle", "sample": f"failed: {e}"}
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def _time_assembly(ctx, stream, prec, schedule="auto", reps=5):
    import torch
    ctx.assemble(prec, schedule=schedule)
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.assemble(prec, schedule=schedule)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return min(ts)


def extras(args, ctx, ofm, wl, stream, F, dev, prec):
    import numpy as np
    import torch
    ex = {}
    # e2e: a new potential from pinned host memory, the assembly, every block
    # read back into pinned host memory, through the C ABI
    try:
        V_host = torch.from_numpy(np.ascontiguousarray(wl.V)).pin_memory()
        nblk = ctx.blocks_count()
        out_host = torch.empty(nblk, dtype=torch.float64).pin_memory()
        n_e2e = max(3, min(args.steps, 5))
        ctx.set_potential(V_host)
        ctx.assemble(prec)
        ctx.get_blocks(out_host)
        torch.cuda.synchronize(dev)
        # synchronous read-back: each step waits for its blocks
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            ctx.set_potential(V_host)
            ctx.assemble(prec)
            ctx.get_blocks(out_host)
        torch.cuda.synchronize(dev)
        dt_sync = (time.perf_counter() - t0) / n_e2e
        # pipelined read-back: step k's blocks travel to the host while step
        # k + 1 is assembled; the timed region ends when the last step's
        # blocks are in host memory
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            ctx.set_potential(V_host)
            ctx.assemble(prec)
            ctx.get_blocks_async(out_host)
        ctx.sync_blocks()
        torch.cuda.synchronize(dev)
        dt = (time.perf_counter() - t0) / n_e2e
        ex["e2e"] = {"value": F / dt_sync / 1e12, "unit": "TFLOP/s",
                     "h2d_bytes_per_step": int(V_host.numel() * 8),
                     "d2h_bytes_per_step": int(nblk * 8), "steps": n_e2e,
                     "timer": "host wall clock",
                     "step": "ofm_set_potential (pinned host V) + ofm_assemble_HS + ofm_get_blocks "
                             "(every [H_ab | S_ab] block into pinned host memory)",
                     "pipelined_read_back": {
                         "value": F / dt / 1e12,
                         "step": "the same with ofm_get_blocks_async (each step's blocks travel "
                                 "while the next step is assembled) and ofm_sync_blocks after "
                                 "the last step"}}
    except Exception as e:
        ex["e2e"] = {"error": str(e)}
    # contraction arithmetic and schedule on the same states: a1-a5 device time
    asm = {}
    # (the FP32 / FP64 plain forms on the CUDA cores take the same region
    # plan; FP64 last, it doubles the operand planes and partial slots)
    for p in ("bf16x3", "bf16", "tf32", "fp32", "fp64"):
        try:
            asm[p] = _time_assembly(ctx, stream, p, reps=1 if p == "fp64" else 5)
        except ofm.OFMError as e:
            asm[p] = str(e)
    ex["assembly_ms_by_precision"] = asm
    for plain in ("fp32", "fp64"):
        if isinstance(asm.get(plain), float):
            ex[f"speedup_vs_{plain}_cuda_cores"] = {p: asm[plain] / t for p, t in asm.items()
                                                   if isinstance(t, float)}
    sch = {}
    for s in ("pair", "region"):
        try:
            sch[s] = _time_assembly(ctx, stream, prec, schedule=s, reps=3)
        except ofm.OFMError as e:
            sch[s] = str(e)
    ex["assembly_ms_by_schedule"] = sch
    ctx.assemble(prec)
    return ex


def alkane_extra(ofm, stream, dev):
    """The alkane chain (256x32x32, 31 boxes, 32 states): the whole method
    per step (a0 eigensolve + a1-a5 + a6 window), and each window
    eigenvalue's error against the FP64 oracle's spectrum of the same
    workload (tests/golden/alkane_oracle.json, written by the oracle) for
    every contraction arithmetic, on the GPU's own states."""
    import numpy as np
    import torch
    from ofm_inputs import make_workload
    wl = make_workload("alkane")
    rule = wl.window
    golden = json.load(open(os.path.join(ROOT, "tests", "golden", "alkane_oracle.json")))
    Eo = np.array(golden["ofm_spectrum"])
    i0 = rule.n_occ
    m = int(np.sum((Eo >= Eo[i0]) & (Eo <= Eo[i0] + rule.width)))
    res = {"workload": wl.name, "window": f"E_{i0 + 1} .. E_{i0 + 1} + {rule.width} Ha",
           "window_count_oracle": m}
    ctx = ofm.Context(stream)
    V_dev = torch.from_numpy(np.ascontiguousarray(wl.V)).to(dev)

    def full_step():
        ctx.build_fragments(wl.grid, V_dev, wl.frags, storage="fp32")
        ctx.fragment_eigs()
        ctx.assemble("bf16x3")
        return ctx.window_from_index(i0, rule.width)

    full_step()
    ts = []
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        E, n = full_step()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    F = ctx.plan_info()["pair_flops"]
    res["full_step_ms"] = min(ts)
    res["full_step_tflops"] = F / min(ts) / 1e9
    res["window_count"] = n
    # the block-sparse pencil product Y = H X (ofm_pencil_apply) with one
    # column per window eigenvalue: device time and achieved bandwidth
    try:
        nb = ctx.plan_info()["basis_size"]
        with torch.cuda.stream(stream):
            X = torch.randn((max(1, m), nb), dtype=torch.float64, device=dev)
            Y = torch.empty_like(X)
        stream.synchronize()
        ctx.pencil_apply("H", X, Y)
        ctx.set_profiling(True)
        for _ in range(5):
            ctx.pencil_apply("H", X, Y)
        st = ctx.kernel_stats()["pencil"]
        ctx.set_profiling(False)
        ms = st["ms"] / st["launches"]
        res["pencil_apply"] = {"columns": int(X.shape[0]), "ms": ms,
                               "achieved_gbs": st["bytes"] / st["launches"] / (ms * 1e-3) / 1e9,
                               "achieved_tflops_fp64": st["flops"] / st["launches"] / (ms * 1e-3) / 1e12,
                               "bytes_per_launch": st["bytes"] / st["launches"]}
    except Exception as e:
        res["pencil_apply"] = {"error": str(e)}
    errs = {}
    for p in ("bf16x3", "tf32", "bf16", "fp32"):
        ctx.assemble(p)
        got = ctx.eigs_by_index(i0, i0 + m)
        d = got - Eo[i0:i0 + m]
        errs[p] = {"max_abs_ha": float(np.max(np.abs(d))), "mean_abs_ha": float(np.mean(np.abs(d))),
                   "per_eigenvalue_ha": [float(f"{x:.3e}") for x in d]}
    ctx.close()
    # the all-FP64 path: FP64 states (FP64 eigensolve) and FP64 contraction
    c64 = ofm.Context(stream)
    c64.build_fragments(wl.grid, V_dev, wl.frags, storage="fp64")
    c64.fragment_eigs()
    c64.assemble("fp64")
    got = c64.eigs_by_index(i0, i0 + m)
    d = got - Eo[i0:i0 + m]
    errs["fp64"] = {"max_abs_ha": float(np.max(np.abs(d))), "mean_abs_ha": float(np.mean(np.abs(d))),
                    "per_eigenvalue_ha": [float(f"{x:.3e}") for x in d]}
    c64.close()
    res["window_error_vs_oracle"] = errs
    return res


def _errs(got, ref):
    import numpy as np
    d = got - ref
    return {"max_abs_ha": float(np.max(np.abs(d))), "mean_abs_ha": float(np.mean(np.abs(d))),
            "per_eigenvalue_ha": [float(f"{x:.3e}") for x in d]}


def polymer_extra(ofm, stream, dev):
    """The amorphous polymer (128^3 grid, 56 uneven boxes 16^3..40^3, 8-64
    states, basis 2033) end to end from the GPU's own states: FP64 storage,
    eigensolve, assembly and window (timed, and each window eigenvalue
    against the FP64 oracle's spectrum in tests/golden/polymer_oracle.json);
    then every contraction arithmetic on FP32 states, where the pencil's
    nearly singular S (lambda_min 2e-9 in the oracle) decides the outcome."""
    import numpy as np
    import torch
    from ofm_inputs import make_workload
    wl = make_workload("polymer")
    rule = wl.window
    golden = json.load(open(os.path.join(ROOT, "tests", "golden", "polymer_oracle.json")))
    Eo = np.array(golden["ofm_spectrum"])
    i0 = rule.n_occ
    m = int(np.sum((Eo >= Eo[i0]) & (Eo <= Eo[i0] + rule.width)))
    res = {"workload": wl.name, "boxes": len(wl.frags), "basis": int(len(Eo)),
           "window": f"E_{i0 + 1} .. E_{i0 + 1} + {rule.width} Ha", "window_count_oracle": m,
           "S_min_eig_oracle": golden["S_min_eig"]}
    V_dev = torch.from_numpy(np.ascontiguousarray(wl.V)).to(dev)
    ctx = ofm.Context(stream)

    def full_step():
        ctx.build_fragments(wl.grid, V_dev, wl.frags, storage="fp64")
        ctx.fragment_eigs()
        ctx.assemble("fp64")
        return ctx.window_from_index(i0, rule.width, max_out=len(Eo))

    full_step()
    ts = []
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        E, n = full_step()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    res["fp64_full_step_ms"] = min(ts)
    res["window_count"] = int(n)
    res["window_error_vs_oracle"] = {"fp64": _errs(ctx.eigs_by_index(i0, i0 + m), Eo[i0:i0 + m])}
    ctx.close()
    c32 = ofm.Context(stream)
    c32.build_fragments(wl.grid, V_dev, wl.frags, storage="fp32")
    _, r32, st32 = c32.fragment_eigs(allow_not_converged=True)
    res["fp32_states"] = {"eigensolver_status": ofm.status_name(st32),
                          "max_residual": float(r32.max())}
    for p in ("bf16x3", "tf32", "bf16", "fp32", "fp64"):
        try:
            c32.assemble(p)
            res["window_error_vs_oracle"][f"{p}_on_fp32_states"] = _errs(
                c32.eigs_by_index(i0, i0 + m), Eo[i0:i0 + m])
        except ofm.OFMError as e:
            res["window_error_vs_oracle"][f"{p}_on_fp32_states"] = {"status": str(e)}
    c32.close()
    return res


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
