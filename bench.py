#!/usr/bin/env python
"""Benchmark: power-flow solves per second of the tensor power flow on one GB300 per rank.

Workload (default): a 1,000-bus synthetic radial feeder (999 PQ buses) and one year of one-minute
load columns (T = 525,600), solved to max |dV| <= 1e-10 pu from a flat start.  One "step" is one
full tpf_solve of all T columns.  ``--method sparse`` (default) is the sparse formulation
(Algorithm 2): one launch, each column's whole sweep loop on chip, FP32 sweeps with double-float
anchors.  ``--method dense`` is Algorithm 1's dense product on the tensor cores (fp16 operands,
FP32 accumulation, residual form).  Both return results within 1e-8 pu of the FP64 oracle.

Reported on one JSON line (rank 0):
  value       PF/s, device-resident inputs (S, V on the GPU), CUDA events around the K steps,
              max over ranks; rank r solves its own year of loads of the same feeder (load seed
              = feeder seed + r), so N ranks solve N x columns with no exchange (weak scaling)
  e2e         PF/s through tpf_solve_host with pinned HOST buffers: H2D of S, solve, D2H of V,
              iteration counts and mismatches inside the timed region
  roofline    the headline path's dominant kernel: mx_tree (sparse; FP32 flops over the derived
              FP32 peak) or tc_gemm (dense; 8 n^2 flops per iterating column per sweep over the
              measured bf16 peak)
  dense_method / sparse_method   the other formulation on the same workload, with its roofline
  fp64_gpu    the plain FP64 GPU fixed-point iteration (direct form), timed on a column sample
  cpu_baseline the CPU oracle on the host cores, on a bounded column sample; the same leg checks
              the GPU results against the oracle (iterated to 1e-13) on sampled columns
  cpu_newton_raphson  the oracle's sparse Newton-Raphson on 16 sampled columns, one core (context
              for the paper's NR comparison)
  learned_start  config-5 leg: the MLP warm start on a 200-bus feeder
  scenario_tensor  config-3 leg: 500-bus feeder, [200 x 8,760] complex64 scenario tensor with fused
              voltage-band statistics
  feeder_batch  config-4 leg: 4,096 feeders of 20-2,000 buses in one tpf_solve_batch call
  zip_loads   the headline workload with ZIP loads (Eq. 3) on the sparse formulation
  three_phase a 500-bus three-phase feeder (Eq. 1 with phases = 3) on the sparse formulation
  large_feeder the paper's largest grid, 5,000 buses, over the one-minute year (16 buses per thread)
  table1_100_bus Table I's 100-bus row: 100-bus feeder over the one-minute year, with the paper's times
  small_feeder config-1 leg: 34-bus feeder over one day (1,440 columns), FP64 and both mixed
              formulations, CUDA-event and launch-inclusive host time per call, every column checked
  clocks      nvidia-smi samples taken during the timed region

``--impl reference`` times the CPU oracle as the reference arm on the same workload.
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

METRIC = "PF solves/s at ≤1e-8 pu vs FP64 oracle: mixed+learned-start vs plain FP64 FPI"

# dram__bytes_read.sum + dram__bytes_write.sum of one tc_gemm launch from an ncu capture of the
# 1,000-bus feeder over 16,384 columns (203.8 MB + 77.4 MB), per iterating column; scaled by the
# columns each launch of this run processes.  None once the kernel has changed since the capture.
GEMM_TRAFFIC_BYTES_PER_COLUMN = (203.764224e6 + 77.426432e6) / 16384
# The same for the sparse tree kernel mx_tree started from the learned prediction (the headline
# step's solve): 1,313.1 MB read (S and the half-precision prediction) + 1,002.8 MB written for
# 65,536 columns of the 1,000-bus feeder.
TREE_TRAFFIC_BYTES_PER_COLUMN = (1313.136e6 + 1002.844e6) / 65536
# From the flat start: 262.2 MB read + 210.6 MB written for the first 16,384 columns of the year.
TREE_FLAT_TRAFFIC_BYTES_PER_COLUMN = (262.154496e6 + 210.563328e6) / 16384
# Algorithmic FP32 flop per bus per sweep of the tree formulation: load current conj(S/V) 12,
# prefix sum 2, subtree difference 2, z L 6, subtree-end subtraction 2, path prefix 2, update 4,
# |step|^2 and max 6.
TREE_FLOPS_PER_BUS_SWEEP = 36


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--buses", type=int, default=1000)
    p.add_argument("--columns", type=int, default=525600)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--tol", type=float, default=1e-10)
    p.add_argument("--fp64-sample", type=int, default=8192)
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--check-columns", type=int, default=10000)
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-learned", action="store_true")
    p.add_argument("--method", choices=["sparse", "dense"], default="sparse")
    p.add_argument("--no-scenario", action="store_true")
    p.add_argument("--no-zip", action="store_true")
    p.add_argument("--no-poly", action="store_true")
    p.add_argument("--ref-seconds", type=float, default=120.0, help="reference arm: seconds for all its steps")
    p.add_argument("--poly-buses", type=int, default=500)
    p.add_argument("--poly-columns", type=int, default=65536)
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--no-large", action="store_true")
    p.add_argument("--no-small", action="store_true", help="skip the 34-bus one-day (1,440-column) case")
    p.add_argument("--no-table1", action="store_true", help="skip the 100-bus one-year case of Table I")
    p.add_argument("--large-buses", type=int, default=5000)
    p.add_argument("--large-columns", type=int, default=525600)
    p.add_argument("--scen", type=int, default=200)
    p.add_argument("--hours", type=int, default=8760)
    p.add_argument("--scen-buses", type=int, default=500)
    p.add_argument("--batch-feeders", type=int, default=4096)
    p.add_argument("--no-other", action="store_true", help="skip timing the other formulation")
    p.add_argument("--headline", choices=["learned", "flat"], default="learned",
                   help="the headline step: learned-start solve (prediction + warm solve) or flat start")
    p.add_argument("--train-columns", type=int, default=100000)
    p.add_argument("--epochs", type=int, default=100)
    return p.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def allmax(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(args):
    from paper_2403_04578_gb300 import inputs as G

    f = G.make_feeder(args.buses, args.seed)
    return f, {
        "workload": f"{args.buses}-bus radial feeder x {args.columns:,} one-minute load columns (one year); "
                    f"flat start, per-column stop at max|dV| <= {args.tol:g} pu",
        "buses": args.buses,
        "pq_buses": f.n_pq,
        "columns": args.columns,
        "feeder_seed": args.seed,
        "load_scale": round(f.load_scale, 6),
        "l2": "no flush: S alone is %.1f GB, far above the 129 MB L2" % (args.columns * f.n_pq * 16 / 1e9),
    }


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def check_columns(args, full_T):
    """The evenly spaced columns of the year on which GPU results are checked against the oracle."""
    return np.linspace(0, full_T - 1, min(args.check_columns, full_T)).astype(np.int64)


def cpu_oracle_leg(f, S_host, args, full_T, cc=None, it_main=None, V_checks=None):
    """Time the CPU oracle on a bounded column sample, and check GPU results against it.

    cc: the checked columns; V_checks: {name: V of those columns from a GPU path} (the first is the
    headline's, whose iteration counts it_main are compared too)."""
    from oracle import oracle as O

    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    case = O.Case.from_feeder(f)
    t_setup = time.perf_counter() - t0
    # Probe the per-column cost, then size the sample to about args.cpu_seconds.
    probe_cols = np.linspace(0, full_T - 1, 4 * threads).astype(np.int64)
    t0 = time.perf_counter()
    case.solve(S_host[probe_cols], tol=args.tol, threads=threads)
    per_col = (time.perf_counter() - t0) / probe_cols.size
    n_cols = int(min(full_T, max(probe_cols.size, args.cpu_seconds / max(per_col, 1e-9))))
    cols = np.linspace(0, full_T - 1, n_cols).astype(np.int64)
    t0 = time.perf_counter()
    case.solve(S_host[cols], tol=args.tol, threads=threads)
    dt = time.perf_counter() - t0
    out = {"value": n_cols / dt, "unit": "PF/s", "cores": threads, "kind": "oracle",
           "sample": f"{n_cols} columns evenly spaced over the {full_T:,}-column year, same feeder and tol; "
                     f"K = -Y_dd^-1 setup {t_setup:.1f} s not included"}
    check = {}
    if V_checks:
        Vt, _, _ = case.solve(S_host[cc], tol=1e-13, threads=threads)
        _, it_ref, _ = case.solve(S_host[cc], tol=args.tol, threads=threads)
        for k, (name, Vs) in enumerate(V_checks.items()):
            if Vs is None:
                continue
            check[name] = float(np.abs(Vs - Vt).max())
        check["columns_checked"] = int(cc.size)
        if it_main is not None:
            check["iters_equal_frac"] = float(np.mean(it_main == it_ref))
            check["iters_diff_max"] = int(np.abs(it_main - it_ref).max())
    return out, check


def cpu_newton_leg(f, S_host, full_T, columns=16):
    """The oracle's sparse polar Newton-Raphson (SciPy sparse LU, one core, flat start, power
    mismatch <= 1e-10 pu) on a few columns of the same workload: context for the paper's comparison
    with NR (Sec. V), not a target."""
    from oracle import oracle as O

    Y = O.ybus(f.n_bus, f.from_bus, f.to_bus, f.z_pu)
    case = O.Case.from_feeder(f)
    cols = np.linspace(0, full_T - 1, columns).astype(np.int64)
    t0 = time.perf_counter()
    res = [O.nr_solve(Y, f.slack, f.v0, f.pq_bus, S_host[k], tol=1e-10) for k in cols]
    dt = time.perf_counter() - t0
    Vt, _, _ = case.solve(S_host[cols], tol=1e-13)
    err = max(float(np.abs(r[0] - Vt[i]).max()) for i, r in enumerate(res))
    return {"value": cols.size / dt, "unit": "PF/s", "cores": 1, "kind": "sparse Newton-Raphson (oracle)",
            "sample": f"{cols.size} columns evenly spaced over the {full_T:,}-column year, flat start, "
                      "power mismatch <= 1e-10 pu",
            "converged": int(sum(bool(r[2]) for r in res)), "mean_iterations": float(np.mean([r[1] for r in res])),
            "max_abs_err_pu_vs_fpi_oracle": err}


def train_start_network(f, fd, args, dev, n_train, epochs, seed_offset=100, hidden=256, layers=3):
    """The learned start's network for feeder f (`layers` hidden layers of `hidden` units): n_train
    columns of another load draw (seed + seed_offset, drawn on the device), solved by the library
    (sparse, mixed, tol), then `epochs` epochs of Adam on batches of 1,024 with a cosine learning
    rate from 1e-3 down to 1e-4."""
    import torch

    from paper_2403_04578_gb300 import inputs as G
    from paper_2403_04578_gb300 import tpf

    S_tr = G.load_tensor_device(f, n_train, args.seed + seed_offset, dev)
    V_tr, _, _, st = fd.solve(S_tr, precision="mixed", tol=args.tol, method="sparse")
    net = tpf.LearnedStart(f.n_pq, hidden=hidden, hidden_layers=layers, max_batch=1024, seed=args.seed)
    net.fit_normalization(S_tr, V_tr)
    B = 1024
    steps_per_epoch = n_train // B
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    perm_gen = torch.Generator(device="cpu").manual_seed(args.seed)
    for ep in range(epochs):
        lr = 1e-3 * (0.5 * (1 + np.cos(np.pi * ep / epochs)) * 0.9 + 0.1)
        order = torch.randperm(n_train, generator=perm_gen)[: steps_per_epoch * B].to(dev)
        Sp, Vp = S_tr[order].contiguous(), V_tr[order].contiguous()
        for k in range(steps_per_epoch):
            net.train_step(Sp[k * B:(k + 1) * B], Vp[k * B:(k + 1) * B], lr=lr, want_loss=False)
    loss = net.train_step(S_tr[:B], V_tr[:B], lr=1e-12)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del S_tr, V_tr
    torch.cuda.empty_cache()
    return net, {"train_columns": n_train, "epochs": epochs, "train_seconds": train_s, "final_batch_loss": loss,
                 "network": "-".join([str(2 * f.n_pq)] + [str(hidden)] * layers + [str(2 * f.n_pq)]) +
                            ", GELU, BF16 tensor-core products"}


def learned_e2e(fd, net, Sh, Vh, ith, mmh, args, world):
    """The learned-start solve end to end through the public host-buffer entry point
    (tpf_solve_learned_host): pinned host loads in, pinned V, iteration counts and mismatches out;
    the library pipelines the host-to-device copies, the chunked predictions and solves, and the
    copies back."""
    T, n = Sh.shape

    def one():
        fd.solve_learned_host(net, Sh, tol=args.tol, out=(Vh, ith, mmh))

    one()
    one()  # two warm-up passes: the first touches of the pinned pages and the copy engines' queues
    steps = max(1, args.steps)
    barrier(world)
    t0 = time.perf_counter()
    step_ms = []
    for _ in range(steps):
        ts = time.perf_counter()
        one()
        step_ms.append((time.perf_counter() - ts) * 1e3)
    dt = allmax(world, (time.perf_counter() - t0) / steps)
    return {"value": world * T / dt, "unit": "PF/s", "h2d_bytes_per_step": T * n * 16,
            "d2h_bytes_per_step": T * n * 16 + T * 4 + T * 8, "ms_per_step": dt * 1e3,
            "step_ms": [round(x, 2) for x in step_ms],
            "entry_point": "tpf_solve_learned_host (pinned host buffers; up to 32 chunks pipelined in the library)"}


def learned_start_leg(args, stream):
    """Config 5: a 200-bus feeder, the network trained on 100,000 columns solved by the library, then
    525,600 unseen columns solved by the learned-start solve (fused prediction + warm sparse solve)
    against the flat start (both mixed, sparse formulation, tol as the headline), and the plain FP64
    GPU path from the flat start on a column sample."""
    import torch

    from paper_2403_04578_gb300 import inputs as G
    from paper_2403_04578_gb300 import tpf

    dev = torch.device("cuda", torch.cuda.current_device())
    f = G.make_feeder(200, args.seed)
    fd = tpf.Feeder.from_inputs(f)
    n_eval = args.columns
    net, train_info = train_start_network(f, fd, args, dev, 100_000, args.epochs)
    S_ev = G.load_tensor_device(f, n_eval, args.seed + 200, dev)
    V = torch.empty_like(S_ev)
    it = torch.empty(n_eval, dtype=torch.int32, device=dev)
    mm = torch.empty(n_eval, dtype=torch.float64, device=dev)
    fb = [0]

    def learned():
        fb[0] = fd.solve_learned(net, S_ev, V, it, mm, tol=args.tol)[3]

    ms_learned = timed_device(learned, 3, stream)
    it_learned = it.float().mean().item()
    V_learned = V.cpu().numpy()
    ms_predict = timed_device(lambda: net.predict(S_ev, V), 3, stream)
    ms_flat = timed_device(lambda: fd.solve(S_ev, V, it, mm, precision="mixed", tol=args.tol, start="flat",
                                            method="sparse"), 3, stream)
    it_flat = it.float().mean().item()
    F = min(args.fp64_sample, n_eval)
    Sf = S_ev[:F].contiguous()
    ms_fp64 = timed_device(lambda: fd.solve(Sf, precision="fp64", tol=args.tol), 2, stream)
    out = {
        "workload": f"200-bus feeder, network {2 * f.n_pq}-256-256-256-{2 * f.n_pq} (GELU, BF16), trained "
                    f"{train_info['epochs']} epochs on {train_info['train_columns']:,} library-solved columns; "
                    f"evaluated on {n_eval:,} unseen columns",
        "value": n_eval / (ms_learned / 1e3), "unit": "PF/s", "method": "tpf_solve_learned (sparse, warm start)",
        "ms_per_step": ms_learned, "predict_ms_complex128": ms_predict,
        "flat_start_mixed": n_eval / (ms_flat / 1e3), "flat_ms_per_step": ms_flat,
        "speedup_learned_vs_flat": ms_flat / ms_learned,
        "plain_fp64_gpu": F / (ms_fp64 / 1e3),
        "speedup_vs_plain_fp64": (n_eval / (ms_learned / 1e3)) / (F / (ms_fp64 / 1e3)),
        "mean_sweeps_learned": it_learned, "mean_sweeps_flat": it_flat, "fallback_columns": fb[0],
        **{k: v for k, v in train_info.items() if k != "network"},
    }
    fd.close()
    net.close()
    return out, f, S_ev, V_learned


def secondary(fn, *a):
    """Run a secondary workload; a failure is recorded in the JSON line (traceback on stderr)
    instead of losing the headline measurement."""
    try:
        return fn(*a)
    except Exception as e:  # noqa: BLE001 -- reported, not hidden
        import traceback

        traceback.print_exc()
        return {"error": f"{type(e).__name__}: {e}"}


def timed_device(fn, reps, stream):
    """Mean CUDA-event time (ms) of `reps` calls after one warm-up call."""
    import torch

    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps


def scenario_leg(args, stream, check):
    """Config 3: a 500-bus feeder and a [200 scenarios x 8,760 hours] complex64 load tensor
    (1,752,000 power flows), solved with voltage-band statistics fused into the solve."""
    import torch

    from paper_2403_04578_gb300 import inputs as G
    from paper_2403_04578_gb300 import tpf

    dev = torch.device("cuda", torch.cuda.current_device())
    f = G.make_feeder(args.scen_buses, args.seed, peak_factor=1.8)
    S = G.scenario_tensor_device(f, args.scen, args.hours, args.seed, dev)
    T = args.scen * args.hours
    fd = tpf.Feeder.from_inputs(f)
    V = torch.empty(S.shape, dtype=torch.complex64, device=dev)
    band = (0.95, 1.05)
    res = {}

    def run(v=V):
        res.update(fd.solve_tensor(S, V=v, start="flat", v_band=band, tol=args.tol))

    ms = timed_device(run, max(1, min(args.steps, 3)), stream)
    ms_stats = timed_device(lambda: run(None), max(1, min(args.steps, 3)), stream) if V is not None else None
    out = {"workload": f"{args.scen_buses}-bus feeder x [{args.scen} scenarios x {args.hours:,} hours] complex64 "
                       f"loads (factor U(0.5,1.8), 30% PV); sparse method; band {band[0]}-{band[1]} pu statistics",
           "value": T / (ms / 1e3), "unit": "PF/s", "ms_per_step": ms,
           "stats_only": {"value": T / (ms_stats / 1e3), "ms_per_step": ms_stats, "note": "V not written"},
           "converged": int((res["iters"] > 0).sum().item()), "columns": T,
           "buses_out_of_band_per_column_mean": float(res["viol"].float().mean().item()),
           "min_v_pu": float(res["vmin"].min().item()), "max_v_pu": float(res["vmax"].max().item())}
    if check:
        from oracle import oracle as O

        idx = torch.linspace(0, T - 1, args.check_columns, device=dev).long()
        Sf = S.reshape(T, -1)[idx].contiguous()
        r = fd.solve_tensor(Sf, v_complex64=False, v_band=band, tol=args.tol)
        Vt, _, _ = O.Case.from_feeder(f).solve(Sf.cpu().numpy().astype(np.complex128), tol=1e-13,
                                               threads=os.cpu_count() or 1)
        out["max_abs_err_pu"] = float(np.abs(r["V"].cpu().numpy() - Vt).max())
        out["columns_checked"] = int(idx.numel())
    fd.close()
    del S, V
    torch.cuda.empty_cache()
    return out


def batch_leg(args, stream, check):
    """Config 4: 4,096 feeders, bus counts log-uniform in [20, 2,000], T in {96, 288, 1,440}
    (one day at 15, 5 or 1 minute), all solved by one tpf_solve_batch call."""
    import torch

    from paper_2403_04578_gb300 import inputs as G
    from paper_2403_04578_gb300 import tpf

    dev = torch.device("cuda", torch.cuda.current_device())
    specs = G.batch_specs(args.batch_feeders)
    t0 = time.perf_counter()
    feeders = [G.make_feeder(nb, sd) for nb, _, sd in specs]
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    fds = [tpf.Feeder.from_inputs(f) for f in feeders]
    t_create = time.perf_counter() - t0
    S = [G.load_tensor_device(f, T, sd, dev, step_minutes=G.step_minutes_for(T))
         for f, (_, T, sd) in zip(feeders, specs)]
    V = [torch.empty_like(s) for s in S]
    it = [torch.empty(s.shape[0], dtype=torch.int32, device=dev) for s in S]
    mm = [torch.empty(s.shape[0], dtype=torch.float64, device=dev) for s in S]
    cols = sum(T for _, T, _ in specs)
    res = {}

    def run():
        r = tpf.solve_batch(fds, S, V=V, iters=it, mismatch=mm, start="flat", tol=args.tol)
        res["conv"], res["stats"], res["st"] = r[3], r[4], r[5]

    ms = timed_device(run, max(1, min(args.steps, 3)), stream)
    out = {"workload": f"{args.batch_feeders} feeders, buses log-uniform in [20, 2000], T in {{96, 288, 1440}}; "
                       "sparse method, one tpf_solve_batch call",
           "value": cols / (ms / 1e3), "unit": "PF/s", "ms_per_step": ms, "columns": cols,
           "bus_columns": int(sum(f.n_pq * T for f, (_, T, _) in zip(feeders, specs))),
           "converged": int(res["conv"].sum()), "gpu_launches_per_step": res["stats"]["kernel_launches"],
           "tpf_create_s_total": t_create, "feeder_generation_s": t_gen}
    # The same batch prepared once (tpf_batch_create) and solved by replaying its CUDA graph.
    t0 = time.perf_counter()
    bg = tpf.BatchGraph(fds, S, V=V, iters=it, mismatch=mm, start="flat", tol=args.tol)
    t_prep = time.perf_counter() - t0

    def replay():
        bg.launch(stream)
        res["gconv"], _, res["gst"] = bg.wait()

    ms_g = timed_device(replay, max(1, min(args.steps, 3)), stream)
    out["graph_replay"] = {"value": cols / (ms_g / 1e3), "unit": "PF/s", "ms_per_step": ms_g,
                           "converged": int(res["gconv"].sum()), "prepare_s": t_prep,
                           "note": "tpf_batch_launch + tpf_batch_wait: one graph launch per batch solve"}
    bg.close()
    if check:
        from oracle import oracle as O

        errs, checked = [], 0
        pick = [k for k, f in enumerate(feeders) if f.n_bus <= 600][:: max(1, args.batch_feeders // 256)][:16]
        for k in pick:
            cc = torch.linspace(0, S[k].shape[0] - 1, 8, device=dev).long()
            Vt, _, _ = O.Case.from_feeder(feeders[k]).solve(S[k][cc].cpu().numpy(), tol=1e-13,
                                                            threads=os.cpu_count() or 1)
            errs.append(float(np.abs(V[k][cc].cpu().numpy() - Vt).max()))
            checked += int(cc.numel())
        out["max_abs_err_pu"] = max(errs) if errs else None
        out["columns_checked"] = checked
        out["feeders_checked"] = len(pick)
    for fd in fds:
        fd.close()
    del S, V
    torch.cuda.empty_cache()
    return out


def large_leg(args, stream, check):
    """The paper's largest grid (Table I: 5,000 bus-phases, one-minute year): a 5,000-bus feeder and
    525,600 columns on the sparse formulation's large-feeder kernel (16 buses per thread, device
    scratch, chunked launches); sampled columns against the oracle's sparse Newton-Raphson."""
    import torch

    from paper_2403_04578_gb300 import inputs as G
    from paper_2403_04578_gb300 import tpf

    dev = torch.device("cuda", torch.cuda.current_device())
    f = G.make_feeder(args.large_buses, args.seed)
    T = args.large_columns
    S = G.load_tensor_device(f, T, args.seed, dev)
    fd = tpf.Feeder.from_inputs(f)
    V = torch.empty_like(S)
    it = torch.empty(T, dtype=torch.int32, device=dev)
    mm = torch.empty(T, dtype=torch.float64, device=dev)
    ms = timed_device(lambda: fd.solve(S, V, it, mm, precision="mixed", method="sparse", start="flat", tol=args.tol),
                      max(1, min(args.steps, 2)), stream)
    st = fd.stats()
    out = {"workload": f"{args.large_buses}-bus radial feeder x {T:,} one-minute columns (Table I's largest grid "
                       "over the year); sparse formulation, 16 buses per thread",
           "value": T / (ms / 1e3), "unit": "PF/s", "ms_per_step": ms, "converged": st["converged"],
           "launches_per_step": st["kernel_launches"], "mean_sweeps": float(it.abs().float().mean().item())}
    if check:
        from oracle import oracle as O

        Y = O.ybus(f.n_bus, f.from_bus, f.to_bus, f.z_pu)
        errs = []
        for k in np.linspace(0, T - 1, 4).astype(np.int64):
            Vn, _, ok = O.nr_solve(Y, f.slack, f.v0, f.pq_bus, S[int(k)].cpu().numpy(), tol=1e-11)
            errs.append(float(np.abs(V[int(k)].cpu().numpy() - Vn).max()) if ok else float("inf"))
        out["max_abs_err_pu_vs_newton"] = max(errs)
        out["columns_checked"] = len(errs)
    fd.close()
    del S, V
    torch.cuda.empty_cache()
    return out


def table1_100_leg(args, stream, check):
    """Table I's 100-bus row over the one-minute year (525,600 columns) on the sparse formulation,
    next to the paper's times for it (context: other hardware); sampled columns against the oracle."""
    import torch

    from paper_2403_04578_gb300 import inputs as G
    from paper_2403_04578_gb300 import tpf

    dev = torch.device("cuda", torch.cuda.current_device())
    f = G.make_feeder(100, args.seed)
    T = 525600
    S = G.load_tensor_device(f, T, args.seed, dev)
    fd = tpf.Feeder.from_inputs(f)
    V = torch.empty_like(S)
    it = torch.empty(T, dtype=torch.int32, device=dev)
    mm = torch.empty(T, dtype=torch.float64, device=dev)
    ms = timed_device(lambda: fd.solve(S, V, it, mm, precision="mixed", method="sparse", start="flat", tol=args.tol),
                      max(1, min(args.steps, 3)), stream)
    out = {"workload": f"100-bus radial feeder x {T:,} one-minute columns (Table I's 100 bus-phase row over the "
                       "year); sparse formulation",
           "value": T / (ms / 1e3), "unit": "PF/s", "ms_per_step": ms, "converged": fd.stats()["converged"],
           "mean_sweeps": float(it.abs().float().mean().item()),
           "paper_minutes": {"tensor_dense_cpu": 0.37, "tensor_gpu": 1.30, "nr_sparse_cpu": 61.85,
                             "note": "Table I, the paper's hardware (context, not a target)"}}
    if check:
        from oracle import oracle as O

        cc = torch.linspace(0, T - 1, 1024, device=dev).long()
        Vt, _, _ = O.Case.from_feeder(f).solve(S[cc].cpu().numpy(), tol=1e-13, threads=os.cpu_count() or 1)
        out["max_abs_err_pu"] = float(np.abs(V[cc].cpu().numpy() - Vt).max())
        out["columns_checked"] = int(cc.numel())
    fd.close()
    del S, V
    torch.cuda.empty_cache()
    return out


def small_leg(args, stream, check):
    """34-bus feeder over one day of one-minute columns (1,440), flat start.  The whole problem is
    about 1.5 MB, so it is launch- and latency-bound: each arithmetic and formulation reports its
    CUDA-event time per call and the host's launch-inclusive time per call; the oracle checks every
    column."""
    import torch

    from paper_2403_04578_gb300 import inputs as G
    from paper_2403_04578_gb300 import tpf

    dev = torch.device("cuda", torch.cuda.current_device())
    f = G.make_feeder(34, args.seed)
    T = 1440
    S_np = G.load_tensor(f, T, args.seed)
    S = torch.from_numpy(S_np).to(dev)
    fd = tpf.Feeder.from_inputs(f)
    V = torch.empty_like(S)
    it = torch.empty(T, dtype=torch.int32, device=dev)
    mm = torch.empty(T, dtype=torch.float64, device=dev)
    reps = 50
    Vt = None
    out = {"workload": f"34-bus radial feeder x {T:,} one-minute load columns (one day); flat start, per-column "
                       f"stop at max|dV| <= {args.tol:g} pu; latency-bound"}
    if check:
        from oracle import oracle as O

        threads = os.cpu_count() or 1
        case = O.Case.from_feeder(f)
        Vt, _, _ = case.solve(S_np, tol=1e-13, threads=threads)
        t0 = time.perf_counter()
        case.solve(S_np, tol=args.tol, threads=threads)
        dt = time.perf_counter() - t0
        out["cpu_oracle"] = {"value": T / dt, "unit": "PF/s", "cores": threads, "kind": "oracle",
                             "sample": f"all {T:,} columns, same tol"}
    for name, precision, method in (("fp64", "fp64", "dense"), ("mixed_sparse", "mixed", "sparse"),
                                    ("mixed_dense", "mixed", "dense")):
        def call(precision=precision, method=method):
            fd.solve(S, V, it, mm, precision=precision, method=method, start="flat", tol=args.tol)

        ms = timed_device(call, reps, stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            call()
        torch.cuda.synchronize()
        host_ms = (time.perf_counter() - t0) * 1e3 / reps
        r = {"value": T / (ms / 1e3), "unit": "PF/s", "ms_per_call": ms, "host_ms_per_call": host_ms,
             "converged": fd.stats()["converged"], "mean_sweeps": float(it.abs().float().mean().item())}
        if Vt is not None:
            Vg = V.cpu().numpy()
            r["max_abs_err_pu"] = float(np.abs(Vg - Vt).max())
            r["columns_checked"] = T
            print(f"small_feeder {name}: V[0,0] = {Vg[0, 0]!r}, oracle {Vt[0, 0]!r}, max err {r['max_abs_err_pu']:.3e}",
                  file=sys.stderr)
        out[name] = r
    fd.close()
    return out


def poly_leg(args, stream, check):
    """Three-phase feeder: 500 buses (1,497 unknowns), mutual coupling 0.4, per-phase unbalance
    +-20 %, 65,536 one-minute columns, sparse formulation; the oracle checks sampled columns."""
    import torch

    from paper_2403_04578_gb300 import inputs as G
    from paper_2403_04578_gb300 import tpf

    dev = torch.device("cuda", torch.cuda.current_device())
    pf = G.make_feeder_poly(args.poly_buses, args.seed)
    T = args.poly_columns
    S = torch.from_numpy(G.load_tensor_poly(pf, T, args.seed).reshape(T, -1)).to(dev)
    fd = tpf.Feeder.poly(pf.n_bus, pf.from_bus, pf.to_bus, pf.z_blocks, 3, v0=pf.v0)
    V = torch.empty_like(S)
    it = torch.empty(T, dtype=torch.int32, device=dev)
    mm = torch.empty(T, dtype=torch.float64, device=dev)
    ms = timed_device(lambda: fd.solve(S, V, it, mm, precision="mixed", method="sparse", start="flat", tol=args.tol),
                      max(1, min(args.steps, 3)), stream)
    out = {"workload": f"{args.poly_buses}-bus three-phase feeder ({3 * pf.n_pq} unknowns), {T:,} one-minute "
                       "columns, sparse formulation",
           "value": T / (ms / 1e3), "unit": "PF/s", "ms_per_step": ms, "converged": fd.stats()["converged"],
           "mean_sweeps": float(it.abs().float().mean().item())}
    if check:
        from oracle import oracle as O

        pc = O.PolyCase(pf.n_bus, pf.from_bus, pf.to_bus, pf.z_blocks, 3, vs=pf.v0)
        cc = torch.linspace(0, T - 1, min(args.check_columns, 1024, T), device=dev).long()
        Vt, _, _ = pc.solve(S[cc].cpu().numpy(), tol=1e-13, threads=os.cpu_count() or 1)
        out["max_abs_err_pu"] = float(np.abs(V[cc].cpu().numpy() - Vt).max())
        out["columns_checked"] = int(cc.numel())
    fd.close()
    del S, V
    torch.cuda.empty_cache()
    return out


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle (FP64, all host cores) on bounded samples of the workload."""
    if rank != 0:
        return
    from paper_2403_04578_gb300 import inputs as G
    from oracle import oracle as O

    f, config = workload(args)
    threads = os.cpu_count() or 1
    case = O.Case.from_feeder(f)
    budget = args.ref_seconds  # seconds for all warm-up and timed steps
    # The sample spreads over the whole year: n_blocks noise chunks at evenly spaced positions
    # (each chunk regenerated on its own, CHUNK one-minute columns, about 2.8 days), and evenly
    # spaced columns inside each chunk, so every hour of the day and every season is represented.
    n_chunks_year = (args.columns + G.CHUNK - 1) // G.CHUNK
    n_blocks = min(16, n_chunks_year)
    starts = np.unique(np.linspace(0, n_chunks_year - 1, n_blocks).astype(np.int64)) * G.CHUNK
    blocks = [G.load_tensor(f, min(G.CHUNK, args.columns - int(t0)), args.seed, t0=int(t0)) for t0 in starts]
    t0 = time.perf_counter()
    case.solve(blocks[0][: 2 * threads], tol=args.tol, threads=threads)
    per_col = (time.perf_counter() - t0) / (2 * threads)
    per_step = int(max(threads, min(n_blocks * G.CHUNK, budget / (args.steps + args.warmup) / per_col)))
    per_block = max(1, per_step // len(blocks))
    Ss = np.ascontiguousarray(np.concatenate(
        [b[np.linspace(0, b.shape[0] - 1, min(per_block, b.shape[0])).astype(np.int64)] for b in blocks]))
    per_step = Ss.shape[0]
    for _ in range(args.warmup):
        case.solve(Ss, tol=args.tol, threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        case.solve(Ss, tol=args.tol, threads=threads)
        times.append(time.perf_counter() - t0)
    dt = sum(times) / len(times)
    value = per_step / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "PF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
            "cpu_baseline": {"value": value, "unit": "PF/s", "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} columns per step: {per_block} evenly spaced columns in each of "
                                       f"{len(blocks)} {G.CHUNK}-column blocks at evenly spaced positions over the "
                                       f"{args.columns:,}-column year"},
            "e2e": {"value": value, "unit": "PF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_steps(fd, Sd, Vd, itd, mmd, args, method, steps, stream, world, clocks_index=None, net=None):
    """Time `steps` full solves of every column with CUDA events; returns per-step numbers.  With
    `net`, a step is the learned-start solve (prediction of V_0 by the network, then the sparse
    mixed solve from it)."""
    import torch

    kern_ms = gemm_ms = gemm_cols = gemm_launch = 0.0
    launches = 0
    step_ms = []
    barrier(world)
    torch.cuda.synchronize()
    sampler = ClockSampler(clocks_index) if clocks_index is not None else None
    if sampler:
        sampler.__enter__()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        if net is not None:
            fd.solve_learned(net, Sd, Vd, itd, mmd, tol=args.tol, profile=True)
        else:
            fd.solve(Sd, Vd, itd, mmd, precision="mixed", tol=args.tol, start="flat", profile=True, method=method)
        b.record(stream)
        s = fd.stats()
        kern_ms += s["residual_ms"] if method == "sparse" else s["gemm_ms"]
        gemm_ms += s["gemm_ms"]
        gemm_cols += s["gemm_columns"]
        gemm_launch += s["gemm_launches"]
        launches += s["kernel_launches"]
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
    e1.record(stream)
    torch.cuda.synchronize()
    if sampler:
        sampler.__exit__(None, None, None)
    barrier(world)
    total_ms = e0.elapsed_time(e1)
    return {"ms_per_step": allmax(world, total_ms / steps), "kernel_ms": kern_ms / steps, "gemm_ms": gemm_ms,
            "gemm_cols": gemm_cols, "gemm_launch": gemm_launch, "launches": launches, "step_ms": step_ms,
            "stats": fd.stats(), "clocks": sampler.summary() if sampler else None}


def main():
    args = parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch

    import __graft_entry__

    torch.cuda.set_device(local)
    __graft_entry__.build()
    from paper_2403_04578_gb300 import inputs as G
    from paper_2403_04578_gb300 import tpf

    f, config = workload(args)
    config["method"] = args.method
    T, n = args.columns, f.n_pq
    Sh = torch.empty((T, n), dtype=torch.complex128, pin_memory=True)
    # Each rank solves its own year of loads: the columns shard across ranks with no exchange.
    G.load_tensor(f, T, args.seed + rank, out=Sh.numpy())
    config["sharding"] = "rank r solves its own load year (load seed = feeder seed + r); no collective"
    Sd = Sh.to(f"cuda:{local}")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fd = tpf.Feeder.from_inputs(f)
    create_ms = (time.perf_counter() - t0) * 1e3
    Vd = torch.empty_like(Sd)
    itd = torch.empty(T, dtype=torch.int32, device=Sd.device)
    mmd = torch.empty(T, dtype=torch.float64, device=Sd.device)
    stream = torch.cuda.current_stream()
    peaks, peak_src = measured_peaks()

    # The headline path: all T columns per step, inputs resident on the device.  The sparse
    # kernel's launch shape is autotuned on the first 16,384 columns.
    if args.method == "sparse":
        config["sparse_buses_per_thread"] = fd.autotune(Sd[: min(T, 16384)], tol=args.tol)
    for _ in range(args.warmup):
        fd.solve(Sd, Vd, itd, mmd, precision="mixed", tol=args.tol, start="flat", method=args.method)
    torch.cuda.synchronize()
    main_run = timed_steps(fd, Sd, Vd, itd, mmd, args, args.method, args.steps, stream, world, clocks_index=local)
    ms_per_step = main_run["ms_per_step"]
    value = world * T / (ms_per_step / 1e3)
    stats = main_run["stats"]
    column_sweeps = int(itd.abs().sum().item())
    # GPU results on the checked columns (compared with the oracle after every timed region).
    checking = rank == 0 and not args.no_cpu
    cc = check_columns(args, T)
    cc_dev = torch.from_numpy(cc).to(Sd.device)
    V_checks = {}
    it_main = None
    if checking:
        V_checks["max_abs_err_pu"] = Vd[cc_dev].cpu().numpy()
        it_main = itd[cc_dev].cpu().numpy()

    def gemm_roofline(run):
        achieved = 8.0 * n * n * run["gemm_cols"] / (run["gemm_ms"] / 1e3) / 1e12
        peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
        traffic = None
        if GEMM_TRAFFIC_BYTES_PER_COLUMN is not None and args.buses == 1000:
            traffic = GEMM_TRAFFIC_BYTES_PER_COLUMN * run["gemm_cols"] / max(run["gemm_launch"], 1)
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "tc_gemm",
                "peak_source": f"{peak_src} bf16 sustained (fp16 has the bf16 rate)",
                "traffic_note": "ncu DRAM bytes per iterating column (capture of 16,384 columns of the "
                                "1,000-bus feeder) x columns per launch",
                "share_of_step": run["gemm_ms"] / sum(run["step_ms"]),
                "ms_per_launch": run["gemm_ms"] / max(run["gemm_launch"], 1)}

    def tree_roofline(run, sweeps, per_column=TREE_TRAFFIC_BYTES_PER_COLUMN):
        # FP32 peak from the unit counts: SMs x 128 FP32 lanes x 2 flop (FMA) x max SM clock.
        sm_count = torch.cuda.get_device_properties(local).multi_processor_count
        peak = sm_count * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
        achieved = TREE_FLOPS_PER_BUS_SWEEP * n * sweeps / (run["kernel_ms"] / 1e3) / 1e12
        traffic = None
        if per_column is not None and args.buses == 1000:
            traffic = per_column * T
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "mx_tree",
                "peak_source": f"FP32: {sm_count} SMs x 128 lanes x 2 flop x {peaks.get('sm_max_mhz', 2070.0):.0f} MHz",
                "flops_note": f"{TREE_FLOPS_PER_BUS_SWEEP} flop per bus per sweep x {n} buses x {sweeps:,} "
                              "column-sweeps (anchors and the final residual not counted)",
                "traffic_note": ("ncu DRAM bytes per column (capture of the first 16,384 columns of the 1,000-bus "
                                 "year, flat start)" if per_column == TREE_FLAT_TRAFFIC_BYTES_PER_COLUMN else
                                 "ncu DRAM bytes per column (capture of 65,536 columns of the 1,000-bus year from "
                                 "the learned start)") + " x columns per launch",
                "hbm_frac": (per_column or 0) * T / (run["kernel_ms"] / 1e3) / 1e9 / float(peaks.get("hbm_gbs", 6800.0))
                            if per_column else None,
                "share_of_step": run["kernel_ms"] * len(run["step_ms"]) / sum(run["step_ms"]),
                "ms_per_launch": run["kernel_ms"]}

    roofline = (tree_roofline(main_run, column_sweeps, TREE_FLAT_TRAFFIC_BYTES_PER_COLUMN) if args.method == "sparse"
                else gemm_roofline(main_run))
    flat = {"value": value, "unit": "PF/s", "ms_per_step": ms_per_step, "mean_sweeps": column_sweeps / T,
            "gpu_launches": main_run["launches"], "roofline": roofline,
            "step_ms": [round(x, 3) for x in main_run["step_ms"]],
            "note": "flat start V_0 = 1 (Algorithm 1), sparse mixed solve"}

    # The learned start on the same workload: the network is trained once per feeder (on other load
    # columns, not timed: a per-feeder set-up cost, reported), and a step is the prediction of V_0
    # for every column plus the sparse mixed solve from it.
    learned = net = None
    if args.method == "sparse" and args.headline == "learned":
        net, train_info = train_start_network(f, fd, args, Sd.device, args.train_columns, args.epochs)
        for _ in range(args.warmup):
            fd.solve_learned(net, Sd, Vd, itd, mmd, tol=args.tol)
        _, _, _, fallback, _ = fd.solve_learned(net, Sd, Vd, itd, mmd, tol=args.tol)
        torch.cuda.synchronize()
        lrun = timed_steps(fd, Sd, Vd, itd, mmd, args, "sparse", args.steps, stream, world, clocks_index=local,
                           net=net)
        l_sweeps = int(itd.abs().sum().item())
        learned = {"value": world * T / (lrun["ms_per_step"] / 1e3), "unit": "PF/s", "ms_per_step": lrun["ms_per_step"],
                   "mean_sweeps": l_sweeps / T, "fallback_columns": fallback, "converged": lrun["stats"]["converged"],
                   "gpu_launches": lrun["launches"], "roofline": tree_roofline(lrun, l_sweeps),
                   "solve_kernel_ms": lrun["kernel_ms"], "predict_ms": lrun["ms_per_step"] - lrun["kernel_ms"],
                   "step_ms": [round(x, 3) for x in lrun["step_ms"]],
                   "clocks": lrun["clocks"], **train_info}
        if checking:
            V_checks["learned_max_abs_err_pu"] = Vd[cc_dev].cpu().numpy()

    # End to end through the host-buffer entry point.
    e2e = None
    if not args.no_e2e:
        Vh = torch.empty((T, n), dtype=torch.complex128, pin_memory=True)
        ith = torch.empty(T, dtype=torch.int32, pin_memory=True)
        mmh = torch.empty(T, dtype=torch.float64, pin_memory=True)
        for _ in range(2):  # warm-up: the first touches of the pinned pages and the copy engines' queues
            fd.solve_host(Sh, precision="mixed", tol=args.tol, out=(Vh, ith, mmh), method=args.method)
        e2e_steps = max(1, args.steps)
        barrier(world)
        t0 = time.perf_counter()
        step_ms = []
        for _ in range(e2e_steps):
            ts = time.perf_counter()
            fd.solve_host(Sh, precision="mixed", tol=args.tol, out=(Vh, ith, mmh), method=args.method)
            step_ms.append((time.perf_counter() - ts) * 1e3)
        dt = allmax(world, (time.perf_counter() - t0) / e2e_steps)
        flat["e2e"] = e2e = {"value": world * T / dt, "unit": "PF/s", "h2d_bytes_per_step": T * n * 16,
               "d2h_bytes_per_step": T * n * 16 + T * 4 + T * 8, "ms_per_step": dt * 1e3,
               "step_ms": [round(x, 2) for x in step_ms],
               "entry_point": "tpf_solve_host (pinned host buffers)"}
        if learned is not None:
            learned["e2e"] = learned_e2e(fd, net, Sh, Vh, ith, mmh, args, world)

    # The other formulation on the same workload.
    other = "dense" if args.method == "sparse" else "sparse"
    other_obj = None
    if not args.no_other:
        fd.solve(Sd, Vd, itd, mmd, precision="mixed", tol=args.tol, start="flat", method=other)
        torch.cuda.synchronize()
        run = timed_steps(fd, Sd, Vd, itd, mmd, args, other, max(1, min(args.steps, 3)), stream, world)
        other_obj = {"value": world * T / (run["ms_per_step"] / 1e3), "unit": "PF/s",
                     "ms_per_step": run["ms_per_step"], "gpu_launches_per_step": run["launches"] / len(run["step_ms"]),
                     "sweeps": run["stats"]["sweeps"], "converged": run["stats"]["converged"]}
        other_obj["roofline"] = gemm_roofline(run) if other == "dense" else tree_roofline(
            run, int(itd.abs().sum().item()))
        if checking:
            V_checks[f"{other}_max_abs_err_pu"] = Vd[cc_dev].cpu().numpy()

    # ZIP loads (Eq. 3) on the same workload: per-bus shares of constant power / current /
    # impedance drawn once; the oracle checks the ZIP power balance of sampled columns.
    zip_obj = None
    if not args.no_zip:
        alpha = np.random.default_rng(args.seed).dirichlet([2, 1, 1], n).T.copy()
        fd.set_zip(alpha)
        zrun = timed_steps(fd, Sd, Vd, itd, mmd, args, "sparse", max(1, min(args.steps, 3)), stream, world)
        zip_obj = {"value": world * T / (zrun["ms_per_step"] / 1e3), "unit": "PF/s", "ms_per_step": zrun["ms_per_step"],
                   "alpha": "per bus (alpha_P, alpha_I, alpha_Z) ~ Dirichlet(2, 1, 1)",
                   "mean_sweeps": float(itd.abs().float().mean().item()), "converged": zrun["stats"]["converged"]}
        if rank == 0 and not args.no_cpu:
            from oracle import oracle as O

            cc = np.linspace(0, T - 1, min(args.check_columns, T)).astype(np.int64)
            Vz = Vd[torch.from_numpy(cc).to(Vd.device)].cpu().numpy()
            c = O.Case.from_feeder(f)
            zip_obj["max_power_mismatch_pu"] = float(c.mismatch_zip(Sh.numpy()[cc], alpha, Vz).max())
            zip_obj["columns_checked"] = int(cc.size)
        fd.set_zip(None)

    # Plain FP64 GPU FPI on a column sample (the comparison path of the metric).
    F = min(args.fp64_sample, T)
    Sf = Sd[:F].contiguous()
    fd.solve(Sf, precision="fp64", tol=args.tol)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(2):
        fd.solve(Sf, precision="fp64", tol=args.tol)
    b.record(stream)
    b.synchronize()
    fp64_pfs = F / (a.elapsed_time(b) / 2 / 1e3)
    fp64 = {"value": fp64_pfs, "unit": "PF/s", "sample": f"first {F} columns", "sweeps": fd.stats()["sweeps"],
            "formulation": "dense (Algorithm 1, K = -Y_dd^-1), FP64"}

    # Plain FP64 GPU FPI in the sparse formulation on the whole workload: the same O(n) tree
    # substitution as the headline path, every operation in FP64.  Against it the headline ratio
    # isolates what mixed precision buys.
    fp64s = None
    if args.method == "sparse":
        ms64 = timed_device(lambda: fd.solve(Sd, Vd, itd, mmd, precision="fp64", method="sparse", start="flat",
                                             tol=args.tol), 2, stream)
        s64 = fd.stats()
        fp64s = {"value": T / (ms64 / 1e3), "unit": "PF/s", "ms_per_step": ms64,
                 "columns": T, "formulation": "sparse (Algorithm 2, tree substitution), FP64",
                 "mean_sweeps": float(itd.abs().float().mean().item()), "converged": s64["converged"],
                 "gpu_launches_per_step": s64["kernel_launches"]}
        if checking:
            V_checks["fp64_sparse_max_abs_err_pu"] = Vd[cc_dev].cpu().numpy()

    # The headline step: the learned-start solve when it ran, else the flat start.
    head = learned if learned is not None else flat
    if learned is not None:
        value, ms_per_step, e2e = learned["value"], learned["ms_per_step"], learned.get("e2e")
        roofline, clocks, launches = learned["roofline"], learned["clocks"], learned["gpu_launches"]
        config["start"] = (f"learned: V_0 predicted by a {learned['network']} network trained on "
                           f"{learned['train_columns']:,} other columns ({learned['epochs']} epochs, not timed), "
                           "then the sparse mixed solve from it")
    else:
        clocks, launches = main_run["clocks"], main_run["launches"]
        config["start"] = "flat"
    line = {"metric": METRIC, "value": value, "unit": "PF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": ("f32 sweeps + double-float anchors" if args.method == "sparse"
                      else "f16 tensor-core products + f32/double-float elementwise"),
            "data": "synthetic", "config": config, "roofline": roofline,
            "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
            "sweeps": stats["sweeps"], "anchors_or_anchor_sweeps": stats["precise_sweeps"],
            "mean_sweeps": head["mean_sweeps"], "tpf_create_ms": create_ms,
            "headline_start": "learned" if learned is not None else "flat",
            "flat_start": flat,
            "fp64_gpu": fp64,
            "speedup_vs_fp64_gpu": (value / world) / fp64_pfs,
            "speedup_vs_fp64_gpu_note": "formulation plus precision: the mixed sparse path against the FP64 "
                                        "dense path (8 n^2 against 36 n flop per bus-sweep)",
            }
    if learned is not None:
        line["learned_start_headline"] = {k: v for k, v in learned.items() if k not in ("roofline", "clocks", "e2e")}
        line["speedup_learned_vs_flat"] = learned["value"] / flat["value"]
    if fp64s is not None:
        line["fp64_gpu_sparse"] = fp64s
        line["speedup_vs_fp64_gpu_sparse"] = (value / world) / fp64s["value"]
        line["speedup_vs_fp64_gpu_sparse_note"] = "precision only: both paths run the sparse formulation"
    if other_obj is not None and other == "dense":
        line["speedup_dense_mixed_vs_fp64_dense"] = other_obj["value"] / world / fp64_pfs
    if checking:
        cpu, check = cpu_oracle_leg(f, Sh.numpy(), args, T, cc, it_main, V_checks)
        line["cpu_baseline"] = cpu
        line["cpu_newton_raphson"] = secondary(cpu_newton_leg, f, Sh.numpy(), T)
        if other_obj is not None and f"{other}_max_abs_err_pu" in check:
            other_obj["max_abs_err_pu"] = check.pop(f"{other}_max_abs_err_pu")
        if fp64s is not None and "fp64_sparse_max_abs_err_pu" in check:
            fp64s["max_abs_err_pu"] = check.pop("fp64_sparse_max_abs_err_pu")
        # The headline's accuracy is the learned solve's when it is the headline; the flat start's
        # iteration counts are compared with the oracle's.
        flat["max_abs_err_pu"] = check["max_abs_err_pu"]
        if "learned_max_abs_err_pu" in check:
            check["max_abs_err_pu"] = learned["max_abs_err_pu"] = check.pop("learned_max_abs_err_pu")
            line["learned_start_headline"]["max_abs_err_pu"] = check["max_abs_err_pu"]
            check["iters_compared"] = "flat start"
        line["accuracy"] = check
    if other_obj is not None:
        line[f"{other}_method"] = other_obj
    if zip_obj is not None:
        line["zip_loads"] = zip_obj
    del Sd, Vd, Sh
    torch.cuda.empty_cache()
    if not args.no_learned:
        ls, f200, S_ev, V_ls = learned_start_leg(args, stream)
        if rank == 0 and not args.no_cpu:
            from oracle import oracle as O

            cc = np.linspace(0, S_ev.shape[0] - 1, args.check_columns).astype(np.int64)
            S_s = S_ev[torch.from_numpy(cc).to(S_ev.device)].cpu().numpy()
            Vt, _, _ = O.Case.from_feeder(f200).solve(S_s, tol=1e-13, threads=os.cpu_count() or 1)
            ls["max_abs_err_pu"] = float(np.abs(V_ls[cc] - Vt).max())
            ls["columns_checked"] = int(cc.size)
        line["learned_start"] = ls
    if not args.no_scenario:
        line["scenario_tensor"] = secondary(scenario_leg, args, stream, rank == 0 and not args.no_cpu)
    if not args.no_batch:
        line["feeder_batch"] = secondary(batch_leg, args, stream, rank == 0 and not args.no_cpu)
    if not args.no_poly:
        line["three_phase"] = secondary(poly_leg, args, stream, rank == 0 and not args.no_cpu)
    if not args.no_large:
        line["large_feeder"] = secondary(large_leg, args, stream, rank == 0 and not args.no_cpu)
    if not args.no_small:
        line["small_feeder"] = secondary(small_leg, args, stream, rank == 0 and not args.no_cpu)
    if not args.no_table1:
        line["table1_100_bus"] = secondary(table1_100_leg, args, stream, rank == 0 and not args.no_cpu)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if net is not None:
        net.close()
    fd.close()


if __name__ == "__main__":
    main()
