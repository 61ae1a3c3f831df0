"""Benchmark: field updates/s of the PQMC auxiliary-field sweep at 40x40 on GB300.

Workload (one step = one full sweep, forward l = 1..M then backward l = M..1):
  standard 2D Hubbard, 40 x 40 periodic (N = 1600), t = 1, U = 6 (real spin decoupling),
  filling 0.875 (700 particles per spin), dtau = 0.05, M = 80 slices, FP32 bulk G,
  delayed update (k sites per delayed step), FP64 re-orthonormalisation and G recompute
  every 5 slices (the FP32 drift of G stays under 1e-3 there; the workload's own 10 slices let
  it reach 4e-2, reported beside the headline).  One walker per GPU (weak scaling across ranks,
  no collective on the data path).  Inputs are synthetic and seeded (trial state, fields,
  Philox uniforms).

The timed sweeps replay each slice-step from the CUDA graph the library captured for it (the
recomputes launch directly); the same sweeps are then repeated with direct launches under the
library's phase profiler for the breakdown.  The JSON line reports the device-timed sweep
throughput (value), the update-only rate, local and block-force-bias comparisons on a bounded
sample of slices, the FP32 drift of G against the FP64 recompute, the roofline of the dominant
kernel (measured live with CUDA events on the launching stream), the clocks seen during the
timed region, an end-to-end number through the C ABI with host buffers, and the FP64 oracle
timed on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2506_09611_gb300 import inputs, tune  # noqa: E402

METRIC = "field updates/s at 40x40 Hubbard on 1 GB300, delayed/blockFB vs local; G err"
UNIT = "field updates/s"
L, U, T_HOP, DTAU, M, FILLING = 40, 6.0, 1.0, 0.05, 80, 0.875
# FP64 recompute periods: the workload's own (10 slices; the FP64-bulk, precision and 16 x 16 legs)
# and the FP32 headline's, short enough that the median relative drift of the FP32 G at the
# recompute points stays under DRIFT_TOL (measured: 4e-4 at 5 slices, 4e-2 at 10).
STAB_WORKLOAD, STAB, DRIFT_TOL = 10, 5, 1e-3
NS = inputs.n_sigma_for(L, FILLING)
N = L * L
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
CPU_SLICES = 16  # oracle slice-steps of the cpu_baseline sample (about 10 s on 16 Arm cores)
BATCH_WALKERS = 256


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--k", type=int, default=64, help="delay rank (sites per delayed step)")
    ap.add_argument("--nb", type=int, default=16, help="block size of the block force-bias sample")
    ap.add_argument("--cmp-slices", type=int, default=20, help="slices of the local / block-FB samples")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the mixed walker population leg")
    ap.add_argument("--no-soc", action="store_true", help="skip the spin-orbit-coupled leg")
    ap.add_argument("--no-dense", action="store_true", help="skip the dense tensor-core wrap leg")
    ap.add_argument("--no-tform", action="store_true", help="skip the T-form sweep")
    ap.add_argument("--no-cpqmc", action="store_true", help="skip the constrained-path AFQMC leg")
    ap.add_argument("--no-stab-sweep", action="store_true", help="skip the FP32 recompute-period legs")
    ap.add_argument("--no-precision", action="store_true", help="skip the per-precision accuracy report")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-bulk sweep")
    ap.add_argument("--no-ksweep", action="store_true", help="skip the 40x40 delay-rank sweep")
    ap.add_argument("--no-config16", action="store_true", help="skip the 16x16 local / delayed legs")
    ap.add_argument("--soc-slices", type=int, default=20, help="timed slice-steps per mode of the SOC leg")
    ap.add_argument("--gemm", default="tc3", choices=["tc3", "simt", "tf32"],
                    help="FP32 GEMM engine: tcgen05 three-term TF32 split, FP32 SIMT, or one TF32 pass")
    return ap.parse_args()


def optional_leg(name, fn):
    """Run an auxiliary leg of the JSON line.  The device-timed sweep above it is the headline;
    a leg that raises is reported in the line as {"error": ...} instead of losing the line."""
    try:
        return fn()
    except Exception as ex:  # noqa: BLE001 -- reported, not swallowed
        print(f"bench: {name} leg failed: {ex!r}", file=sys.stderr, flush=True)
        return {"error": f"{type(ex).__name__}: {ex}"}


def max_over_ranks(dist, ms, device):
    """The slowest rank's time: every rank's timed region ends at the same barrier, so the job's
    time is the maximum (all_reduce MAX over the process group)."""
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, updates_per_step, steps, ms_total):
    """Whole-job field updates/s: each rank sweeps its own walker (weak scaling, no collective on the
    data path), so the job does world x updates_per_step per step in the slowest rank's time."""
    return world * updates_per_step * steps / (ms_total / 1e3)


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_oracle_sample(n_slices, k, warm=0):
    """The FP64 oracle on the host cores: G(0) of the 40x40 workload (M = 10, not timed), then
    n_slices slice-steps (wrap + delayed update) timed.  Returns (field updates/s, cores, secs)."""
    import oracle

    Ms = 10
    P = inputs.trial_state(L, L, NS)
    X = inputs.initial_fields(Ms, N, seed=1)
    model = oracle.Model(L, L, T_HOP, U, DTAU, Ms)
    w = oracle.Walker(model, P, P, X)
    order = [(l, +1) for l in range(1, Ms + 1)] + [(l, -1) for l in range(Ms, 0, -1)]
    times = []
    for it in range(warm + n_slices):
        ell, d = order[it % len(order)]
        u = inputs.uniforms(1, 0, it, 2 * N)
        t0 = time.perf_counter()
        w.sweep_slice(ell, d, "delayed", u, k=k)
        if it >= warm:
            times.append(time.perf_counter() - t0)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return N * len(times) / sum(times), cores, sum(times)


def soc_oracle_sample():
    """The FP64 SOC oracle on the host cores: G(0) of the 24 x 24 workload with M = 2 (not timed),
    then four slice-steps (wrap + block force bias, nb = 16: forward 1, 2, backward 2, 1) timed."""
    import oracle

    Ns = SOC_L * SOC_L
    m = oracle.SocModel(SOC_L, T_HOP, SOC_LAM, SOC_U, DTAU, 2)
    w = oracle.SocWalker(m, inputs.soc_trial_state(SOC_L, Ns, lam=SOC_LAM), inputs.initial_fields(2, Ns, seed=1))
    t0 = time.perf_counter()
    for visit, (ell, d) in enumerate(((1, +1), (2, +1), (2, -1), (1, -1))):
        w.sweep_slice(ell, d, "blockfb", inputs.uniforms(1, 0, visit, 2 * Ns), nb=16)
    secs = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return 4 * Ns / secs, cores, secs


def arm_config(k):
    """The workload both arms report (the reference arm times a bounded sample of it)."""
    return {"workload": f"{L}x{L} standard Hubbard, U/t={U}, n={FILLING} ({NS} per spin), "
                        f"dtau={DTAU}, M={M}, FP32 bulk G, delayed k={k}, FP64 recompute "
                        f"every {STAB} slices (median FP32 drift of G at the recompute points under "
                        f"{DRIFT_TOL:g}), separable wrap (exp(-dtau K) = Ex (x) Ex)",
            "step": f"one full sweep (2M = {2 * M} slice-steps: wrap + delayed update, each replayed from its "
                    f"captured CUDA graph) + {2 * M // STAB} FP64 recomputes",
            "walkers_per_gpu": 1, "l2": "flushed between timed steps (256 MB write)"}


def reference_arm(args, rank):
    if rank != 0:
        return
    v, cores, secs = run_oracle_sample(args.steps, args.k, warm=args.warmup)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": arm_config(args.k),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step one slice-step (wrap + delayed update of the {N} sites) of the "
                                   f"FP64 oracle: {args.steps} timed after {args.warmup} warm-up slice-steps; "
                                   f"G(0) from the oracle's own FP64 init with M=10 (not timed)"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return reference_arm(args, rank)

    import torch

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_2506_09611_gb300 import afqmc

    afqmc.load()
    stream = torch.cuda.current_stream()
    seed = 1 + rank
    P = inputs.trial_state(L, L, NS)
    X = inputs.initial_fields(M, N, seed=seed)
    Pcat = np.concatenate([P.ravel(), P.ravel()])
    ctx = afqmc.Context(M, dtau=DTAU, U=U, t=T_HOP, precision="fp32", stab_every=STAB, seed=seed, gemm=args.gemm)
    ctx.init_walkers([L], [NS], [NS], Pcat, X, stream=stream)
    order = [(l, +1) for l in range(1, M + 1)] + [(l, -1) for l in range(M, 0, -1)]

    def sweep(mode, k, nb, drift=None, slices=None):
        for (ell, d) in (order if slices is None else slices):
            ctx.sweep_slice(ell, d, mode, k=k, nb=nb, stream=stream)
            pos = ell if d > 0 else ell - 1
            if pos % STAB == 0:  # FP64 re-orthonormalisation + recompute point
                if drift is not None:
                    drift.append((float(ctx.recompute_G(stream=stream)[0]), pos, d))
                else:
                    afqmc.afqmc_recompute_G(ctx.h, None, stream)

    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    drifts = []
    for _ in range(args.warmup):
        sweep("delayed", args.k, args.nb, drift=drifts)
    torch.cuda.synchronize()

    # ---------------- timed region: K full sweeps ----------------
    # Every slice-step replays the CUDA graph the library captured for it (one untimed sweep
    # captures them all); the FP64 recomputes launch directly.  The library counts each replayed
    # graph's kernels as launches.
    ctx.set_graphs(True)
    sweep("delayed", args.k, args.nb)
    torch.cuda.synchronize()
    launches0 = afqmc.afqmc_launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local_rank) as clk:
        for i in range(args.steps):
            flush_buf.zero_()  # L2 flush between timed steps (256 MB > 129 MB L2), outside the events
            ev[i][0].record(stream)
            sweep("delayed", args.k, args.nb)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    launches = afqmc.afqmc_launch_count() - launches0
    ctx.set_graphs(False)
    ms_steps = [a.elapsed_time(b) for a, b in ev]
    ms_total = sum(ms_steps)
    if dist is not None:
        ms_total = max_over_ranks(dist, ms_total, "cuda")
        dist.barrier()
    updates_per_step = N * M * 2
    value = job_throughput(world, updates_per_step, args.steps, ms_total)
    clocks = clk.summary()

    # ---------------- the same sweeps with direct launches, under the phase profiler ----------------
    # (the phases, the per-kernel rooflines and the update-only rate come from this pass)
    ctx.set_profiling(True)
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms_direct = 0.0
    for i in range(args.steps):
        flush_buf.zero_()
        d0.record(stream)
        sweep("delayed", args.k, args.nb)
        d1.record(stream)
        torch.cuda.synchronize()
        ms_direct += d0.elapsed_time(d1)
    prof = ctx.profile()
    ctx.set_profiling(False)
    direct = {"value": updates_per_step * args.steps / (ms_direct / 1e3), "ms_per_step": ms_direct / args.steps,
              "note": "the same sweeps with every kernel launched directly, under the phase profiler"}

    # update-only (the paper's "time for update per sweep"): prep + window chains + flushes
    # (the flush runs on a second stream under the window loop; its interval is not added)
    upd_ms = prof["prep"]["ms"] + prof["chain"]["ms"]
    update_only = updates_per_step * args.steps / (upd_ms / 1e3)

    # ---------------- bounded comparison samples (same context, continuing the chain) ------------
    cmp, cmp_prof = compare_modes(afqmc, ctx, stream, args.k, args.nb, args.cmp_slices)
    speedup = {m: cmp[m]["update_only"] / cmp["local"]["update_only"] for m in ("delayed", "blockfb")}
    ksweep = None
    if not args.no_ksweep:
        ksweep = optional_leg("k_sweep", lambda: delayed_k_sweep(afqmc, ctx, stream, (32, 64, 128), 10, N))

    # ---------------- roofline of the dominant kernel ----------------
    pk, pk_src = peaks()
    optional_leg("fp64_peak", lambda: fp64_gemm_tflops(torch))
    kernels = kernel_rooflines(prof, args.gemm, pk, pk_src, args.steps)
    roof = dict(kernels[0]) if kernels else None
    l2_gbs = optional_leg("l2_copy", lambda: l2_copy_bandwidth(torch))
    kernels += local_and_chain_rooflines(cmp_prof, pk, pk_src, l2_gbs if isinstance(l2_gbs, float) else None)


    # ---------------- end to end through the C ABI with host buffers ----------------
    e2e = None
    if not args.no_e2e:
        e2e = optional_leg("e2e", lambda: end_to_end(afqmc, torch, stream, args, seed, rank))

    X_eq = ctx.fields(0).copy()  # the headline walker's fields after its sweeps (equilibrated)
    ctx.close()
    multi = None
    if not args.no_batch:
        multi = optional_leg("walkers_40x40", lambda: walkers_40x40_leg(afqmc, torch, stream, args, seed))
    batch = None
    if not args.no_batch:
        batch = optional_leg("batched_population", lambda: batched_population(afqmc, torch, stream, args, seed))
    soc_res = None
    if not args.no_soc:
        soc_res = optional_leg("soc", lambda: soc_leg(torch, stream, args, seed))
    tf = None
    if not args.no_tform:
        tf = optional_leg("tform", lambda: tform_leg(afqmc, torch, stream, args, seed))
    cpq = None
    if not args.no_cpqmc:
        cpq = optional_leg("cpqmc", lambda: cpqmc_leg(afqmc, torch, stream, seed))
    dense = None
    if not args.no_dense:
        dense = optional_leg("dense_wrap", lambda: dense_wrap_leg(afqmc, torch, stream, args, seed,
                                                                  prof["wrap"]["ms"] / args.steps))
    c16 = None
    if not args.no_config16:
        c16 = optional_leg("config_16x16", lambda: config_16x16_leg(afqmc, torch, stream, args, seed))
    prec = None
    if not args.no_precision:
        prec = {"from_trial_fields": optional_leg("precision_report", lambda: precision_report(afqmc, stream, args,
                                                                                              seed)),
                "from_equilibrated_fields": optional_leg(
                    "precision_report_eq", lambda: precision_report(afqmc, stream, args, seed, X=X_eq,
                                                                    variants=(("fp32_separable", "tc3", "separable"),
                                                                              ("fp32_dense_tc3", "tc3", "dense"))))}
    stabs = None
    if not args.no_stab_sweep:
        stabs = optional_leg("stab_sweep", lambda: stab_sweep_leg(afqmc, torch, stream, args, seed, X_eq))
    f64 = None
    if not args.no_fp64:
        f64 = optional_leg("fp64_bulk", lambda: fp64_bulk_leg(afqmc, torch, stream, args, seed))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        def cpu_leg():
            v, cores, secs = run_oracle_sample(CPU_SLICES, args.k)
            return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                    "sample": "%d slice-steps (wrap + delayed update, k=%d) of the FP64 oracle at 40x40 from its "
                              "own G(0) (M=10 init not timed); %.1f s of CPU work" % (CPU_SLICES, args.k, secs)}

        cpu = optional_leg("cpu_baseline", cpu_leg)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": arm_config(args.k),
            "update_only": {"value": update_only, "unit": UNIT,
                            "note": "prep + the window loop (decisions; the rank-m flushes overlap on a second "
                                    "stream): the paper's update time"},
            "phases_ms_per_step": {k: v["ms"] / args.steps for k, v in prof.items()
                                   if k not in ("elim", "wrap_gemm", "flush_gemm", "lu_o", "solve", "dgemm")},
            "compare_sample": cmp,
            "speedup_update_only_vs_local": speedup,
            "k_sweep_40x40": ksweep,
            "config_16x16": c16,
            "G_err_fp32_vs_fp64_recompute": {"max": max(x[0] for x in drifts) if drifts else None,
                                             "median": statistics.median(x[0] for x in drifts) if drifts else None,
                                             "slices_between_recomputes": STAB,
                                             "tolerance_median": DRIFT_TOL,
                                             "within_tolerance": (statistics.median(x[0] for x in drifts) <= DRIFT_TOL)
                                             if drifts else None,
                                             "by_point": [{"slice": p, "dir": dd, "drift": v} for v, p, dd in drifts],
                                             "note": "the warm-up sweeps' recompute points: ||G_fp32 - G_fp64|| / "
                                                     "||G_fp64|| after the %d slices since the previous one" % STAB},
            "roofline": roof,
            "fp64_peak": dict(FP64_MEASURED) if FP64_MEASURED else None,
            "roofline_kernels": kernels[1:],
            "clocks": clocks,
            "gpu_launches": launches,
            "e2e": e2e,
            "direct_launches": direct,
            "walkers_40x40": multi,
            "batched_population": batch,
            "soc": soc_res,
            "dense_wrap": dense,
            "tform": tf,
            "cpqmc": cpq,
            "precision_report": prec,
            "fp32_recompute_periods": stabs,
            "fp64_bulk": f64,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def compare_modes(afqmc, ctx, stream, k, nb, n_slices, stab=STAB, elem_bytes=4):
    """Local, block force-bias and delayed updates on the same walker: each mode sweeps slices
    1..n_slices forward under the library's phase profiler (its recomputes included), then the walker
    walks back to slice 0 with the delayed update so that the next mode starts from the same place.
    update_only = sites / (prep + site loop) time, the paper's "time for update"; the window loop's
    interval ends after the last rank-m product, so overlapped flushes count only where they delay
    the loop.  Returns the per-mode summary and the raw per-mode profiles and counts."""
    cmp, raw = {}, {}
    sample = [(l, +1) for l in range(1, n_slices + 1)]
    back = [(l, -1) for l in range(n_slices, 0, -1)]
    for mode in ("local", "blockfb", "delayed"):
        ctx.set_profiling(True)
        stats = []
        for (ell, d) in sample:
            st = ctx.sweep_slice(ell, d, mode, k=k, nb=nb, want_stats=True, stream=stream)
            stats.append((st[0].proposals, st[0].accepts, st[0].flipped))
            if ell % stab == 0:
                afqmc.afqmc_recompute_G(ctx.h, None, stream)
        p = ctx.profile()
        ctx.set_profiling(False)
        for (ell, d) in back:
            ctx.sweep_slice(ell, d, "delayed", k=k, nb=nb, stream=stream)
            if (ell - 1) % stab == 0:
                afqmc.afqmc_recompute_G(ctx.h, None, stream)
        umode = (p["local"]["ms"] if mode == "local" else p["chain"]["ms"]) + p["prep"]["ms"]
        n_upd = N * len(sample)
        props = sum(x[0] for x in stats)
        acc = sum(x[1] for x in stats)
        flips = sum(x[2] for x in stats)
        cmp[mode] = {"update_only": n_upd / (umode / 1e3),
                     "with_wrap": n_upd / ((umode + p["wrap"]["ms"]) / 1e3),
                     "acceptance": acc / max(props, 1), "slices": len(sample),
                     "k" if mode == "delayed" else ("nb" if mode == "blockfb" else "kind"):
                         (k if mode == "delayed" else (nb if mode == "blockfb" else "rank-1 update per accept"))}
        raw[mode] = {"prof": p, "proposals": props, "accepts": acc, "flipped": flips, "slices": len(sample),
                     "elem_bytes": elem_bytes}
    return cmp, raw


def local_and_chain_rooflines(raw, pk, pk_src, l2_gbs):
    """The local update's rank-1 read-modify-write and the delayed window chain, from the comparison
    sample's intervals.
    * local_kernel: each accepted flip reads and writes both spins' G once: 2 x 2 x N^2 x s bytes
      (s = element size); achieved = those bytes x accepts / the kernel's time (one launch per slice).
      G of both spins (20.5 MB in FP32) stays in the 129 MB L2, so the fraction is given against the
      measured HBM copy bandwidth and against an L2-resident copy measured in this run.
    * window chain (window kernel + next-window block, one CTA per walker): latency-bound; reported as
      time per proposed site and per accept."""
    out = []
    lo = raw["local"]
    ph = lo["prof"]["local"]
    if ph["intervals"] and lo["accepts"]:
        per_acc = 2 * 2 * N * N * lo["elem_bytes"]
        ach = per_acc * lo["accepts"] / (ph["ms"] / 1e3) / 1e9
        out.append({"kernel": "local_kernel (rank-1 update per accepted flip, both spins, one cooperative launch "
                              "per slice)", "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / pk["hbm_gbs"], "l2_copy_gbs": l2_gbs,
                    "frac_of_l2_copy": (ach / l2_gbs) if l2_gbs else None,
                    "traffic": None, "launches": ph["intervals"], "ms_per_launch": ph["ms"] / ph["intervals"],
                    "us_per_accept": ph["ms"] * 1e3 / lo["accepts"], "work_per_accept": per_acc,
                    "accepts_per_launch": lo["accepts"] / ph["intervals"],
                    "peak_source": "measured HBM copy (of %s); G is L2-resident: l2_copy_gbs is a copy of an "
                                   "80 MB working set (src + dst) timed in this run" % pk_src})
    de = raw["delayed"]
    ch = de["prof"]["chain"]
    if ch["intervals"] and de["accepts"]:
        out.append({"kernel": "window chain (window_kernel + next_block_kernel, delayed, one CTA)",
                    "bound": "latency", "ns_per_site": ch["ms"] * 1e6 / de["proposals"],
                    "ns_per_accept": ch["ms"] * 1e6 / de["accepts"], "ms_per_slice": ch["ms"] / de["slices"],
                    "acceptance": de["accepts"] / max(de["proposals"], 1),
                    "note": "the serial Metropolis chain of the delayed update; the bound it is compared "
                            "with is stated in the design notes (one 1024-thread block barrier plus one "
                            "warp scan per accept)"})
    return out


def l2_copy_bandwidth(torch, mb=40, reps=100):
    """Copy bandwidth of an L2-resident working set (src + dst = 2 x mb MB < 129 MB L2): read + write
    bytes / time, CUDA events over `reps` back-to-back copies after a warm-up."""
    n = mb * 1024 * 1024 // 4
    a = torch.ones(n, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    for _ in range(10):
        b.copy_(a)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        b.copy_(a)
    e1.record()
    torch.cuda.synchronize()
    return 2.0 * n * 4 * reps / (e0.elapsed_time(e1) / 1e3) / 1e9


PREC_SLICES = 10  # one recompute period of the headline workload


def precision_report(afqmc, stream, args, seed, X=None, variants=None):
    """Accuracy of each FP32 bulk variant at the headline workload (40 x 40, U = 6, delayed k), over
    one recompute period from the FP64 G(0): slices 1..10 forward, then the FP64 recompute.
    Reference: an FP64-bulk walker running free (decisions, ratios and G after every slice).
    For each variant (the dense wrap with the tensor-core three-term TF32 split, with one TF32 pass,
    or on the FP32 FMA pipes; the separable wrap's L-point passes in FP32, the default):
      replay: the variant replays the reference's decisions.  Per slice: ||G - G_64||_F / ||G_64||_F
              (mean over the spins), the largest relative ratio error over the sites, and the number
              of decisions that would flip (u < |R| with the variant's ratio against the reference's,
              the same uniforms); at slice 10 the drift the FP64 recompute reports.
      free:   the variant runs free with the reference's seed: the first (slice, site) whose decision
              differs from the reference's, or null if none within the period."""
    P = inputs.trial_state(L, L, NS)
    if X is None:
        X = inputs.initial_fields(M, N, seed=seed)
    Pcat = np.concatenate([P.ravel(), P.ravel()])
    S = min(PREC_SLICES, STAB_WORKLOAD)

    def make(precision, gemm, wrap):
        c = afqmc.Context(M, dtau=DTAU, U=U, t=T_HOP, precision=precision, stab_every=STAB_WORKLOAD, seed=seed,
                          gemm=gemm)
        c.init_walkers([L], [NS], [NS], Pcat, X, stream=stream)
        if wrap:
            c.set_wrap(wrap)
        return c

    ref = make("fp64", "tc3", None)
    refG, refdec, refrat = [], [], []
    try:
        for ell in range(1, S + 1):
            ref.sweep_slice(ell, +1, "delayed", k=min(args.k, 64), stream=stream)
            refdec.append(ref.decisions(0)[:N].copy())
            refrat.append(ref.ratios(0)[:N].copy())
            refG.append([ref.G(0, 0), ref.G(0, 1)])
    finally:
        ref.close()
    out = {}
    for name, gemm, wrap in (variants or (("fp32_dense_tc3", "tc3", "dense"), ("tf32_dense", "tf32", "dense"),
                                          ("fp32_dense_simt", "simt", "dense"),
                                          ("fp32_separable", "tc3", "separable"))):
        c = make("fp32", gemm, wrap)
        errs, rerr, flips = [], [], []
        try:
            for ell in range(1, S + 1):
                rep = np.zeros(2 * N, np.uint8)
                rep[:N] = refdec[ell - 1]
                c.sweep_slice(ell, +1, "delayed", k=args.k, replay=rep, stream=stream)
                r = c.ratios(0)[:N]
                r64 = refrat[ell - 1]
                u = inputs.uniforms(seed, 0, ell - 1, 2 * N)[:N]
                rerr.append(float(np.max(np.abs(r - r64) / np.maximum(np.abs(r64), 1e-300))))
                flips.append(int(np.sum((u < np.abs(r)) != (u < np.abs(r64)))))
                errs.append(float(np.mean([np.linalg.norm(c.G(0, s) - refG[ell - 1][s]) /
                                           np.linalg.norm(refG[ell - 1][s]) for s in range(2)])))
            drift = float(c.recompute_G(stream=stream)[0]) if S == STAB_WORKLOAD else None
        finally:
            c.close()
        c = make("fp32", gemm, wrap)
        first = None
        try:
            for ell in range(1, S + 1):
                c.sweep_slice(ell, +1, "delayed", k=args.k, stream=stream)
                diff = np.nonzero(c.decisions(0)[:N] != refdec[ell - 1])[0]
                if diff.size:
                    first = {"slice": ell, "site": int(diff[0]), "decisions_before": (ell - 1) * N + int(diff[0])}
                    break
        finally:
            c.close()
        growth = [errs[i + 1] / errs[i] for i in range(len(errs) - 1) if errs[i] > 0]
        out[name] = {"G_rel_err_per_slice": errs, "G_err_growth_per_slice_median":
                     statistics.median(growth) if growth else None,
                     "max_rel_ratio_err_per_slice": rerr, "decision_flips_per_slice": flips,
                     "recompute_drift_at_period_end": drift, "first_divergence_free_running": first}
    return {"workload": f"{L}x{L}, U={U}, delayed k={args.k}, slices 1..{S} from the FP64 G(0) of the given fields",
            "reference": "FP64 bulk on the GPU, free-running (its G matches the FP64 oracle to 1e-10 in the "
                         "parity tests)", "sites_per_slice": N, "variants": out}


def stab_sweep_leg(afqmc, torch, stream, args, seed, X, stabs=(2, STAB_WORKLOAD)):
    """The FP32 headline sweep at other recompute periods, from the equilibrated fields X of the
    headline walker: per period, one untimed sweep, then one sweep timed with CUDA events on the
    launching stream and the drift ||G_fp32 - G_fp64|| / ||G_fp64|| at each of its recompute points
    (median and max) -- the accuracy bought by recomputing more often, and its cost."""
    P = inputs.trial_state(L, L, NS)
    order = [(l, +1) for l in range(1, M + 1)] + [(l, -1) for l in range(M, 0, -1)]
    out = {}
    for stab in stabs:
        c = afqmc.Context(M, dtau=DTAU, U=U, t=T_HOP, precision="fp32", stab_every=stab, seed=seed, gemm=args.gemm)
        try:
            c.init_walkers([L], [NS], [NS], np.concatenate([P.ravel(), P.ravel()]), X, stream=stream)
            drifts = []

            def sweep(collect):
                for (ell, d) in order:
                    c.sweep_slice(ell, d, "delayed", k=args.k, nb=args.nb, stream=stream)
                    pos = ell if d > 0 else ell - 1
                    if pos % stab == 0:
                        if collect:
                            drifts.append(float(c.recompute_G(stream=stream)[0]))
                        else:
                            afqmc.afqmc_recompute_G(c.h, None, stream)

            sweep(False)
            ms = tune.time_on_stream(torch, stream, lambda: sweep(False))
            sweep(True)
            out[f"stab_{stab}"] = {"value": N * M * 2 / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                                   "recomputes_per_sweep": 2 * M // stab,
                                   "drift_median": statistics.median(drifts), "drift_max": max(drifts)}
        finally:
            c.close()
    return out


def fp64_bulk_leg(afqmc, torch, stream, args, seed):
    """The headline sweep at FP64 bulk (G, the window chain, the flush and the wrap all in FP64; the
    paper's arithmetic is complex FP64): one full sweep (2M slice-steps + recomputes every 10
    slices) timed with CUDA events after a warm-up of 2 slice-steps there and back, then the same
    local / block force-bias / delayed comparison sample as the FP32 line (4 slices each)."""
    P = inputs.trial_state(L, L, NS)
    X = inputs.initial_fields(M, N, seed=seed)
    c = afqmc.Context(M, dtau=DTAU, U=U, t=T_HOP, precision="fp64", stab_every=STAB_WORKLOAD, seed=seed,
                      gemm=args.gemm)
    try:
        c.init_walkers([L], [NS], [NS], np.concatenate([P.ravel(), P.ravel()]), X, stream=stream)
        k64 = min(args.k, 64)
        for (ell, d) in ((1, +1), (2, +1), (2, -1), (1, -1)):
            c.sweep_slice(ell, d, "delayed", k=k64, nb=args.nb, stream=stream)
        afqmc.afqmc_recompute_G(c.h, None, stream)  # back at slice 0: a recompute point
        order = [(l, +1) for l in range(1, M + 1)] + [(l, -1) for l in range(M, 0, -1)]

        def sweep():
            for (ell, d) in order:
                c.sweep_slice(ell, d, "delayed", k=k64, nb=args.nb, stream=stream)
                pos = ell if d > 0 else ell - 1
                if pos % STAB_WORKLOAD == 0:
                    afqmc.afqmc_recompute_G(c.h, None, stream)

        ms = tune.time_on_stream(torch, stream, sweep)
        cmp, _ = compare_modes(afqmc, c, stream, k64, args.nb, 4, elem_bytes=8)
        return {"value": N * M * 2 / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "k": k64,
                "compare_sample": cmp,
                "speedup_update_only_vs_local": {m: cmp[m]["update_only"] / cmp["local"]["update_only"]
                                                 for m in ("delayed", "blockfb")},
                "note": "one sweep of the headline workload with every step in FP64 (k <= 64: the FP64 window "
                        "holds 64 sites)"}
    finally:
        c.close()


def delayed_k_sweep(afqmc, ctx, stream, ks, n_slices, Nsites, stab=STAB):
    """Update-only rate of the local update and of the delayed update at each delay rank k on one
    walker: slices 1..n_slices forward under the phase profiler, then back to slice 0 (delayed,
    untimed) so that every mode starts from the same place."""
    out = {}
    sample = [(l, +1) for l in range(1, n_slices + 1)]
    back = [(l, -1) for l in range(n_slices, 0, -1)]
    for mode, k in [("local", 1)] + [("delayed", k) for k in ks]:
        ctx.set_profiling(True)
        acc = prop = 0
        for (ell, d) in sample:
            st = ctx.sweep_slice(ell, d, mode, k=k, want_stats=True, stream=stream)
            acc += st[0].accepts
            prop += st[0].proposals
            if ell % stab == 0:
                afqmc.afqmc_recompute_G(ctx.h, None, stream)
        p = ctx.profile()
        ctx.set_profiling(False)
        for (ell, d) in back:
            ctx.sweep_slice(ell, d, "delayed", k=max(ks), stream=stream)
            if (ell - 1) % stab == 0:
                afqmc.afqmc_recompute_G(ctx.h, None, stream)
        t = (p["local"]["ms"] if mode == "local" else p["chain"]["ms"]) + p["prep"]["ms"]
        out["local" if mode == "local" else f"delayed_k{k}"] = {
            "update_only": Nsites * n_slices / (t / 1e3),
            "with_wrap": Nsites * n_slices / ((t + p["wrap"]["ms"]) / 1e3), "acceptance": acc / max(prop, 1)}
    base = out["local"]["update_only"]
    for v in out.values():
        v["speedup_update_only_vs_local"] = v["update_only"] / base
    return out


def config_16x16_leg(afqmc, torch, stream, args, seed):
    """The 16 x 16 workload (N = 256, U/t = 4, filling 0.875: 112 per spin, dtau = 0.05, M = 80):
    local update against the delayed update with k in {8, 16, 32, 64}, FP64 and FP32 bulk, on
    20-slice samples of one walker (its recomputes every 10 slices included)."""
    L2, U2, M2 = 16, 4.0, 80
    n2 = inputs.n_sigma_for(L2, FILLING)
    P = inputs.trial_state(L2, L2, n2)
    X = inputs.initial_fields(M2, L2 * L2, seed=seed)
    res = {}
    for prec in ("fp64", "fp32"):
        c = afqmc.Context(M2, dtau=DTAU, U=U2, t=T_HOP, precision=prec, stab_every=STAB_WORKLOAD, seed=seed,
                          gemm=args.gemm)
        try:
            c.init_walkers([L2], [n2], [n2], np.concatenate([P.ravel(), P.ravel()]), X, stream=stream)
            res[prec] = delayed_k_sweep(afqmc, c, stream, (8, 16, 32, 64), 20, L2 * L2, stab=STAB_WORKLOAD)
        finally:
            c.close()
    return {"workload": f"{L2}x{L2} Hubbard, U/t={U2}, n={FILLING} ({n2} per spin), dtau={DTAU}, M={M2}",
            "unit": UNIT, "by_precision": res}


# Nominal dense FP64 rate of a GB300: 1.25 TFLOP/s at the 2070 MHz maximum SM clock, i.e. 2 FP64
# FMA per SM per clock on 152 SMs.  The FP64 rooflines use the rate measured in the same run
# (fp64_gemm_tflops: a cuBLAS DGEMM through torch, as the bf16 peak is a cuBLAS GEMM) when it
# succeeded, else this nominal figure.
FP64_FMA_PER_SM_CLK = 2
FP64_MEASURED = {}
# TF32 tensor rate relative to bf16 (nominal dense 1.1 vs 2.25 PFLOP/s).
TF32_OVER_BF16 = 1.1 / 2.25
# Digit-plane pairs of each FP64-accurate recompute product: the split's cost model picks 6-bit
# digits (s = 9, levels p + q <= 10: 45 pairs) for U_L U_R and U_R Z at 40x40 and for both SOC
# products at 24x24; each pair is one bf16 tensor-core pass over M x N x K.
OZ_PAIRS = 45
# DRAM bytes per launch (read + write) from one ncu capture of the current kernel on this
# workload; None where the phase spans several kernels or no capture of the current kernel exists.
NCU_TRAFFIC = {"elim": None, "lu_o": None,
               "solve": 25.807104e6 + 0.080896e6,      # lu_solve_kernel, 700 x 700, 1600 right-hand sides
               "wrap_gemm": 30.749184e6 + 0.02432e6,   # tc_gemm_kernel<160, split3>, 1600^3, both spins
               "flush_gemm": 22.055936e6 + 0.0,        # rankm_kernel, 1600 x 1600 x m, both spins (writes stay in L2)
               # sep_line_circ_kernel<float, 40>: the four passes of one wrap (cold cache: 20.53 MB read per
               # pass, writes absorbed by L2)
               "sep": 20.528128e6 + 20.528128e6 + 20.528384e6 + 20.553728e6}


def fp32_alu_peak(pk):
    return 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def fp64_alu_peak(pk):
    if "tflops" in FP64_MEASURED:
        return FP64_MEASURED["tflops"]
    return 152 * FP64_FMA_PER_SM_CLK * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def fp64_peak_source(pk, pk_src):
    if "tflops" in FP64_MEASURED:
        return "measured cuBLAS DGEMM %d^3 in this run: %.3f TFLOP/s (of measured)" % (FP64_MEASURED["n"],
                                                                                      FP64_MEASURED["tflops"])
    return ("nominal FP64 1.25 TFLOP/s: 152 SMs x %d FMA x 2 flop x %.0f MHz (of %s peaks)"
            % (FP64_FMA_PER_SM_CLK, pk.get("sm_max_mhz", 2070.0), pk_src))


def fp64_gemm_tflops(torch, n=4096, reps=3):
    """The FP64 denominator: a cuBLAS DGEMM (torch.mm on float64) of n x n x n, CUDA events over
    `reps` products after one warm-up; records it in FP64_MEASURED."""
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    c = torch.mm(a, b)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        torch.mm(a, b, out=c)
    e1.record()
    torch.cuda.synchronize()
    tf = 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) / 1e3) / 1e12
    FP64_MEASURED.update({"tflops": tf, "n": n})
    return tf


def kernel_rooflines(prof, gemm, pk, pk_src, steps, wrap="separable", wrap_tile=0):
    """Per-kernel rooflines from the nested per-launch intervals of the timed region:
    achieved = algorithmic work of the launches / their summed CUDA-event durations.
    Returns a list sorted by total time (the first entry is the dominant kernel)."""
    out = []
    # FP64 recompute: blocked pivoted LU of the propagated N x ns factor (both spins per
    # interval), LU of U_L U_R (ns x ns) and the solve (U_L U_R) Z = U_L with N right-hand sides.
    fp64 = fp64_alu_peak(pk)
    src64 = fp64_peak_source(pk, pk_src)
    dg = prof.get("dgemm", {"ms": 0.0, "intervals": 0})
    n_rc = prof.get("lu_o", {"intervals": 0})["intervals"]
    # The FP32-bulk recompute forms (U_L U_R)^{-1} (a solve with ns right-hand sides) and
    # Z = (U_L U_R)^{-1} U_L as a third digit-split product; otherwise the solve has N right-hand sides.
    inv = n_rc > 0 and dg["intervals"] >= 3 * n_rc
    # (the pivot-ordered identity: column c's forward substitution starts at row c, ns^3 / 3 flop
    # forward and ns^3 backward per matrix)
    solve = (("solve", "lu_solve_kernel (FP64 (U_L U_R)^-1 from the LU, the identity in pivot order, both spins)",
              2 * (4.0 / 3.0) * NS ** 3) if inv else
             ("solve", "lu_solve_kernel (FP64 (U_L U_R) Z = U_L, N right-hand sides, both spins)",
              2 * 2.0 * NS ** 2 * N))
    for name, label, flop in (
            ("elim", "lu_panel_kernel + lu_update_kernel (FP64 LU of the propagated N x ns factor, both spins)",
             2 * (N * NS ** 2 - NS ** 3 / 3.0)),
            ("lu_o", "lu_panel_kernel + lu_update_kernel (FP64 LU of U_L U_R, ns x ns, both spins)",
             2 * (2.0 / 3.0) * NS ** 3),
            solve):
        ph = prof.get(name, {"ms": 0.0, "intervals": 0})
        if ph["intervals"] > 0:
            ach = flop * ph["intervals"] / (ph["ms"] / 1e3) / 1e12
            out.append({"kernel": label, "bound": "alu", "achieved": ach, "peak": fp64, "unit": "TFLOP/s",
                        "frac": ach / fp64, "traffic": None if (name == "solve" and inv) else NCU_TRAFFIC.get(name),
                        "launches": ph["intervals"],
                        "ms_per_launch": ph["ms"] / ph["intervals"], "ms_per_step": ph["ms"] / steps,
                        "work_per_launch": flop, "peak_source": src64})
    if dg["intervals"] > 0:
        # FP64-equivalent flop per product (both spins), averaged over a recompute's products:
        # U_L U_R (ns x ns x N), [(U_L U_R)^{-1} U_L (ns x N x ns),] U_R Z (N x N x ns)
        if inv:
            flop64 = 2.0 * (2 * 2.0 * NS * NS * N + 2.0 * N * N * NS) / 3.0
            what = "U_L U_R, (U_L U_R)^-1 U_L and U_R Z"
        else:
            flop64 = 2.0 * NS * N * (NS + N)
            what = "U_L U_R and U_R Z"
        ach64 = flop64 * dg["intervals"] / (dg["ms"] / 1e3) / 1e12
        ach = OZ_PAIRS * ach64
        out.append({"kernel": "digit-split FP64 products %s (bf16 tcgen05, 45 plane pairs, both spins)" % what,
                    "bound": "tensor", "achieved": ach, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                    "frac": ach / pk["bf16_tflops"], "traffic": None, "launches": dg["intervals"],
                    "ms_per_launch": dg["ms"] / dg["intervals"], "ms_per_step": dg["ms"] / steps,
                    "work_per_launch": OZ_PAIRS * flop64, "fp64_equivalent_tflops": ach64,
                    "fp64_equivalent_vs_fp64_peak": ach64 / fp64,
                    "peak_source": "measured bf16 burst (of %s); achieved counts every plane-pair pass, includes "
                                   "the digit split and the FP64 epilogues" % pk_src})
    wg = prof.get("wrap_gemm", {"ms": 0.0, "intervals": 0})
    if wg["intervals"] > 0 and wrap == "separable":
        # one interval = one wrap (both sides) of both spins: four L-point passes over N^2 elements,
        # each L multiply-adds per element.  The line passes (the default) are four launches that
        # each read and write G; the tile form two.
        flop = 2.0 * 2.0 * 4.0 * L * N * N
        npass = 4 if wrap_tile == 0 else 2
        byts = npass * 2 * 2 * N * N * 4
        ach = flop * wg["intervals"] / (wg["ms"] / 1e3) / 1e12
        peak = fp32_alu_peak(pk)
        name = ("sep_line_kernel (separable wrap: 4 line passes, both spins, FP32)" if wrap_tile == 0 else
                "sep_kernel (separable wrap: 2 tile passes of width %d, both spins, FP32)" % wrap_tile)
        out.append({"kernel": name, "bound": "alu",
                    "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                    "traffic": NCU_TRAFFIC.get("sep") if wrap_tile == 0 else None, "launches": wg["intervals"],
                    "launches_per_interval": npass,
                    "ms_per_launch": wg["ms"] / wg["intervals"], "ms_per_step": wg["ms"] / steps,
                    "work_per_launch": flop, "bytes_per_launch": byts,
                    "gbs": byts * wg["intervals"] / (wg["ms"] / 1e3) / 1e9,
                    "peak_source": "FP32 FMA pipes: 152 SMs x 128 lanes x 2 flop x sm_max_mhz (derived); "
                                   "one 'launch' here is one wrap (both sides, %d kernel launches); "
                                   "arithmetic intensity %.0f flop/B puts it above the HBM ridge"
                                   % (npass, flop / byts)})
    elif wg["intervals"] > 0:
        flop = 2.0 * 2.0 * N ** 3  # one launch = one N x N x N product for both spins
        ach = flop * wg["intervals"] / (wg["ms"] / 1e3) / 1e12
        if gemm == "simt":
            peak, src, bound = fp32_alu_peak(pk), "FP32 FMA pipes: 152 x 128 x 2 x sm_max_mhz", "alu"
        else:
            peak = pk["bf16_tflops"] * TF32_OVER_BF16
            src = "TF32 = measured bf16 burst %.1f x nominal 1.1/2.25 (of %s)" % (pk["bf16_tflops"], pk_src)
            if gemm == "tc3":
                src += "; three TF32 MMAs per product (hi*hi + hi*lo + lo*hi), so frac <= 1/3"
            bound = "tensor"
        out.append({"kernel": "wrap GEMM (%s, both spins per launch)" % gemm, "bound": bound, "achieved": ach,
                    "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": NCU_TRAFFIC["wrap_gemm"],
                    "launches": wg["intervals"], "ms_per_launch": wg["ms"] / wg["intervals"],
                    "ms_per_step": wg["ms"] / steps, "work_per_launch": flop, "peak_source": src})
    fg = prof.get("flush_gemm", {"ms": 0.0, "intervals": 0})
    if fg["intervals"] > 0:
        byts = 2 * 2 * N * N * 4  # read + write of both spins' G (FP32); X and Y' panels are O(N m)
        ach = byts * fg["intervals"] / (fg["ms"] / 1e3) / 1e9
        out.append({"kernel": "rankm_kernel: the rank-m flush product G -= X Y' (SIMT FP32, both spins)", "bound": "hbm",
                    "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
                    "traffic": NCU_TRAFFIC["flush_gemm"], "launches": fg["intervals"],
                    "ms_per_launch": fg["ms"] / fg["intervals"], "ms_per_step": fg["ms"] / steps,
                    "work_per_launch": byts,
                    "peak_source": "measured copy bandwidth (of %s); G (2 x 10 MB) is L2-resident" % pk_src})
    out.sort(key=lambda r: -r["ms_per_step"])
    return out


def walkers_40x40_leg(afqmc, torch, stream, args, seed, counts=(4, 8)):
    """The headline workload with several walkers per GPU: n independent 40 x 40 walkers (seeds
    per walker) in one group, so every launch of a slice covers all of them (n window chains side by
    side, one flush product over 2n matrices, one batched recompute).  Per n: one untimed sweep
    that also captures the slice-steps' graphs, then one sweep timed with CUDA events on the
    stream.  Rate = n x N x 2M / time."""
    P = inputs.trial_state(L, L, NS)
    order = [(l, +1) for l in range(1, M + 1)] + [(l, -1) for l in range(M, 0, -1)]
    out = {"workload": "n walkers of the headline workload (40x40, U=6, n=0.875, k=64, FP32 bulk, recompute "
                       "every %d slices) in one group per GPU" % STAB, "unit": UNIT}
    for n in counts:
        X = np.concatenate([inputs.initial_fields(M, N, seed=seed, walker=wi).ravel() for wi in range(n)])
        c = afqmc.Context(M, dtau=DTAU, U=U, t=T_HOP, precision="fp32", stab_every=STAB, seed=seed, gemm=args.gemm)
        try:
            c.init_walkers([L] * n, [NS] * n, [NS] * n, np.concatenate([np.concatenate([P.ravel(), P.ravel()])] * n),
                           X, stream=stream)

            def sweep():
                for (ell, d) in order:
                    c.sweep_slice(ell, d, "delayed", k=args.k, nb=args.nb, stream=stream)
                    pos = ell if d > 0 else ell - 1
                    if pos % STAB == 0:
                        afqmc.afqmc_recompute_G(c.h, None, stream)

            c.set_graphs(True)
            sweep()
            ms = tune.time_on_stream(torch, stream, sweep)
            out[f"walkers_{n}"] = {"value": n * N * M * 2 / (ms / 1e3), "ms_per_step": ms}
        finally:
            c.close()
    return out


def batched_population(afqmc, torch, stream, args, seed):
    """The mixed walker population: BATCH_WALKERS walkers with L drawn uniformly from
    {8, 12, 16, 24} (seeded), U/t = 4, filling 0.875, M = 40, FP32 bulk with the FP64 recompute every
    10 slices, delayed update.  Walkers of one lattice form a group whose launches cover them all;
    the groups run concurrently.  k is tuned over {16, 32, 64} on one warm-up sweep each; the
    timed sweeps run with and without CUDA-graph replay."""
    Ls = inputs.batch_lattices(BATCH_WALKERS, seed=5)
    Mb, Sb, Ub = 40, 10, 4.0
    ns = [inputs.n_sigma_for(int(L), FILLING) for L in Ls]
    P = np.concatenate([np.concatenate([inputs.trial_state(int(L), int(L), n).ravel()] * 2)
                        for L, n in zip(Ls, ns)])
    X = np.concatenate([inputs.initial_fields(Mb, int(L) * int(L), seed=seed, walker=wi).ravel()
                        for wi, L in enumerate(Ls)])
    ctx = afqmc.Context(Mb, dtau=DTAU, U=Ub, t=T_HOP, precision="fp32", stab_every=Sb, seed=seed, gemm=args.gemm)
    ctx.init_walkers([int(L) for L in Ls], ns, ns, P, X, stream=stream)
    order = [(l, +1) for l in range(1, Mb + 1)] + [(l, -1) for l in range(Mb, 0, -1)]

    def sweep(k):
        for (ell, d) in order:
            ctx.sweep_slice(ell, d, "delayed", k=k, stream=stream)
            pos = ell if d > 0 else ell - 1
            if pos % Sb == 0:
                afqmc.afqmc_recompute_G(ctx.h, None, stream)

    def timed(k, n):
        return tune.time_on_stream(torch, stream, lambda: sweep(k), n)

    def trial(k):
        sweep(k)  # first sweep with this k (warm-up)
        return timed(k, 1)

    kchoice, ktrials = tune.tune(None, "", "k", (16, 32, 64), trial)
    kbest = kchoice.value
    k_ms = {t.value: t.ms for t in ktrials}
    upd = sum(int(L) * int(L) for L in Ls) * 2 * Mb
    ms_direct = timed(kbest, 2)
    ctx.set_graphs(True)
    sweep(kbest)  # captures every slice
    ms_graph = timed(kbest, 2)
    ctx.close()
    sizes = {int(L): int((Ls == L).sum()) for L in sorted(set(Ls.tolist()))}
    return {"metric": "field updates/s, mixed walker population, delayed update", "unit": UNIT,
            "walkers": int(len(Ls)), "walkers_per_L": sizes, "M": Mb, "U": Ub, "stab_every": Sb,
            "k_tuning_ms_per_sweep": k_ms, "k": kbest,
            "value": upd / (min(ms_direct, ms_graph) / 1e3),
            "direct_launches": {"value": upd / (ms_direct / 1e3), "ms_per_sweep": ms_direct},
            "cuda_graphs": {"value": upd / (ms_graph / 1e3), "ms_per_sweep": ms_graph},
            "note": "one sweep = 2M slice-steps of every walker + 8 FP64 recomputes; walkers of one lattice "
                    "share every launch, groups run on concurrent streams"}


SOC_L, SOC_LAM, SOC_U, SOC_M, SOC_STAB = 24, 0.5, -4.0, 80, 10


def soc_leg(torch, stream, args, seed):
    """The spin-orbit-coupled workload: 24 x 24 Rashba-Hubbard lattice (2N = 1152 complex orbitals),
    lambda/t = 0.5, U/t = -4 (spin-y decoupling), half filling (576 particles), dtau = 0.05, M = 80,
    FP32 (complex64) bulk G with the FP64 recompute every 10 slices.  Per mode, a fresh walker sweeps
    slices 1..10 untimed, then the timed sample of slices 11..10+S (with its recomputes) under
    per-phase CUDA events; the local update is the baseline."""
    from paper_2506_09611_gb300 import soc

    n_e = SOC_L * SOC_L
    Ns = SOC_L * SOC_L
    P = inputs.soc_trial_state(SOC_L, n_e, lam=SOC_LAM)
    X = inputs.initial_fields(SOC_M, Ns, seed=seed)
    out = {}
    S = args.soc_slices
    for name, mode, k, nb in (("local", "local", 1, 1), ("delayed_k32", "delayed", 32, 1),
                              ("delayed_k64", "delayed", 64, 1), ("blockfb_nb4", "blockfb", 1, 4),
                              ("blockfb_nb16", "blockfb", 1, 16), ("blockfb_nb64", "blockfb", 1, 64)):
        ctx = soc.SocContext(SOC_L, SOC_M, n_e, 1, "fp32", args.gemm, SOC_STAB, T_HOP, SOC_LAM, SOC_U, DTAU, seed)
        ctx.init(P, X, stream=stream)

        def run(a, b, decisions=None):
            for ell in range(a, b + 1):
                ctx.sweep_slice(ell, +1, mode, k=k, nb=nb, stream=stream)
                if decisions is not None:
                    decisions.append(ctx.decisions(0))
                if ell % SOC_STAB == 0:
                    soc.afqmc_soc_recompute_G(ctx.h, None, stream)

        run(1, 10)
        torch.cuda.synchronize()
        x0 = ctx.fields(0)
        ctx.set_profiling(True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run(11, 10 + S)
        b.record(stream)
        torch.cuda.synchronize()
        prof = ctx.profile()
        ctx.set_profiling(False)
        ms = a.elapsed_time(b)
        flips = int((ctx.fields(0) != x0).sum())
        dec = []
        run(11 + S, min(SOC_M, 12 + S), dec)  # decision sample (untimed): acceptance
        if mode == "blockfb":
            nbk = (Ns + nb - 1) // nb
            acc = float(np.mean([d[Ns:Ns + nbk].mean() for d in dec]))
        else:
            acc = float(np.mean([d[:Ns].mean() for d in dec]))
        upd = Ns * S
        t_upd = prof["prep"]["ms"] + prof["chain"]["ms"] + prof["flush"]["ms"]
        if name == "blockfb_nb16":
            soc_prof = prof
        out[name] = {"update_only": upd / (t_upd / 1e3), "with_wrap": upd / ((t_upd + prof["wrap"]["ms"]) / 1e3),
                     "with_recompute": upd / (ms / 1e3), "acceptance": acc, "flip_rate": flips / upd,
                     "ms_per_slice": {p: prof[p]["ms"] / S for p in prof if prof[p]["intervals"]},
                     "launches_per_slice": sum(v["launches"] for v in prof.values()) / S}
        ctx.close()
    base = out["local"]["update_only"]
    # rooflines of the dominant SOC kernels, from the block force-bias (nb = 16) run's intervals
    pk, pk_src = peaks()
    fp64 = fp64_alu_peak(pk)
    N2, ld2, nv = 2 * Ns, 2 * ((2 * Ns + 31) // 32 * 32), 2 * n_e
    prof = soc_prof
    roofs = []
    wg = prof["wrap_gemm"]
    if wg["intervals"]:
        flop = 2.0 * N2 * ld2 * ld2  # one realified product: the four real products of a complex GEMM
        ach = flop * wg["intervals"] / (wg["ms"] / 1e3) / 1e12
        peak = pk["bf16_tflops"] * TF32_OVER_BF16
        roofs.append({"kernel": "SOC wrap GEMM (realified complex, tc3)", "bound": "tensor", "achieved": ach,
                      "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                      "traffic": 31.897344e6 + 0.003072e6 if args.gemm == "tc3" else None,  # ncu, tc_gemm<144, split3>
                      "launches": wg["intervals"],
                      "ms_per_launch": wg["ms"] / wg["intervals"], "work_per_launch": flop,
                      "peak_source": "TF32 = measured bf16 burst x 1.1/2.25 (of %s); three TF32 MMAs per product"
                                     % pk_src})
    dg = prof.get("dgemm", {"ms": 0.0, "intervals": 0})
    if dg["intervals"]:
        R4 = 2 * N2
        flop64 = (2.0 * nv * nv * R4 + 2.0 * R4 * N2 * nv) / 2.0  # O = L R and P = R Z, averaged
        ach64 = flop64 * dg["intervals"] / (dg["ms"] / 1e3) / 1e12
        roofs.append({"kernel": "digit-split FP64 products (bf16 tcgen05, 45 plane pairs)", "bound": "tensor",
                      "achieved": OZ_PAIRS * ach64, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                      "frac": OZ_PAIRS * ach64 / pk["bf16_tflops"], "launches": dg["intervals"],
                      "ms_per_launch": dg["ms"] / dg["intervals"], "work_per_launch": OZ_PAIRS * flop64,
                      "fp64_equivalent_tflops": ach64, "fp64_equivalent_vs_fp64_peak": ach64 / fp64,
                      "peak_source": "measured bf16 burst (of %s)" % pk_src})
    for name, label, flop in (
            ("elim", "FP64 LU of the realified 4N x 2N_e factor", 2 * (2 * N2 * nv ** 2 - nv ** 3 / 3.0)),
            ("lu_o", "FP64 LU of the realified U_L U_R (2N_e x 2N_e)", (2.0 / 3.0) * nv ** 3),
            ("solve", "FP64 solve with 2N right-hand sides", 2.0 * nv ** 2 * N2)):
        ph = prof[name]
        if ph["intervals"]:
            ach = flop * ph["intervals"] / (ph["ms"] / 1e3) / 1e12
            roofs.append({"kernel": label, "bound": "alu", "achieved": ach, "peak": fp64, "unit": "TFLOP/s",
                          "frac": ach / fp64, "launches": ph["intervals"], "ms_per_launch": ph["ms"] / ph["intervals"],
                          "work_per_launch": flop, "peak_source": fp64_peak_source(pk, pk_src)})
    cpu = None
    if not args.no_cpu_baseline:
        v, cores, secs = soc_oracle_sample()
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "four slice-steps (wrap + block force bias nb = 16) of the FP64 oracle at 24x24 from its "
                         "own G(0) (M = 2 init not timed); %.1f s of CPU work" % secs}
    return {"metric": "field updates/s, spin-orbit-coupled Hubbard 24x24 (complex G 1152x1152)", "unit": UNIT,
            "rooflines": roofs, "cpu_baseline": cpu,
            "config": {"L": SOC_L, "lambda": SOC_LAM, "U": SOC_U, "n_e": n_e, "dtau": DTAU, "M": SOC_M,
                       "stab_every": SOC_STAB, "precision": "fp32 (complex64) bulk, FP64 recompute",
                       "gemm": args.gemm, "timed_slices": S},
            "modes": out,
            "speedup_update_only_vs_local": {m: v["update_only"] / base for m, v in out.items() if m != "local"},
            "speedup_with_wrap_vs_local": {m: v["with_wrap"] / out["local"]["with_wrap"] for m, v in out.items()
                                           if m != "local"}}


def end_to_end(afqmc, torch, stream, args, seed, rank):
    """Per step through the public API with pinned host buffers: afqmc_create +
    afqmc_init_walkers (H2D trial state and fields) + one full sweep + afqmc_measure_energy +
    afqmc_get_fields (D2H configuration) + afqmc_destroy, wall-clock."""
    P = inputs.trial_state(L, L, NS)
    X = inputs.initial_fields(M, N, seed=seed)
    Ph = torch.from_numpy(np.concatenate([P.ravel(), P.ravel()])).pin_memory().numpy()
    Xh = torch.from_numpy(X.copy()).pin_memory().numpy()
    order = [(l, +1) for l in range(1, M + 1)] + [(l, -1) for l in range(M, 0, -1)]
    times = []
    for it in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c = afqmc.Context(M, dtau=DTAU, U=U, t=T_HOP, precision="fp32", stab_every=STAB, seed=seed)
        c.init_walkers([L], [NS], [NS], Ph, Xh, stream=stream)
        for (ell, d) in order:
            c.sweep_slice(ell, d, "delayed", k=args.k, nb=args.nb, stream=stream)
            pos = ell if d > 0 else ell - 1
            if pos % STAB == 0:
                afqmc.afqmc_recompute_G(c.h, None, stream)
        e, s = c.measure_energy(stream=stream)
        Xout = c.fields(0)
        c.close()
        times.append(time.perf_counter() - t0)
    t = times[-1]
    return {"value": N * M * 2 / t, "unit": UNIT, "h2d_bytes_per_step": int(Ph.nbytes + Xh.nbytes),
            "d2h_bytes_per_step": int(Xout.nbytes + 16),
            "note": "create + init_walkers (FP64 left stack and G(0)) + 1 sweep + energy + fields readback"}


CP_L, CP_U, CP_WALKERS, CP_STEPS, CP_EVERY = 16, 4.0, 32, 10, 5


def cpqmc_leg(afqmc, torch, stream, seed):
    """Constrained-path AFQMC (Sec. IV.D): an ensemble of CP_WALKERS walkers on the 16 x 16 Hubbard
    model (U = 4, n = 0.875, dtau = 0.05, FP64) guided by the trial determinant, each step
    e^{-dtau K} with its overlap weight and then the slice's fields by the heat bath (local: one
    site per window; delayed: windows of k sites) or by block force bias, with the comb and a
    re-orthonormalisation every CP_EVERY steps.  Per scheme: two untimed steps, then CP_STEPS steps
    timed with CUDA events on the stream (afqmc_cp_step returns the weights to the host, so each
    step ends synchronised).  Rate = walkers x N field draws per step / time."""
    ns = inputs.n_sigma_for(CP_L, FILLING)
    P = inputs.trial_state(CP_L, CP_L, ns)
    n = CP_L * CP_L
    out = {"workload": f"{CP_L}x{CP_L} Hubbard, U/t={CP_U}, n={FILLING} ({ns} per spin), dtau={DTAU}, "
                       f"{CP_WALKERS} walkers, FP64, comb + re-orthonormalisation every {CP_EVERY} steps",
           "unit": "field updates/s", "steps": CP_STEPS}
    rng = np.random.default_rng(seed)
    for mode, k, nb in (("local", 1, 1), ("delayed", 16, 1), ("delayed", 32, 1), ("blockfb", 1, 8)):
        cp = afqmc.CPContext(CP_L, ns, CP_WALKERS, P, dtau=DTAU, U=CP_U, t=T_HOP, seed=seed)
        try:
            for _ in range(2):
                cp.step(mode, k, nb, stream=stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for i in range(CP_STEPS):
                cp.step(mode, k, nb, stream=stream)
                if (i + 1) % CP_EVERY == 0:
                    cp.comb(float(rng.uniform()), stream=stream)
                    cp.reorth(stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            el, emean = cp.energy(stream=stream)
            key = mode if mode == "local" else (f"delayed_k{k}" if mode == "delayed" else f"blockfb_nb{nb}")
            out[key] = {"value": CP_WALKERS * n * CP_STEPS / (ms / 1e3), "ms_per_step": ms / CP_STEPS,
                        "energy_per_site": float(emean) / n}
        finally:
            cp.close()
    base = out["local"]["value"]
    out["speedup_vs_local"] = {k: v["value"] / base for k, v in out.items() if isinstance(v, dict) and "value" in v}
    return out


def tform_leg(afqmc, torch, stream, args, seed):
    """The headline workload in the paper's own walker state (afqmc_set_form(T): U_R, U_L and
    T = (U_L U_R)^{-1} per spin, Sec. II.C): one warm-up sweep, `steps` timed sweeps with CUDA events
    on the launching stream (L2 flushed between them), then one profiled sweep for the phases."""
    P = inputs.trial_state(L, L, NS)
    X = inputs.initial_fields(M, N, seed=seed)
    order = [(l, +1) for l in range(1, M + 1)] + [(l, -1) for l in range(M, 0, -1)]
    c = afqmc.Context(M, dtau=DTAU, U=U, t=T_HOP, precision="fp32", stab_every=STAB, seed=seed, gemm=args.gemm,
                      form="T")
    try:
        c.init_walkers([L], [NS], [NS], np.concatenate([P.ravel(), P.ravel()]), X, stream=stream)

        def sweep():
            for (ell, d) in order:
                c.sweep_slice(ell, d, "delayed", k=args.k, nb=args.nb, stream=stream)
                pos = ell if d > 0 else ell - 1
                if pos % STAB == 0:
                    afqmc.afqmc_recompute_G(c.h, None, stream)

        sweep()  # warm-up
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        ms = []
        for _ in range(max(1, args.steps)):
            flush.zero_()
            ms.append(tune.time_on_stream(torch, stream, sweep))
        c.set_profiling(True)
        sweep()
        prof = c.profile()
        c.set_profiling(False)
        ms_sweep = statistics.median(ms)
        return {"value": N * M * 2 / (ms_sweep / 1e3), "unit": UNIT, "ms_per_step": ms_sweep,
                "phases_ms_per_step": {k: v["ms"] for k, v in prof.items() if v["intervals"]},
                "note": "T form: the window kernel of the G form on blocks 1 - U_R[J,:] T U_L[:,J]; each window's "
                        "update T <- T - (T U_L[:,I]) W (U_R[I,:] T) and the rows I of U_R run on the main stream "
                        "(no pipelined flush yet); the recompute forms T only"}
    finally:
        c.close()


def dense_wrap_leg(afqmc, torch, stream, args, seed, sep_wrap_ms):
    """The same 40 x 40 sweep with the dense wrap (afqmc_set_wrap(dense): two N x N x N products per
    slice-step on the tcgen05 tensor cores, three-term TF32 split for FP32 accuracy): one warm-up
    sweep, then `steps` timed sweeps with CUDA events on the launching stream (L2 flushed between
    them), the wrap phase from the library's profiler next to the headline's separable wrap, and
    the tensor-core product's roofline."""
    P = inputs.trial_state(L, L, NS)
    X = inputs.initial_fields(M, N, seed=seed)
    order = [(l, +1) for l in range(1, M + 1)] + [(l, -1) for l in range(M, 0, -1)]
    c = afqmc.Context(M, dtau=DTAU, U=U, t=T_HOP, precision="fp32", stab_every=STAB, seed=seed, gemm=args.gemm)
    try:
        c.init_walkers([L], [NS], [NS], np.concatenate([P.ravel(), P.ravel()]), X, stream=stream)
        c.set_wrap("dense")

        def sweep():
            for (ell, d) in order:
                c.sweep_slice(ell, d, "delayed", k=args.k, nb=args.nb, stream=stream)
                pos = ell if d > 0 else ell - 1
                if pos % STAB == 0:
                    afqmc.afqmc_recompute_G(c.h, None, stream)

        sweep()  # warm-up
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        ms = []
        for _ in range(max(1, args.steps)):
            flush.zero_()
            ms.append(tune.time_on_stream(torch, stream, sweep))
        c.set_profiling(True)
        sweep()
        prof = c.profile()
        c.set_profiling(False)
        ms_sweep = statistics.median(ms)
        pk, pk_src = peaks()
        roof = [r for r in kernel_rooflines(prof, args.gemm, pk, pk_src, 1, wrap="dense")
                if r["kernel"].startswith("wrap GEMM")]
        return {"value": N * M * 2 / (ms_sweep / 1e3), "unit": UNIT, "ms_per_step": ms_sweep,
                "wrap_ms_per_step": prof["wrap"]["ms"], "separable_wrap_ms_per_step": sep_wrap_ms,
                "wrap_gemm_roofline": roof[0] if roof else None,
                "note": "the headline workload with afqmc_set_wrap(dense): the tcgen05 tensor-core wrap"}
    finally:
        c.close()


if __name__ == "__main__":
    main()
