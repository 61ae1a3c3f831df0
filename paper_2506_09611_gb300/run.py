"""Command-line driver: one walker of the square-lattice Hubbard model (or, with --soc, of the
spin-orbit-coupled model on the 2N complex orbitals) swept for a given number of slice-steps
through the C ABI (used for kernel profiling and quick timing).

    python -m paper_2506_09611_gb300.run --L 40 --U 6 --slices 20 --mode delayed --k 64
    python -m paper_2506_09611_gb300.run --soc --L 24 --U -4 --lam 0.5 --slices 12 --mode blockfb --nb 16
    python -m paper_2506_09611_gb300.run --L 40 --tune tune.json --slices 20 --mode blockfb
    python -m paper_2506_09611_gb300.run --L 40 --wrap separable --slices 20

With --tune CACHE the delay rank and the block size are first chosen by timed trial walks
(tune.autotune_walker: k by time, n_b by time under the acceptance floor) or read from the JSON
cache for this device and workload; the walk then runs with the chosen values.

The walk goes forward from slice 1 and turns at slice M, with the FP64 recompute at every
multiple of --stab, exactly as in a full sweep; the inputs are the seeded synthetic trial
state and fields of the package's input module.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import afqmc, inputs, tune


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=40)
    ap.add_argument("--U", type=float, default=6.0)
    ap.add_argument("--t", type=float, default=1.0)
    ap.add_argument("--dtau", type=float, default=0.05)
    ap.add_argument("--M", type=int, default=80)
    ap.add_argument("--filling", type=float, default=0.875)
    ap.add_argument("--stab", type=int, default=10)
    ap.add_argument("--slices", type=int, default=20, help="slice-steps to run after initialisation")
    ap.add_argument("--mode", default="delayed", choices=["local", "delayed", "blockfb"])
    ap.add_argument("--k", type=int, default=64)
    ap.add_argument("--nb", type=int, default=16)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--gemm", default="tc3", choices=["tc3", "simt", "tf32"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--soc", action="store_true", help="the spin-orbit-coupled model at half filling")
    ap.add_argument("--lam", type=float, default=0.5)
    ap.add_argument("--wrap", default=None, choices=["dense", "separable"],
                    help="wrap products: dense N x N, or L-point passes with exp(-dtau K) = Ex (x) Ex (the "
                         "default for the Hubbard model)")
    ap.add_argument("--wrap-tile", type=int, default=0,
                    help="tile width of the separable wrap (0: the default line passes; --tune chooses it with --wrap separable)")
    ap.add_argument("--tune", metavar="CACHE", help="choose k and nb by timed trials (cached in this JSON file)")
    ap.add_argument("--tune-slices", type=int, default=10, help="slices of each trial walk (out and back)")
    ap.add_argument("--floor", type=float, default=tune.ACCEPTANCE_FLOOR, help="block force-bias acceptance floor")
    a = ap.parse_args(argv)
    if a.soc and a.wrap == "separable":
        ap.error("--wrap separable covers the Hubbard model only (the spin-orbit propagator does not factor)")
    if a.wrap is None:
        a.wrap = "dense" if a.soc else "separable"
    if a.soc:
        return main_soc(a)

    import torch

    afqmc.load()
    stream = torch.cuda.current_stream()
    L, N = a.L, a.L * a.L
    ns = inputs.n_sigma_for(L, a.filling)
    P = inputs.trial_state(L, L, ns)
    X = inputs.initial_fields(a.M, N, seed=a.seed)
    ctx = afqmc.Context(a.M, dtau=a.dtau, U=a.U, t=a.t, precision=a.precision, stab_every=a.stab, seed=a.seed,
                        gemm=a.gemm)
    ctx.init_walkers([L], [ns], [ns], np.concatenate([P.ravel(), P.ravel()]), X, stream=stream)
    ctx.set_wrap(a.wrap)
    if a.wrap == "separable" and a.wrap_tile:
        ctx.set_wrap_tile(a.wrap_tile)
    tuned = None
    if a.tune:
        key = tune.workload_key(device=torch.cuda.get_device_name(), L=L, n_up=ns, n_dn=ns, U=a.U, t=a.t,
                                dtau=a.dtau, M=a.M, stab=a.stab, precision=a.precision, gemm=a.gemm, wrap=a.wrap)
        r = tune.autotune_walker(ctx, torch, stream, lambda st: afqmc.afqmc_recompute_G(ctx.h, None, st),
                                 min(a.tune_slices, a.M), a.stab, floor=a.floor, cache=tune.TuneCache(a.tune),
                                 key=key, k_max=128 if a.precision == "fp32" else 64,
                                 tile_candidates=(0, 4, 8, 16) if a.wrap == "separable" else None)
        a.k, a.nb = r["k"].value, r["nb"].value
        tuned = {"k": r["k"].value, "k_ms": r["k"].ms, "nb": r["nb"].value, "nb_ms": r["nb"].ms,
                 "nb_acceptance": r["nb"].acceptance, "cached": not r["k_trials"] and not r["nb_trials"]}
        if "tile" in r:
            tuned["wrap_tile"] = r["tile"].value
    order = [(l, +1) for l in range(1, a.M + 1)] + [(l, -1) for l in range(a.M, 0, -1)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(a.slices):
        ell, d = order[i % len(order)]
        ctx.sweep_slice(ell, d, a.mode, k=a.k, nb=a.nb, stream=stream)
        pos = ell if d > 0 else ell - 1
        if pos % a.stab == 0:
            afqmc.afqmc_recompute_G(ctx.h, None, stream)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    e, s = ctx.measure_energy(stream=stream)
    ctx.close()
    out = {"L": L, "slices": a.slices, "mode": a.mode, "k": a.k, "nb": a.nb, "precision": a.precision,
           "gemm": a.gemm, "wrap": a.wrap, "wrap_tile": a.wrap_tile, "seconds": dt, "field_updates_per_s": N * a.slices / dt,
           "energy": float(e[0])}
    if tuned is not None:
        out["tuned"] = tuned
    print(json.dumps(out))


def main_soc(a):
    import torch

    from . import soc

    afqmc.load()
    stream = torch.cuda.current_stream()
    L, N = a.L, a.L * a.L
    n_e = N  # half filling
    P = inputs.soc_trial_state(L, n_e, t=a.t, lam=a.lam)
    X = inputs.initial_fields(a.M, N, seed=a.seed)
    ctx = soc.SocContext(L, a.M, n_e, 1, a.precision, a.gemm, a.stab, a.t, a.lam, a.U, a.dtau, a.seed)
    ctx.init(P, X, stream=stream)
    tuned = None
    if a.tune:
        def counted(ell, d, nb):  # one block force-bias slice; accepted blocks from the decisions
            ctx.sweep_slice(ell, d, "blockfb", k=a.k, nb=nb, stream=stream)
            nblk = (N + nb - 1) // nb
            return int(ctx.decisions(0)[N:N + nblk].sum()), nblk

        key = tune.workload_key(device=torch.cuda.get_device_name(), model="soc", L=L, n_e=n_e, U=a.U, t=a.t,
                                lam=a.lam, dtau=a.dtau, M=a.M, stab=a.stab, precision=a.precision, gemm=a.gemm)
        kmax = soc.KMAX[a.precision]
        r = tune.autotune_walker(ctx, torch, stream, lambda st: soc.afqmc_soc_recompute_G(ctx.h, None, st),
                                 min(a.tune_slices, a.M), a.stab, floor=a.floor, cache=tune.TuneCache(a.tune),
                                 key=key, k_max=kmax, nb_max=kmax, counted=counted)
        a.k, a.nb = r["k"].value, r["nb"].value
        tuned = {"k": r["k"].value, "k_ms": r["k"].ms, "nb": r["nb"].value, "nb_ms": r["nb"].ms,
                 "nb_acceptance": r["nb"].acceptance, "cached": not r["k_trials"] and not r["nb_trials"]}
    order = [(l, +1) for l in range(1, a.M + 1)] + [(l, -1) for l in range(a.M, 0, -1)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(a.slices):
        ell, d = order[i % len(order)]
        ctx.sweep_slice(ell, d, a.mode, k=a.k, nb=a.nb, stream=stream)
        pos = ell if d > 0 else ell - 1
        if pos % a.stab == 0:
            soc.afqmc_soc_recompute_G(ctx.h, None, stream)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    e = ctx.measure_energy(stream=stream)
    ctx.close()
    out = {"model": "soc", "L": L, "slices": a.slices, "mode": a.mode, "k": a.k, "nb": a.nb,
           "precision": a.precision, "gemm": a.gemm, "seconds": dt, "field_updates_per_s": N * a.slices / dt,
           "energy": [e[0].real, e[0].imag]}
    if tuned is not None:
        out["tuned"] = tuned
    print(json.dumps(out))


if __name__ == "__main__":
    main()
