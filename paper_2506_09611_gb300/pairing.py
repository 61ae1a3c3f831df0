"""Production runs of the attractive Hubbard model with the paper's decoupling and its pairing
benchmarks (Sec. II.B and Sec. IV): the imaginary spin-z channel (Eqs. HSspinDecomp,
BIOpForHubbard) in the spin-coupled engine with lam = 0, a spin-balanced trial state
(P_dn = conj(P_up), so the walk is sign-free), and at the middle slice l = M/2 of every half sweep
the double occupancy D, the on-site pairing correlator <Delta^2> and the k-space pairing matrix,
from which the condensate fraction n_c = lambda_max / (N_e / 2) follows (afqmc_soc_measure_pairing).

    python -m paper_2506_09611_gb300.pairing --L 20 --U -4 --filling 1.0 --dtau 0.05 --two-theta 46 \\
        --walkers 32 --warmup 20 --sweeps 40 --mode delayed --k 32 --out pairing.json

Statistics.  Walkers are independent chains: D and <Delta^2> take the mean over the walkers of each
walker's time average and its standard error; n_c (largest eigenvalue of the Hermitian part of the
averaged M[k][k'] - delta_kk' <n_{k up}> <n_{-k dn}>) takes a jackknife over the walkers.
"""
import argparse
import json
import time

import numpy as np

from . import afqmc, inputs, soc

# Flux (theta_x, theta_y) whose ordering of the twisted plane waves fills the open shell of the trial
# determinant: small and incommensurate, so that it splits every degenerate level without moving any
# across a shell.
TWIST = (0.1, 0.07)


def trial(L, ns, kind="twist"):
    """The trial determinant of a pairing run (2N x 2 ns, P_dn = conj(P_up)).  "twist": the plane
    waves of the ns lowest twisted energies for spin up and the opposite momenta for spin down.  At
    half filling it is a pseudospin singlet: eta^2 = 0 for the eta-pairing operators
    eta+ = sum_i (-1)^i c+_iup c+_idn, which commute with H, and the half-filled ground state has
    eta = 0.  "random": the lowest eigenvectors of the hopping plus a fixed 1e-6 random perturbation
    (real, the same for both spins); at half filling it has components with eta > 0, which the
    projection removes only at the rate of their small finite-size gap."""
    return inputs.sz_trial_state(L, ns, twist=TWIST if kind == "twist" else None)


def n_c(Mk, nk, L, n_e):
    """Condensate fraction from averaged Mk (N x N) and averaged nk (2N: up, then down)."""
    N = L * L
    minus = np.array([(L - k % L) % L + L * ((L - k // L) % L) for k in range(N)])
    Mm = Mk - np.diag(nk[:N] * nk[N:][minus])
    H = 0.5 * (Mm + Mm.conj().T)
    return float(np.linalg.eigvalsh(H)[-1].real) / (n_e / 2.0)


def jackknife(samples, fn):
    """Mean over the blocks (fn of the full average) and the jackknife error."""
    B = len(samples)
    full = fn(np.mean(samples, axis=0))
    if B < 2:
        return full, float("nan")
    tot = np.sum(samples, axis=0)
    jk = np.array([fn((tot - samples[b]) / (B - 1)) for b in range(B)])
    return float(full), float(np.sqrt((B - 1) / B * np.sum((jk - jk.mean()) ** 2)))


def run(a):
    import torch

    afqmc.load()
    stream = torch.cuda.current_stream()
    L, N = a.L, a.L * a.L
    ns = inputs.n_sigma_for(L, a.filling) if a.ns is None else a.ns
    M = int(round(a.two_theta / a.dtau))
    if M % a.stab or M % 2:
        raise SystemExit(f"M = {M} must be even and a multiple of --stab {a.stab}")
    mid = M // 2
    ctx = soc.SocContext(L, M, 2 * ns, a.walkers, a.precision, a.gemm, a.stab, 1.0, 0.0, a.U, a.dtau, a.seed, hs="sz")
    P = trial(L, ns, a.trial)
    Dsum = np.zeros(a.walkers)
    Psum = np.zeros(a.walkers)
    Msum = np.zeros((a.walkers, N, N), np.complex128)
    nksum = np.zeros((a.walkers, 2 * N), np.complex128)
    rounds = 0
    acc = {"proposals": 0, "accepts": 0}
    t0 = time.perf_counter()
    with ctx:
        ctx.init(P, stream=stream)
        order = [(l, +1) for l in range(1, M + 1)] + [(l, -1) for l in range(M, 0, -1)]
        for sweep in range(a.warmup + a.sweeps):
            for ell, d in order:
                ctx.sweep_slice(ell, d, a.mode, k=a.k, nb=a.nb, stream=stream)
                pos = ell if d > 0 else ell - 1
                if pos % a.stab == 0:
                    ctx.recompute_G(stream=stream)
                if pos == mid and sweep >= a.warmup:
                    r = ctx.measure_pairing(stream=stream)
                    Dsum += r["D"].real
                    Psum += r["Delta2"].real
                    Msum += r["Mk"]
                    nksum += r["nk"]
                    rounds += 1
                    dec = np.concatenate([ctx.decisions(w)[:N] for w in range(a.walkers)])
                    if a.mode != "blockfb":
                        acc["proposals"] += dec.size
                        acc["accepts"] += int(dec.sum())
            if a.verbose:
                print(f"sweep {sweep + 1}/{a.warmup + a.sweeps}: {time.perf_counter() - t0:.1f} s", flush=True)
    secs = time.perf_counter() - t0
    Dw, Pw = Dsum / rounds, Psum / rounds  # per-walker time averages
    D = (float(Dw.mean()), float(Dw.std(ddof=1) / np.sqrt(len(Dw))) if len(Dw) > 1 else float("nan"))
    P2 = (float(Pw.mean()), float(Pw.std(ddof=1) / np.sqrt(len(Pw))) if len(Pw) > 1 else float("nan"))
    packed = np.concatenate([(Msum / rounds).reshape(a.walkers, -1), nksum / rounds], axis=1)
    nc = jackknife(packed, lambda x: n_c(x[:N * N].reshape(N, N), x[N * N:], L, 2 * ns))
    out = {"model": "attractive Hubbard, imaginary spin-z decoupling (spin-coupled engine, lam = 0)",
           "L": L, "U": a.U, "filling": 2 * ns / N, "n_sigma": ns, "dtau": a.dtau, "two_theta": M * a.dtau, "M": M,
           "trial": a.trial, "twist": TWIST if a.trial == "twist" else None, "stab_every": a.stab, "mode": a.mode, "k": a.k, "nb": a.nb, "precision": a.precision, "gemm": a.gemm,
           "walkers": a.walkers, "warmup_sweeps": a.warmup, "sweeps": a.sweeps, "rounds": rounds,
           "seconds": secs, "D": D, "Delta2": P2, "n_c": nc,
           "acceptance": acc["accepts"] / acc["proposals"] if acc["proposals"] else None}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--L", type=int, default=20)
    ap.add_argument("--U", type=float, default=-4.0)
    ap.add_argument("--filling", type=float, default=1.0, help="electrons per site (both spins)")
    ap.add_argument("--ns", type=int, default=None, help="electrons per spin (overrides --filling)")
    ap.add_argument("--dtau", type=float, default=0.05)
    ap.add_argument("--two-theta", type=float, default=46.0, help="projection time 2 Theta (M = 2 Theta / dtau)")
    ap.add_argument("--walkers", type=int, default=32)
    ap.add_argument("--warmup", type=int, default=20, help="sweeps (out and back) before measuring")
    ap.add_argument("--sweeps", type=int, default=40, help="measured sweeps")
    ap.add_argument("--mode", default="delayed", choices=["local", "delayed", "blockfb"])
    ap.add_argument("--k", type=int, default=32)
    ap.add_argument("--nb", type=int, default=16)
    ap.add_argument("--stab", type=int, default=10)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--gemm", default="tc3", choices=["tc3", "simt", "tf32"])
    ap.add_argument("--trial", default="twist", choices=["twist", "random"], help="trial determinant (see trial())")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--out", default=None)
    ap.add_argument("--verbose", action="store_true")
    a = ap.parse_args(argv)
    out = run(a)
    s = json.dumps(out)
    if a.out:
        with open(a.out, "w") as f:
            f.write(s + "\n")
    print(s)
    return out


if __name__ == "__main__":
    main()
