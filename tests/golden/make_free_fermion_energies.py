"""Write free_fermion_energies.txt: U = 0 ground-state energies of the configured lattices.

At U = 0 the trial state's energy is the sum of the lowest single-particle levels (Eq. 2DHubbard:
eps_k = -2t (cos kx + cos ky) on the periodic L x L lattice, two spins; Eq. 2DSocHubbard: the two
bands eps_k +- |L_k| with L_k = 2 lam (sin ky - i sin kx), N_e particles in total).  The values are
written from these dispersion relations alone -- no oracle, no GPU path -- and the pins check that
the oracle reproduces them.  Run from the repository root:  python tests/golden/make_free_fermion_energies.py
"""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

# (name, kind, L, particles, t, lam, citation)
CASES = [
    ("hubbard_4x4", "hubbard", 4, 7, 1.0, 0.0, "Eq. 2DHubbard; 7 per spin"),
    ("hubbard_16x16", "hubbard", 16, 112, 1.0, 0.0, "Eq. 2DHubbard; filling 0.875, 112 per spin"),
    ("hubbard_40x40", "hubbard", 40, 700, 1.0, 0.0, "Eq. 2DHubbard; filling 0.875, 700 per spin"),
    ("soc_4x4", "soc", 4, 12, 1.0, 0.5, "Eq. 2DSocHubbard; lam = 0.5, 12 particles"),
    ("soc_24x24", "soc", 24, 576, 1.0, 0.5, "Eq. 2DSocHubbard; lam = 0.5, half filling, 576 particles"),
]


def levels(kind, L, t, lam):
    k = 2 * np.pi * np.arange(L) / L
    kx, ky = np.meshgrid(k, k, indexing="xy")
    eps = -2.0 * t * (np.cos(kx) + np.cos(ky))
    if kind == "hubbard":
        return np.sort(eps.ravel())
    absL = 2.0 * lam * np.sqrt(np.sin(ky) ** 2 + np.sin(kx) ** 2)
    return np.sort(np.concatenate([(eps - absL).ravel(), (eps + absL).ravel()]))


def energy(kind, L, n, t, lam):
    e = levels(kind, L, t, lam)
    return 2.0 * e[:n].sum() if kind == "hubbard" else e[:n].sum()


def lines():
    out = ["# name  kind  L  particles  t  lam  E(U=0)  citation"]
    for name, kind, L, n, t, lam, cite in CASES:
        out.append(f"{name} {kind} {L} {n} {t!r} {lam!r} {energy(kind, L, n, t, lam):.12f} # {cite}")
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "free_fermion_energies.txt"), "w") as f:
        f.write("\n".join(lines()) + "\n")
