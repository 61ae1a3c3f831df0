"""Seeded synthetic inputs shared by the tests, the bench and the oracle legs.

This module holds none of the update method's arithmetic: it only produces
the inputs the paper's workloads are made of (Sec. II.A, II.B):

* ``trial_state``  -- the trial Slater determinant P (N x n_sigma): the lowest
  n_sigma orbitals of the nearest-neighbour hopping matrix.  Every lattice of
  interest has an open shell at the Fermi level, so a fixed 1e-6 symmetric
  perturbation (seed 0) picks one orthonormal set inside the degenerate shell.
* ``initial_fields`` -- i.i.d. +-1 auxiliary fields (p = 1/2) for M slices.
* ``uniforms``      -- the Metropolis / proposal uniforms of one slice visit.
  They come from the counter-based Philox4x64-10 generator (Salmon et al.,
  SC'11) as implemented by numpy: block counter (j + 1, visit, 0, 0), key
  (seed, walker), word 0 of each block, u = (word >> 11) * 2^-53.  The CUDA
  library draws the same stream on the device with its own Philox; a GPU test
  checks the two bit for bit.
* ``batch_lattices`` -- the mixed-size walker population.
* ``soc_hamiltonian`` / ``soc_trial_state`` -- the spin-orbit-coupled model of
  Appendix A on the 2N orbital basis (i spin up, N + i spin down) and its trial
  state: the lowest N_e orbitals of H0 + 1e-6 * S with S a fixed random
  time-reversal-invariant Hermitian matrix, so the occupied set is closed under
  time reversal (the condition for a sign-free weight with the spin-y fields).
"""
from __future__ import annotations

import numpy as np


def hopping_matrix(Lx: int, Ly: int, t: float = 1.0) -> np.ndarray:
    """Periodic nearest-neighbour hopping, K_ij = -t per bond (site i = x + Lx*y)."""
    N = Lx * Ly
    K = np.zeros((N, N))
    for y in range(Ly):
        for x in range(Lx):
            i = x + Lx * y
            for (xx, yy) in (((x + 1) % Lx, y), ((x - 1) % Lx, y), (x, (y + 1) % Ly), (x, (y - 1) % Ly)):
                K[i, xx + Lx * yy] -= t
    return K


def trial_state(Lx: int, Ly: int, n_sigma: int, t: float = 1.0, seed: int = 0) -> np.ndarray:
    """Lowest n_sigma eigenvectors of K + 1e-6 * S (S a fixed random symmetric matrix)."""
    K = hopping_matrix(Lx, Ly, t)
    rng = np.random.Generator(np.random.Philox(key=np.array([seed, 0xC0FFEE], dtype=np.uint64)))
    S = rng.standard_normal(K.shape)
    S = 0.5 * (S + S.T)
    w, v = np.linalg.eigh(K + 1e-6 * S)
    return np.ascontiguousarray(v[:, :n_sigma])


def initial_fields(M: int, N: int, seed: int = 1, walker: int = 0) -> np.ndarray:
    """M x N int8 fields, i.i.d. +-1 with probability 1/2."""
    rng = np.random.Generator(np.random.Philox(key=np.array([seed, 0xF1E1D + walker], dtype=np.uint64)))
    return np.where(rng.random((M, N)) < 0.5, 1, -1).astype(np.int8)


def philox_words(seed: int, walker: int, visit: int, count: int) -> np.ndarray:
    """Word 0 of the Philox4x64-10 blocks with counters (j+1, visit, 0, 0), j < count."""
    bg = np.random.Philox(key=np.array([seed, walker], dtype=np.uint64),
                          counter=np.array([0, visit, 0, 0], dtype=np.uint64))
    raw = bg.random_raw(4 * count)
    return raw[0::4].copy()


def uniforms(seed: int, walker: int, visit: int, count: int) -> np.ndarray:
    """Uniforms in [0, 1) with 53 random bits, in the device generator's layout."""
    w = philox_words(seed, walker, visit, count)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def batch_lattices(n_walkers: int, seed: int = 5, sizes=(8, 12, 16, 24)) -> np.ndarray:
    """Linear sizes drawn uniformly from `sizes` for a mixed walker population."""
    rng = np.random.Generator(np.random.Philox(key=np.array([seed, 0xBA7C4], dtype=np.uint64)))
    return np.asarray(sizes)[rng.integers(0, len(sizes), n_walkers)].astype(np.int32)


def n_sigma_for(L: int, filling: float) -> int:
    """Particles per spin at total filling n = N_e / N_s (N_up = N_dn)."""
    return int(round(filling * L * L / 2))


def soc_hamiltonian(L: int, t: float = 1.0, lam: float = 0.5) -> np.ndarray:
    """Real-space 2N x 2N H0 of the Rashba-coupled square lattice (Eq. 2DSocHubbard), written bond
    by bond: -t per nearest-neighbour bond in each spin block, and the spin-flip hopping
    (H0)[(dn, r), (up, r')] = -i lam for r' = r + y, +i lam for r' = r - y, -lam for r' = r + x,
    +lam for r' = r - x, with the up-down block its Hermitian conjugate."""
    N = L * L
    H = np.zeros((2 * N, 2 * N), np.complex128)
    H[:N, :N] = hopping_matrix(L, L, t)
    H[N:, N:] = hopping_matrix(L, L, t)
    for y in range(L):
        for x in range(L):
            r = x + L * y
            for (dx, dy, amp) in ((0, 1, -1j * lam), (0, -1, 1j * lam), (1, 0, -lam), (-1, 0, lam)):
                rp = (x + dx) % L + L * ((y + dy) % L)
                H[N + r, rp] += amp
                H[rp, N + r] += np.conj(amp)
    return H


def soc_trs_perturbation(N: int, seed: int = 0) -> np.ndarray:
    """A fixed random Hermitian S = [[A, B], [-conj(B), conj(A)]] (A Hermitian, B antisymmetric):
    the general time-reversal-invariant one-body matrix on the 2N orbitals."""
    rng = np.random.Generator(np.random.Philox(key=np.array([seed, 0x50C], dtype=np.uint64)))
    A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    A = 0.5 * (A + A.conj().T)
    B = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    B = 0.5 * (B - B.T)
    return np.block([[A, B], [-B.conj(), A.conj()]])


def soc_trial_state(L: int, n_e: int, t: float = 1.0, lam: float = 0.5, seed: int = 0) -> np.ndarray:
    """Lowest n_e orbitals (2N x n_e, complex, orthonormal columns) of H0 + 1e-6 S."""
    H = soc_hamiltonian(L, t, lam) + 1e-6 * soc_trs_perturbation(L * L, seed)
    w, v = np.linalg.eigh(H)
    return np.ascontiguousarray(v[:, :n_e])


def twisted_hopping_matrix(L: int, twist, t: float = 1.0) -> np.ndarray:
    """Nearest-neighbour hopping on the periodic L x L lattice threaded by a flux: the bond from site
    i to its +x (+y) neighbour carries the phase e^{i twist[0] / L} (e^{i twist[1] / L}), so the
    eigenvectors are the plane waves e^{ik.r} with energies -2t (cos(kx + twist[0]/L) +
    cos(ky + twist[1]/L)).  Hermitian; K_ij is the amplitude of c+_i c_j."""
    N = L * L
    K = np.zeros((N, N), np.complex128)
    for y in range(L):
        for x in range(L):
            i = x + L * y
            for (xx, yy), ph in ((((x + 1) % L, y), twist[0] / L), ((x, (y + 1) % L), twist[1] / L)):
                j = xx + L * yy
                K[i, j] -= t * np.exp(-1j * ph)
                K[j, i] -= t * np.exp(1j * ph)
    return K


def sz_trial_state(L: int, n_sigma: int, t: float = 1.0, seed: int = 0, twist=None) -> np.ndarray:
    """The spin-balanced trial determinant of the Hubbard model on the 2N spin orbitals (up block
    first): P = [[P_up, 0], [0, conj(P_up)]], the condition of Sec. II.B under which the imaginary
    spin-z decoupling has no sign problem.  2N x 2 n_sigma complex, orthonormal columns.

    twist None: P_up = trial_state(L, L, n_sigma) (real; the open shell's degeneracy broken by a
    fixed random 1e-6 perturbation).  twist = (theta_x, theta_y): P_up = the lowest n_sigma
    eigenvectors of twisted_hopping_matrix(L, twist), i.e. the plane waves of the n_sigma lowest
    twisted energies (an open shell filled by the flux's ordering), and P_dn holds the opposite
    momenta."""
    N = L * L
    if twist is None:
        Ps = trial_state(L, L, n_sigma, t, seed)
    else:
        w, v = np.linalg.eigh(twisted_hopping_matrix(L, twist, t))
        Ps = v[:, :n_sigma]
    P = np.zeros((2 * N, 2 * n_sigma), np.complex128)
    P[:N, :n_sigma] = Ps
    P[N:, n_sigma:] = np.conj(Ps)
    return P
