"""Host-side statistics of the pairing production run (paper_2506_09611_gb300.pairing): the jackknife
and the condensate fraction n_c = lambda_max(M - delta <n_up> <n_-k dn>) / (N_e / 2) of Sec. IV,
against identities that fix them: for a linear estimator the jackknife error is the standard error
of the block mean; a Slater determinant (the free Fermi sea, through the oracle's Wick contractions)
has n_c = 0; a single coherent pair amplitude of norm^2 N_e / 2 has n_c = 1."""
import numpy as np

import oracle
from paper_2506_09611_gb300 import pairing


def test_jackknife_of_the_mean_is_the_standard_error():
    rng = np.random.default_rng(5)
    x = rng.standard_normal(17) * 0.3 + 2.0
    mean, err = pairing.jackknife(x, lambda v: v)
    assert abs(mean - x.mean()) < 1e-15
    assert abs(err - x.std(ddof=1) / np.sqrt(len(x))) < 1e-14


def test_condensate_fraction_of_the_free_fermi_sea_is_zero():
    L, ns = 4, 5
    N = L * L
    m = oracle.SocModel(L, 1.0, 0.0, 0.0, 0.1, 2, hs="sz")
    k = 2 * np.pi * np.arange(L) / L
    kx, ky = np.meshgrid(k, k)
    occ = np.argsort((-2 * (np.cos(kx) + np.cos(ky))).ravel(), kind="stable")[:ns]
    xs, ys = np.arange(N) % L, np.arange(N) // L
    Pk = np.stack([np.exp(1j * (2 * np.pi * (q % L) / L * xs + 2 * np.pi * (q // L) / L * ys)) / np.sqrt(N)
                   for q in occ], axis=1)
    P = np.zeros((2 * N, 2 * ns), np.complex128)
    P[:N, :ns] = Pk
    P[N:, ns:] = Pk.conj()
    r = m.pairing(np.eye(2 * N) - P @ P.conj().T)
    assert abs(pairing.n_c(r["Mk"], r["nk"], L, 2 * ns)) < 1e-12


def test_condensate_fraction_of_one_coherent_pair_mode_is_one():
    L, n_e = 3, 6
    N = L * L
    rng = np.random.default_rng(2)
    phi = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    phi *= np.sqrt(n_e / 2) / np.linalg.norm(phi)
    Mk = np.outer(phi, phi.conj())
    assert abs(pairing.n_c(Mk, np.zeros(2 * N), L, n_e) - 1.0) < 1e-12
