"""Pins of the oracle's pairing observables (Sec. IV: double occupancy D, the on-site pairing correlator
<Delta^2> and the k-space pairing matrix behind the condensate fraction n_c) against Fock-space brute
force: the mixed expectation <psi_l| O |psi_r> / <psi_l|psi_r> between two random complex Slater
determinants on a 2 x 2 lattice (8 spin orbitals) and, sparse, on 3 x 3 (18), with every operator built from the Fock-space
annihilators and the momentum operators c_k = N^{-1/2} sum_j e^{-i k.r_j} c_j written out.  This fixes
the Wick contractions, their signs and index order, the Fourier convention and the -k of the pair.
Nothing here uses the CUDA library.
"""
import numpy as np
import pytest

import oracle
from tests import bruteforce as bf


def _states(rng, nm, npart):
    R = rng.standard_normal((nm, npart)) + 1j * rng.standard_normal((nm, npart))
    Lm = rng.standard_normal((npart, nm)) + 1j * rng.standard_normal((npart, nm))
    return R, Lm


def _fock_mixed(R, Lm):
    nm = R.shape[0]
    cs = [C.astype(np.complex128) for C in bf.fock_ops(nm)]
    cd = [C.T for C in cs]
    vac = np.zeros(1 << nm, np.complex128)
    vac[0] = 1.0

    def ket(V):
        v = vac.copy()
        for m in range(V.shape[1]):
            v = sum(V[a, m] * cd[a] for a in range(nm)) @ v
        return v

    psi_r = ket(R)
    bra = ket(Lm.conj().T).conj()
    norm = bra @ psi_r
    return cs, cd, (lambda O: complex(bra @ O @ psi_r / norm))


@pytest.mark.parametrize("npart,seed", [(3, 1), (4, 2), (5, 3)])
def test_pairing_observables_equal_fock_space(npart, seed):
    L = 2
    N = L * L
    m = oracle.SocModel(L, 1.0, 0.0, -4.0, 0.1, 2, hs="sz")
    rng = np.random.default_rng(seed)
    R, Lm = _states(rng, 2 * N, npart)
    G = np.eye(2 * N) - R @ np.linalg.solve(Lm @ R, Lm)
    got = m.pairing(G)
    cs, cd, ev = _fock_mixed(R, Lm)
    up = list(range(N))
    dn = [N + i for i in range(N)]
    # double occupancy
    D = sum(ev(cd[up[i]] @ cs[up[i]] @ cd[dn[i]] @ cs[dn[i]]) for i in range(N)) / N
    assert abs(got["D"] - D) < 1e-10
    # <Delta^2> = N^{-2} sum_ij <D+_i D_j + D_i D+_j> / 4
    Dp = [cd[up[i]] @ cd[dn[i]] for i in range(N)]
    Dm = [cs[dn[i]] @ cs[up[i]] for i in range(N)]
    P = sum(ev(Dp[i] @ Dm[j] + Dm[i] @ Dp[j]) for i in range(N) for j in range(N)) / 4 / N ** 2
    assert abs(got["Delta2"] - P) < 1e-10
    # momentum operators
    xs, ys = np.arange(N) % L, np.arange(N) // L

    def ck(k, spin):
        kx, ky = 2 * np.pi * (k % L) / L, 2 * np.pi * (k // L) / L
        ph = np.exp(-1j * (kx * xs + ky * ys)) / np.sqrt(N)
        base = 0 if spin == 0 else N
        return sum(ph[j] * cs[base + j] for j in range(N))

    def minus(k):
        return (L - k % L) % L + L * ((L - k // L) % L)

    c_up = [ck(k, 0) for k in range(N)]
    c_dn = [ck(k, 1) for k in range(N)]
    for k in range(N):
        assert abs(got["nk"][k] - ev(c_up[k].conj().T @ c_up[k])) < 1e-10
        assert abs(got["nk"][N + k] - ev(c_dn[k].conj().T @ c_dn[k])) < 1e-10
    for k in range(N):
        Dk = c_up[k].conj().T @ c_dn[minus(k)].conj().T
        for k2 in range(N):
            Dk2 = c_dn[minus(k2)] @ c_up[k2]
            assert abs(got["Mk"][k, k2] - ev(Dk @ Dk2)) < 1e-10, (k, k2)


def test_free_fermi_sea_values():
    """U = 0 on a closed shell (4 x 4, 5 per spin: the k = 0 level and its four neighbours): D = n_up
    n_dn = (5/16)^2, <n_k> is 1 on the shell and 0 off it, and the raw pairing matrix is diagonal,
    Mk[k][k] = <n_{k up}> <n_{-k dn}> (a Slater determinant has no off-diagonal pair coherence), so
    the condensate fraction of the free state is zero."""
    L, ns = 4, 5
    N = L * L
    m = oracle.SocModel(L, 1.0, 0.0, 0.0, 0.1, 2, hs="sz")
    k = 2 * np.pi * np.arange(L) / L
    kx, ky = np.meshgrid(k, k)
    eps = (-2 * (np.cos(kx) + np.cos(ky))).ravel()
    occ = np.argsort(eps, kind="stable")[:ns]
    assert eps[np.argsort(eps)[ns]] > eps[occ].max() + 1e-9  # a closed shell
    xs, ys = np.arange(N) % L, np.arange(N) // L
    # plane waves of the occupied momenta, spin up and spin down
    Pk = np.stack([np.exp(1j * (2 * np.pi * (q % L) / L * xs + 2 * np.pi * (q // L) / L * ys)) / np.sqrt(N)
                   for q in occ], axis=1)
    P = np.zeros((2 * N, 2 * ns), np.complex128)
    P[:N, :ns] = Pk
    P[N:, ns:] = Pk.conj()
    G = np.eye(2 * N) - P @ P.conj().T
    got = m.pairing(G)
    assert abs(got["D"] - (ns / N) ** 2) < 1e-12
    nk_up = np.zeros(N)
    nk_up[occ] = 1
    assert np.abs(got["nk"][:N] - nk_up).max() < 1e-12
    Mk = got["Mk"]
    assert np.abs(Mk - np.diag(np.diag(Mk))).max() < 1e-12
    minus = [(L - q % L) % L + L * ((L - q // L) % L) for q in range(N)]
    assert np.abs(np.diag(Mk) - got["nk"][:N] * got["nk"][N:][minus]).max() < 1e-12


def _sparse_fock_ops(nm):
    """Annihilation operators of nm modes as sparse matrices (Jordan-Wigner, occupation basis)."""
    import scipy.sparse as sp
    dim = 1 << nm
    st = np.arange(dim)
    ops = []
    for q in range(nm):
        have = (st >> q) & 1 == 1
        src = st[have]
        below = src & ((1 << q) - 1)
        sign = 1.0 - 2.0 * (np.array([bin(int(b)).count("1") for b in below]) & 1)
        ops.append(sp.csr_matrix((sign.astype(np.complex128), (src ^ (1 << q), src)), shape=(dim, dim)))
    return ops


def test_pairing_matrix_momentum_pairs_on_a_3x3_lattice():
    """On 3 x 3 the momenta k and -k differ (on 2 x 2 they coincide), so this fixes the -k of the pair
    D+_k = c+_{k up} c+_{-k dn} and the sign of the Fourier phase: Mk and nk against the sparse
    Fock-space expectation (18 spin orbitals, 4 particles)."""
    L, npart = 3, 4
    N = L * L
    m = oracle.SocModel(L, 1.0, 0.0, -4.0, 0.1, 2, hs="sz")
    rng = np.random.default_rng(9)
    R, Lm = _states(rng, 2 * N, npart)
    G = np.eye(2 * N) - R @ np.linalg.solve(Lm @ R, Lm)
    got = m.pairing(G)
    cs = _sparse_fock_ops(2 * N)
    cd = [C.T.tocsr() for C in cs]
    psi = np.zeros(1 << (2 * N), np.complex128)
    psi[0] = 1.0
    bra = psi.copy()
    for col in range(npart):
        psi = sum(R[a, col] * (cd[a] @ psi) for a in range(2 * N))
        bra = sum(np.conj(Lm[col, a]) * (cd[a] @ bra) for a in range(2 * N))
    bra = bra.conj()
    norm = bra @ psi
    xs, ys = np.arange(N) % L, np.arange(N) // L

    def ck(k, spin):
        ph = np.exp(-1j * (2 * np.pi * (k % L) / L * xs + 2 * np.pi * (k // L) / L * ys)) / np.sqrt(N)
        return sum(ph[j] * cs[spin * N + j] for j in range(N)).tocsr()

    def minus(k):
        return (L - k % L) % L + L * ((L - k // L) % L)

    c_up = [ck(k, 0) for k in range(N)]
    c_dn = [ck(k, 1) for k in range(N)]
    cdag_up = [c.conj().T.tocsr() for c in c_up]
    cdag_dn = [c.conj().T.tocsr() for c in c_dn]
    for k in range(N):
        assert abs(got["nk"][k] - bra @ (cdag_up[k] @ (c_up[k] @ psi)) / norm) < 1e-10
        assert abs(got["nk"][N + k] - bra @ (cdag_dn[k] @ (c_dn[k] @ psi)) / norm) < 1e-10
    assert any(minus(k) != k for k in range(N))
    for k2 in range(N):
        v = c_dn[minus(k2)] @ (c_up[k2] @ psi)  # D_k2 |psi>
        for k in range(N):
            ref = bra @ (cdag_up[k] @ (cdag_dn[minus(k)] @ v)) / norm
            assert abs(got["Mk"][k, k2] - ref) < 1e-10, (k, k2)
