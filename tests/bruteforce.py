"""Independent numpy brute force for pinning the oracle (tests only).

Nothing here calls the oracle or the CUDA library.  Everything is the plain
definition from the paper, evaluated with numpy / scipy library routines:
  B_l^s = exp(H_I^s(x_l)) exp(-dtau K)          (Eq. BlMat; expm from scipy)
  W(X) = prod_s det(P_s^T B_M ... B_1 P_s)       (Eq. ConfgWeight)
  G(l) = 1 - R (L R)^{-1} L                       (Eq. GrFMat, no stabilisation)
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def expK(K, tau):
    return scipy.linalg.expm(-tau * K)


def B_mat(E, c_s, xl):
    return np.diag(np.exp(c_s * xl.astype(np.float64))) @ E


def products(E, c_s, X, P, ell):
    """R = B_ell..B_1 P and L = P^T B_M .. B_{ell+1} (plain products)."""
    M = X.shape[0]
    R = P.copy()
    for j in range(1, ell + 1):
        R = B_mat(E, c_s, X[j - 1]) @ R
    L = P.T.copy()
    for j in range(M, ell, -1):
        L = L @ B_mat(E, c_s, X[j - 1])
    return R, L


def green(E, c_s, X, P, ell):
    R, L = products(E, c_s, X, P, ell)
    return np.eye(E.shape[0]) - R @ np.linalg.solve(L @ R, L)


def overlap(E, c_s, X, P):
    R, L = products(E, c_s, X, P, 0)
    return np.linalg.det(L @ R)


def weight(E, c, X, Pu, Pd, log_scalar=None):
    """W(X) = P(X) prod_s det(...) with P(X) = prod_i s(x_i) (constant factors dropped)."""
    w = overlap(E, c[0], X, Pu) * overlap(E, c[1], X, Pd)
    if log_scalar is not None:
        w *= np.exp(sum(log_scalar(int(v)) for v in X.ravel()))
    return w


def fock_energy(K, U, Ru, Lu, Rd, Ld):
    """<psi_l| H |psi_r> / <psi_l|psi_r> on the full Fock space (Jordan-Wigner), with
    H = sum_{ij s} K_ij c+_is c_js + U sum_i (n_iu n_id - (n_iu + n_id)/2) and the Slater
    determinants |psi_r> = prod_m (c+ R)_m |0>, <psi_l| = <0| prod_m (L c)_m (reversed)."""
    N = K.shape[0]
    nm = 2 * N  # modes: (site, spin) -> i + N*s
    dim = 1 << nm
    # annihilation operators in the occupation basis, JW ordering by mode index
    cs = []
    for q in range(nm):
        C = np.zeros((dim, dim))
        for st in range(dim):
            if st >> q & 1:
                sign = (-1) ** bin(st & ((1 << q) - 1)).count("1")
                C[st ^ (1 << q), st] = sign
        cs.append(C)
    cd = [C.T for C in cs]
    vac = np.zeros(dim)
    vac[0] = 1.0

    def ket(Rs):
        v = vac.copy()
        for s, R in enumerate(Rs):
            for m in range(R.shape[1]):
                op = sum(R[i, m] * cd[i + N * s] for i in range(N))
                v = op @ v
        return v

    psi_r = ket([Ru, Rd])
    psi_l = ket([Lu.T, Ld.T])  # <psi_l| = (ket of the rows of L)^T for real L
    H = np.zeros((dim, dim))
    for s in range(2):
        for i in range(N):
            for j in range(N):
                if K[i, j] != 0.0:
                    H += K[i, j] * cd[i + N * s] @ cs[j + N * s]
    for i in range(N):
        nu = cd[i] @ cs[i]
        nd = cd[i + N] @ cs[i + N]
        H += U * (nu @ nd - 0.5 * (nu + nd))
    return float(psi_l @ H @ psi_r) / float(psi_l @ psi_r)


# ---------------- spin-orbit-coupled model (Appendix A) ----------------

def soc_HI(gamma, xl, hs="sy"):
    """Exponent matrix of B_I(x_l) on the 2N orbitals.
    hs = "sy" (Eq. BIOpForSy): gamma x_i (c+_{i,up} c_{i,dn} - c+_{i,dn} c_{i,up}) has entries
    +gamma x_i at (up i, dn i) and -gamma x_i at (dn i, up i);
    hs = "sz" (Eq. BIOpForHubbard): i gamma x_i (n_{i,up} - n_{i,dn}) has +i gamma x_i at
    (up i, up i) and -i gamma x_i at (dn i, dn i)."""
    N = xl.shape[0]
    H = np.zeros((2 * N, 2 * N), np.complex128 if hs == "sz" else np.float64)
    for i in range(N):
        if hs == "sz":
            H[i, i] = 1j * gamma * xl[i]
            H[N + i, N + i] = -1j * gamma * xl[i]
        else:
            H[i, N + i] = gamma * xl[i]
            H[N + i, i] = -gamma * xl[i]
    return H


def soc_B(E, gamma, xl, hs="sy"):
    return scipy.linalg.expm(soc_HI(gamma, xl.astype(np.float64), hs)) @ E


def soc_products(E, gamma, X, P, ell, hs="sy"):
    M = X.shape[0]
    R = P.copy()
    for j in range(1, ell + 1):
        R = soc_B(E, gamma, X[j - 1], hs) @ R
    L = P.conj().T.copy()
    for j in range(M, ell, -1):
        L = L @ soc_B(E, gamma, X[j - 1], hs)
    return R, L


def soc_green(E, gamma, X, P, ell, hs="sy"):
    R, L = soc_products(E, gamma, X, P, ell, hs)
    return np.eye(E.shape[0]) - R @ np.linalg.solve(L @ R, L)


def soc_overlap(E, gamma, X, P, hs="sy"):
    """det(P^+ B_M ... B_1 P): the configuration weight up to the uniform prior."""
    R, L = soc_products(E, gamma, X, P, 0, hs)
    return np.linalg.det(L @ R)


def fock_ops(nm):
    """Annihilation operators of nm fermion modes in the occupation basis (Jordan-Wigner)."""
    dim = 1 << nm
    cs = []
    for q in range(nm):
        C = np.zeros((dim, dim))
        for st in range(dim):
            if st >> q & 1:
                C[st ^ (1 << q), st] = (-1) ** bin(st & ((1 << q) - 1)).count("1")
        cs.append(C)
    return cs


def soc_fock_energy(H0, U, R, L):
    """<psi_l| H |psi_r> / <psi_l|psi_r> on the Fock space of the 2N orbitals, with
    H = c+ H0 c + U sum_i (n_iu n_id - (n_iu + n_id)/2), |psi_r> = prod_m (c+ R)_m |0> and
    <psi_l| the bra whose orbitals are the rows of L."""
    nm = H0.shape[0]
    N = nm // 2
    cs = fock_ops(nm)
    cd = [C.T for C in cs]
    vac = np.zeros(1 << nm, np.complex128)
    vac[0] = 1.0

    def ket(V):
        v = vac.copy()
        for m in range(V.shape[1]):
            v = sum(V[a, m] * cd[a] for a in range(nm)) @ v
        return v

    psi_r = ket(R)
    bra = ket(L.conj().T).conj()
    H = np.zeros((1 << nm, 1 << nm), np.complex128)
    for a in range(nm):
        for b in range(nm):
            if H0[a, b] != 0:
                H += H0[a, b] * cd[a] @ cs[b]
    for i in range(N):
        nu = cd[i] @ cs[i]
        nd = cd[N + i] @ cs[N + i]
        H += U * (nu @ nd - 0.5 * (nu + nd))
    return complex(bra @ H @ psi_r / (bra @ psi_r))
