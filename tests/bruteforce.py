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
