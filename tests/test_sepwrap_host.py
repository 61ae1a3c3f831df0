"""The separable wrap's tile code -- the CUDA kernel's own source (csrc/sepwrap.cuh) built for the
host and run serially -- against independent arithmetic: each pass against numpy's Kronecker
product (A (x) A) G and G (A (x) A), with A = exp(-tau K_1d) from scipy's expm of the periodic
chain, and the full forward / backward wrap, as the library issues it, against the oracle's dense
wrap G <- D E G E^{-1} D^{-1} (Eqs. BlMat, GrFMat).  Ragged tiles, padding and both precisions."""
import ctypes
import os
import subprocess

import numpy as np
import pytest
import scipy.linalg

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = tmp_path_factory.mktemp("sephost") / "libsephost.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", str(out),
                           os.path.join(ROOT, "tests", "sepwrap_host.cpp")])
    h = ctypes.CDLL(str(out))
    vp, i, l = ctypes.c_void_p, ctypes.c_int, ctypes.c_long
    h.sep_host_pass.argtypes = [i, i, i, i, i, i, vp, l, l, vp, vp, vp, vp, vp, l, i]
    h.sep_host_wrap.argtypes = [i, i, i, i, i, vp, l, l, vp, vp, vp, vp, l]
    yield h
    assert h.sep_host_misaligned() == 0  # no vector access that would fault on the device


def chain_factor(L, t, tau):
    """exp(-tau K_1d) of the periodic chain, K_1d[x][x +- 1] = -t (bonds onto the same pair add up)."""
    K = np.zeros((L, L))
    for x in range(L):
        K[x, (x + 1) % L] -= t
        K[x, (x - 1) % L] -= t
    return scipy.linalg.expm(-tau * K)


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _padded(G, pad, dt):
    """G in a NaN-padded buffer of leading dimension N + pad, starting on a 64-byte boundary (as
    cudaMalloc'd memory does)."""
    batch, N, _ = G.shape
    n = batch * N * (N + pad)
    raw = np.full(n + 64, np.nan, dt)
    off = (-raw.ctypes.data % 64) // raw.itemsize
    buf = raw[off:off + n].reshape(batch, N, N + pad)
    buf[:, :, :N] = G
    return buf


@pytest.mark.parametrize("fp64", [1, 0])
@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("L,w", [(2, 16), (3, 4), (4, 16), (5, 16), (5, 4), (6, 5), (8, 16), (8, 8), (12, 16),
                                 (12, 4), (2, 0), (3, 0), (4, 0), (5, 0), (6, 0), (8, 0), (9, 0), (12, 0),
                                 (13, 0), (16, 0), (20, 0), (24, 0), (32, 0), (40, 0)])
@pytest.mark.parametrize("scaled", [False, True])
@pytest.mark.parametrize("circ", [1, 0])
def test_pass_is_the_kronecker_product(lib, fp64, side, L, w, scaled, circ):
    """circ = 1: A is the periodic chain's factor, passed as circulant (the line passes keep its
    first row); circ = 0: a symmetric A that is not circulant, through the general passes."""
    rng = np.random.default_rng(100 * L + 10 * w + side)
    N, batch = L * L, 2
    pad = 4 if L % 2 == 0 else 3  # ld % 4 == 0 takes the vector path of the row tiles
    dt = np.float64 if fp64 else np.float32
    if circ:
        A = chain_factor(L, 1.0, 0.05 * (1 + L % 3))
    else:
        S = rng.standard_normal((L, L))
        A = np.eye(L) + 0.1 * (S + S.T)
    G = rng.standard_normal((batch, N, N))
    sc = [rng.uniform(0.5, 2.0, (batch, N)) if scaled else None for _ in range(4)]  # rs_in, cs_in, rs_out, cs_out
    buf = _padded(G, pad, dt)
    scd = [None if s is None else np.ascontiguousarray(s, dt) for s in sc]
    lib.sep_host_pass(fp64, side, L, 0, w, batch, _p(buf), N + pad, N * (N + pad), _p(A), *[_p(s) for s in scd], N,
                      circ)
    E = np.kron(A, A)  # site i = x + L y
    for z in range(batch):
        one = np.ones(N)
        ri, ci, ro, co = [one if s is None else s[z] for s in sc]
        Gin = ri[:, None] * G[z] * ci[None, :]
        ref = ro[:, None] * ((E @ Gin) if side == 0 else (Gin @ E)) * co[None, :]
        got = buf[z, :, :N].astype(np.float64)
        tol = 1e-13 if fp64 else 2e-6
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
        assert np.isnan(buf[z, :, N:]).all()  # padding untouched


@pytest.mark.parametrize("fp64", [1, 0])
@pytest.mark.parametrize("direction", [+1, -1])
@pytest.mark.parametrize("L,w", [(3, 16), (4, 16), (6, 16), (6, 4), (8, 16), (8, 8), (3, 0), (4, 0), (5, 0),
                                 (6, 0), (8, 0), (12, 0), (16, 0), (20, 0)])
def test_wrap_matches_the_oracle(lib, fp64, direction, L, w):
    rng = np.random.default_rng(7 * L + w + (direction > 0))
    N, t, U, dtau = L * L, 1.0, 4.0, 0.05
    pad = (-N) % 32  # the library's leading dimension: N rounded up to 32
    dt = np.float64 if fp64 else np.float32
    m = oracle.Model(L, L, t, U, dtau, 4)
    xl = np.where(rng.random(N) < 0.5, 1, -1).astype(np.int8)
    G = rng.standard_normal((2, N, N)) * 0.3 + np.eye(N)
    Ex, Exi = chain_factor(L, t, dtau), chain_factor(L, t, -dtau)
    d = np.stack([np.exp(m.c[s] * xl) for s in range(2)]).astype(dt)
    dinv = np.stack([np.exp(-m.c[s] * xl) for s in range(2)]).astype(dt)
    buf = _padded(G, pad, dt)
    lib.sep_host_wrap(fp64, direction, L, w, 2, _p(buf), N + pad, N * (N + pad), _p(Ex), _p(Exi), _p(d), _p(dinv), N)
    for s in range(2):
        ref = m.wrap(G[s], xl, s, direction)
        got = buf[s, :, :N].astype(np.float64)
        tol = 1e-12 if fp64 else 1e-5
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref), (s, np.linalg.norm(got - ref) / np.linalg.norm(ref))
        assert np.isnan(buf[s, :, N:]).all()


@pytest.mark.parametrize("fp64", [1, 0])
@pytest.mark.parametrize("L,C,w", [(4, 7, 16), (6, 13, 16), (8, 28, 16), (8, 3, 4), (5, 11, 5), (4, 7, 0),
                                   (6, 13, 0), (8, 28, 0), (8, 3, 0), (5, 11, 0), (12, 9, 0)])
def test_factor_passes_move_the_t_form_factors(lib, fp64, L, C, w):
    """The T form's factor wrap (forward slice l): U_R <- D E U_R (N x N_sigma, side 0 with the
    rows scaled by d after) and U_L <- U_L E^{-1} D^{-1} (N_sigma x N, side 1 with the columns
    scaled by dinv after); U_L U_R is unchanged (Sec. II.C)."""
    rng = np.random.default_rng(L * 100 + C)
    N = L * L
    dt = np.float64 if fp64 else np.float32
    dtau, c = 0.1, 0.4
    Ex, Exi = chain_factor(L, 1.0, dtau), chain_factor(L, 1.0, -dtau)
    x = np.where(rng.random(N) < 0.5, 1, -1)
    d, dinv = np.exp(c * x), np.exp(-c * x)
    UR = rng.standard_normal((N, C))
    UL = rng.standard_normal((C, N))
    E, Einv = np.kron(Ex, Ex), np.kron(Exi, Exi)
    ldr, ldl = C + 4, N + 4  # 16-byte multiples of the row pitch for the vector path
    bR = np.full((1, N, ldr), np.nan, dt)
    bR[0, :, :C] = UR
    bL = np.full((1, C, ldl), np.nan, dt)
    bL[0, :, :N] = UL
    dd, di = d.astype(dt), dinv.astype(dt)
    lib.sep_host_pass(fp64, 0, L, C, w, 1, _p(bR), ldr, N * ldr, _p(Ex), None, None, _p(dd), None, N, 1)
    lib.sep_host_pass(fp64, 1, L, C, w, 1, _p(bL), ldl, C * ldl, _p(Exi), None, None, None, _p(di), N, 1)
    refR = d[:, None] * (E @ UR)
    refL = (UL @ Einv) * dinv[None, :]
    tol = 1e-12 if fp64 else 1e-5
    gotR, gotL = bR[0, :, :C].astype(np.float64), bL[0, :, :N].astype(np.float64)
    assert np.linalg.norm(gotR - refR) <= tol * np.linalg.norm(refR)
    assert np.linalg.norm(gotL - refL) <= tol * np.linalg.norm(refL)
    assert np.isnan(bR[0, :, C:]).all() and np.isnan(bL[0, :, N:]).all()
    O0, O1 = UL @ UR, gotL @ gotR  # the overlap the T form keeps fixed across the wrap
    assert np.linalg.norm(O1 - O0) <= 10 * tol * np.linalg.norm(O0) * np.sqrt(N)
