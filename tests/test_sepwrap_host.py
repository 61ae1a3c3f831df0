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
    h.sep_host_pass.argtypes = [i, i, i, i, i, vp, l, l, vp, vp, vp, vp, vp, l]
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
                                 (12, 4)])
@pytest.mark.parametrize("scaled", [False, True])
def test_pass_is_the_kronecker_product(lib, fp64, side, L, w, scaled):
    rng = np.random.default_rng(100 * L + 10 * w + side)
    N, batch = L * L, 2
    pad = 4 if L % 2 == 0 else 3  # ld % 4 == 0 takes the vector path of the row tiles
    dt = np.float64 if fp64 else np.float32
    A = chain_factor(L, 1.0, 0.05 * (1 + L % 3))
    G = rng.standard_normal((batch, N, N))
    sc = [rng.uniform(0.5, 2.0, (batch, N)) if scaled else None for _ in range(4)]  # rs_in, cs_in, rs_out, cs_out
    buf = _padded(G, pad, dt)
    scd = [None if s is None else np.ascontiguousarray(s, dt) for s in sc]
    lib.sep_host_pass(fp64, side, L, w, batch, _p(buf), N + pad, N * (N + pad), _p(A), *[_p(s) for s in scd], N)
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
@pytest.mark.parametrize("L,w", [(3, 16), (4, 16), (6, 16), (6, 4), (8, 16), (8, 8)])
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
