"""FP64 products of the recompute on the tensor cores (digit splitting) against exact references.

The split turns every FP64 element into small integer digits; the tensor cores must then multiply
and accumulate digit planes without any rounding.  Integer inputs whose product is exactly
representable must come back bit for bit; random inputs with a wide dynamic range must agree
with an exact rational evaluation (sampled elements) and with an FP64 product to within a few
FP64 roundings, not the ~1e-8 an inexact FP32 accumulation would leave.  The recompute itself
must give the same G with either engine, and the oracle's G(0).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2506_09611_gb300 import inputs

pytestmark = pytest.mark.gpu

afqmc = pytest.importorskip("paper_2506_09611_gb300.afqmc")
torch = pytest.importorskip("torch")

# (M, N, K): K below and above the exact range of 7-bit digits (K (2^7 - 1)^2 < 2^24 up to K = 1040),
# of 6-bit digits (up to K = 4227), ragged M / N against the 128 x BN tiles, K not a multiple of 4
SHAPES = [(128, 128, 32), (300, 170, 700), (200, 136, 1024), (100, 260, 1600), (257, 129, 2304), (33, 70, 13),
          (1600, 1600, 700)]


def _dgemm(kind, A, B, pad=3):
    M, K = A.shape
    N = B.shape[1]
    Ad = torch.zeros((M, K + pad), dtype=torch.float64)
    Ad[:, :K] = torch.from_numpy(A)
    Bd = torch.zeros((K, N + pad), dtype=torch.float64)
    Bd[:, :N] = torch.from_numpy(B)
    Ad, Bd = Ad.cuda(), Bd.cuda()
    C = torch.full((M, N + pad), float("nan"), dtype=torch.float64, device="cuda")
    afqmc.afqmc_debug_dgemm(kind, M, N, K, Ad.data_ptr(), K + pad, Bd.data_ptr(), N + pad, C.data_ptr(), N + pad,
                            torch.cuda.current_stream())
    assert torch.isnan(C[:, N:]).all()  # padding untouched
    return C[:, :N].cpu().numpy()


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_integer_inputs_are_exact(M, N, K):
    rng = np.random.default_rng(M * 7 + N * 13 + K)
    lim = 2 ** 20 if K <= 2048 else 2 ** 19
    A = rng.integers(-lim, lim, (M, K))
    B = rng.integers(-lim, lim, (K, N))
    exact = A @ B  # int64: |C| <= K lim^2 < 2^53, so exactly representable in FP64
    got = _dgemm(1, A.astype(np.float64), B.astype(np.float64))
    np.testing.assert_array_equal(got, exact.astype(np.float64))


def _wide(rng, M, K, N):
    A = rng.standard_normal((M, K)) * np.exp2(rng.integers(-30, 31, (M, 1)))
    B = rng.standard_normal((K, N)) * np.exp2(rng.integers(-30, 31, (1, N)))
    A[rng.random((M, K)) < 0.05] = 0.0  # exact zeros, and one all-zero row / column
    A[M // 2, :] = 0.0
    B[:, N // 3] = 0.0
    return A, B


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_wide_range_matches_exact_products(M, N, K):
    rng = np.random.default_rng(1000 + M + N + K)
    A, B = _wide(rng, M, K, N)
    got = _dgemm(1, A, B)
    simt = _dgemm(0, A, B)
    absAB = np.abs(A) @ np.abs(B)
    # every element against the FP64 SIMT product: both within a few roundings of sum |a||b|
    assert np.all(np.abs(got - simt) <= 2.0 ** -46 * absAB + 1e-300)
    # sampled elements against the exact rational value
    idx = rng.integers(0, M, 24), rng.integers(0, N, 24)
    for i, j in zip(*idx):
        ex = sum((Fraction(float(A[i, k])) * Fraction(float(B[k, j])) for k in range(K)), Fraction(0))
        bound = 2.0 ** -48 * K * np.abs(A[i]).max() * np.abs(B[:, j]).max()
        assert abs(Fraction(float(got[i, j])) - ex) <= Fraction(bound), (i, j)


def test_nonfinite_input_is_reported():
    A = np.ones((64, 40))
    B = np.ones((40, 64))
    A[3, 7] = np.inf
    with pytest.raises(afqmc.AfqmcError) as e:
        _dgemm(1, A, B)
    assert e.value.code == -4  # AFQMC_ERR_NUMERIC


def test_recompute_engines_agree_24x24():
    """FP64 bulk at 24 x 24 (N = 576, 252 per spin): the digit-split products (default engine) and
    the FP64 SIMT products give the same G(0) and the same recomputed G, both the oracle's."""
    L, ns, M, stab = 24, 252, 4, 2
    N = L * L
    P = inputs.trial_state(L, L, ns)
    X = inputs.initial_fields(M, N, seed=4)
    model = oracle.Model(L, L, 1.0, 4.0, 0.05, M)
    w = oracle.Walker(model, P, P, X)
    ctxs = [afqmc.Context(M, U=4.0, precision="fp64", stab_every=stab, seed=4, gemm=g) for g in ("tc3", "simt")]
    try:
        for c in ctxs:
            c.init_walkers([L], [ns], [ns], np.concatenate([P.ravel(), P.ravel()]), X)
        for s in range(2):
            g0 = [c.G(0, s) for c in ctxs]
            # the engines round differently (4e-13 here: G = 1 - U_R Z cancels), far below the
            # ~1e-7 an inexact FP32 accumulation would leave
            assert np.linalg.norm(g0[0] - g0[1]) / np.linalg.norm(g0[1]) < 1e-11
            assert np.linalg.norm(g0[0] - w.G[s]) / np.linalg.norm(w.G[s]) < 1e-10
        for ell in (1, 2):  # the oracle's decisions, replayed by both engines
            u = inputs.uniforms(4, 0, ell - 1, 2 * N)
            dec, _, _ = w.sweep_slice(ell, +1, "delayed", u, k=32)
            rep = np.zeros(2 * N, np.uint8)
            rep[:N] = dec
            for c in ctxs:
                c.sweep_slice(ell, +1, "delayed", k=32, replay=rep)
        w.recompute(stab)
        for c in ctxs:
            c.recompute_G()
        for s in range(2):
            g = [c.G(0, s) for c in ctxs]
            assert np.linalg.norm(g[0] - g[1]) / np.linalg.norm(g[1]) < 1e-11
            assert np.linalg.norm(g[0] - w.G[s]) / np.linalg.norm(w.G[s]) < 1e-10
    finally:
        for c in ctxs:
            c.close()
