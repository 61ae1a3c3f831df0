"""GPU parity of the spin-orbit-coupled sweep (Appendix A) through the C ABI against the FP64 oracle.

Both sides get the same seeded inputs: the time-reversal-invariant trial state, the initial fields,
and the Philox uniforms of every slice visit.  FP64 runs free: decisions must be identical and G
must agree to 1e-10 (relative Frobenius norm) after every slice; ratios and block force-bias
proposal probabilities are compared too.  FP32 runs replay decisions drawn by the test from its own
seeded generator (the same for both sides) and G must stay within 1e-5.
"""
import numpy as np
import pytest

import oracle
from paper_2506_09611_gb300 import inputs

pytestmark = pytest.mark.gpu

soc = pytest.importorskip("paper_2506_09611_gb300.soc")

FP64_TOL = 1e-10
FP32_TOL = 1e-5


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def make(L, n_e, M, stab, precision="fp64", gemm="tc3", U=-4.0, dtau=0.05, lam=0.5, seed=21):
    P = inputs.soc_trial_state(L, n_e, lam=lam)
    X = inputs.initial_fields(M, L * L, seed=seed)
    ctx = soc.SocContext(L, M, n_e, 1, precision, gemm, stab, 1.0, lam, U, dtau, seed)
    ctx.init(P, X)
    model = oracle.SocModel(L, 1.0, lam, U, dtau, M)
    w = oracle.SocWalker(model, P, X)
    return ctx, w


def order(M):
    return [(ell, +1) for ell in range(1, M + 1)] + [(ell, -1) for ell in range(M, 0, -1)]


@pytest.mark.parametrize("L,n_e,M,stab", [(3, 8, 8, 4), (4, 14, 6, 3), (6, 36, 8, 4)])
def test_init_G0_and_energy_match_oracle(L, n_e, M, stab):
    ctx, w = make(L, n_e, M, stab)
    with ctx:
        assert rel(ctx.G(0), w.G) < FP64_TOL
        e = ctx.measure_energy()[0]
        eo = w.m.energy(w.G)
        assert abs(e - eo) < 1e-9 * max(1.0, abs(eo))


def _free_run(ctx, w, mode, k, nb, seed, steps, stab, tol):
    M, N = w.m.M, w.m.N
    for visit, (ell, d) in enumerate(order(M)[:steps]):
        u = inputs.uniforms(seed, 0, visit, 2 * N)
        dec_o, ratio_o, extra = w.sweep_slice(ell, d, mode, u, k=k, nb=nb)
        ctx.sweep_slice(ell, d, mode, k=k, nb=nb)
        dec_g, rat_g = ctx.decisions(0), ctx.ratios(0)
        if mode == "blockfb":
            nbk = (N + nb - 1) // nb
            np.testing.assert_array_equal(dec_g[:N], (extra["xprop"] > 0).astype(np.uint8))
            np.testing.assert_array_equal(dec_g[N:N + nbk], dec_o, err_msg=f"blocks, slice {ell} dir {d}")
            np.testing.assert_allclose(ctx.lam_plus(0), extra["lam_plus"], rtol=1e-9, atol=1e-12)
            np.testing.assert_allclose(rat_g[N:N + nbk], ratio_o, rtol=1e-8, atol=1e-12)
        else:
            np.testing.assert_array_equal(dec_g[:N], dec_o, err_msg=f"decisions, slice {ell} dir {d}")
            np.testing.assert_allclose(rat_g[:N], ratio_o, rtol=1e-8, atol=1e-12)
        np.testing.assert_array_equal(ctx.fields(0), w.x)
        r = rel(ctx.G(0), w.G)
        assert r < tol, f"{mode} slice {ell} dir {d}: rel err {r}"
        if w.pos % stab == 0:
            drift = ctx.recompute_G()[0]
            w.recompute()
            assert drift < tol
            r = rel(ctx.G(0), w.G)
            assert r < tol, f"after recompute at {w.pos}: {r}"


@pytest.mark.parametrize("mode,k,nb", [("local", 1, 1), ("delayed", 5, 1), ("delayed", 32, 1),
                                       ("blockfb", 1, 1), ("blockfb", 1, 4), ("blockfb", 1, 7), ("blockfb", 1, 16)])
def test_fp64_free_run_matches_oracle(mode, k, nb):
    """nb = 16 = N: the full force-bias update, one block per slice."""
    L, n_e, M, stab = 4, 14, 4, 2
    ctx, w = make(L, n_e, M, stab, seed=5)
    with ctx:
        _free_run(ctx, w, mode, k, nb, 5, 2 * M, stab, FP64_TOL)


def test_fp64_ragged_lattice_all_modes():
    """3 x 3 lattice: 2N = 18 orbitals (a padded row), windows and blocks with a ragged tail."""
    for mode, k, nb in (("delayed", 4, 1), ("blockfb", 1, 4)):
        ctx, w = make(3, 8, 4, 2, seed=9)
        with ctx:
            _free_run(ctx, w, mode, k, nb, 9, 8, 2, FP64_TOL)


def test_fp64_larger_lattice_spans_tiles():
    """8 x 8 lattice (2N = 128): GEMM tiles of 64 and several windows of 32 sites."""
    ctx, w = make(8, 64, 4, 2, seed=3)
    with ctx:
        _free_run(ctx, w, "delayed", 32, 1, 3, 3, 2, FP64_TOL)


def _replay(rng, N, mode, nb):
    rep = np.zeros(2 * N, np.uint8)
    rep[:N] = rng.random(N) < 0.5
    if mode == "blockfb":
        rep[N:N + (N + nb - 1) // nb] = rng.random((N + nb - 1) // nb) < 0.7
    return rep


@pytest.mark.parametrize("gemm", ["tc3", "simt"])
@pytest.mark.parametrize("mode,k,nb", [("delayed", 16, 1), ("blockfb", 1, 8), ("local", 1, 1)])
def test_fp32_replay_within_tolerance(gemm, mode, k, nb):
    L, n_e, M, stab = 6, 36, 6, 3
    ctx, w = make(L, n_e, M, stab, precision="fp32", gemm=gemm, seed=13)
    rng = np.random.default_rng(1234)
    N = L * L
    with ctx:
        for visit, (ell, d) in enumerate(order(M)[:5]):
            rep = _replay(rng, N, mode, nb)
            u = inputs.uniforms(13, 0, visit, 2 * N)
            w.sweep_slice(ell, d, mode, u, k=k, nb=nb, replay=rep)
            ctx.sweep_slice(ell, d, mode, k=k, nb=nb, replay=rep)
            np.testing.assert_array_equal(ctx.fields(0), w.x)
            r = rel(ctx.G(0), w.G)
            assert r < FP32_TOL, f"{gemm} {mode} slice {ell}: {r}"
            if w.pos % stab == 0:
                ctx.recompute_G()
                w.recompute()
                assert rel(ctx.G(0), w.G) < 1e-7  # the FP64 recompute stored in FP32


def test_backward_half_sweep_and_recompute_fp64():
    """Forward to M and back: wraps in both directions, the left-stack recompute path."""
    L, n_e, M, stab = 4, 14, 4, 2
    ctx, w = make(L, n_e, M, stab, seed=17)
    with ctx:
        _free_run(ctx, w, "delayed", 8, 1, 17, 2 * M, stab, FP64_TOL)
        assert ctx.info()["slice"] == 0


def test_state_errors():
    ctx, w = make(3, 8, 4, 2)
    with ctx:
        with pytest.raises(soc.afqmc.AfqmcError):
            ctx.sweep_slice(2, +1, "delayed", k=4)  # not at slice 1
        with pytest.raises(soc.afqmc.AfqmcError):
            ctx.sweep_slice(1, +1, "delayed", k=999)  # window too large
        ctx.sweep_slice(1, +1, "delayed", k=4)
        ctx.sweep_slice(2, +1, "delayed", k=4)
        with pytest.raises(soc.afqmc.AfqmcError):
            ctx.sweep_slice(3, +1, "delayed", k=4)  # recompute due at slice 2
        ctx.recompute_G()
        ctx.sweep_slice(3, +1, "delayed", k=4)


@pytest.mark.parametrize("mode,k,nb", [("blockfb", 1, 16), ("blockfb", 1, 64), ("delayed", 64, 1)])
def test_fp32_full_size_24x24_one_slice(mode, k, nb):
    """The 24 x 24 lattice (2N = 1152 complex orbitals, half filling) at the bench's launch
    configurations: one replayed slice against the oracle, G within 1e-5.  nb = 64 is the block
    size whose window (a 128 x 128 complex block, inverted by Gauss-Jordan with 2 x 2 pivots) runs
    without the pipelined flush."""
    L, n_e, M, stab = 24, 576, 2, 2
    ctx, w = make(L, n_e, M, stab, precision="fp32", gemm="tc3", seed=29)
    N = L * L
    rng = np.random.default_rng(77)
    with ctx:
        rep = _replay(rng, N, mode, nb)
        u = inputs.uniforms(29, 0, 0, 2 * N)
        _, _, extra = w.sweep_slice(1, +1, mode, u, k=k, nb=nb, replay=rep)
        ctx.sweep_slice(1, +1, mode, k=k, nb=nb, replay=rep)
        np.testing.assert_array_equal(ctx.fields(0), w.x)
        assert rel(ctx.G(0), w.G) < FP32_TOL
        if mode == "blockfb":  # proposal probabilities from the FP32 block
            np.testing.assert_allclose(ctx.lam_plus(0), extra["lam_plus"], atol=1e-4)


def test_two_walkers_with_device_drawn_fields_fp64():
    """Two walkers in one context, fields drawn on the device (read back and given to the oracle):
    each walker's G(0) and its free-running slices match its own oracle chain."""
    L, n_e, M, stab, seed = 4, 14, 4, 2, 31
    P = inputs.soc_trial_state(L, n_e)
    ctx = soc.SocContext(L, M, n_e, 2, "fp64", "tc3", stab, 1.0, 0.5, -4.0, 0.05, seed)
    with ctx:
        ctx.init(P, None)
        model = oracle.SocModel(L, 1.0, 0.5, -4.0, 0.05, M)
        ws = []
        for j in range(2):
            X = ctx.fields(j)
            assert set(np.unique(X)) <= {-1, 1}
            w = oracle.SocWalker(model, P, X)
            assert rel(ctx.G(j), w.G) < FP64_TOL
            ws.append(w)
        assert not np.array_equal(ctx.fields(0), ctx.fields(1))
        N = L * L
        for visit, (ell, d) in enumerate(order(M)[:4]):
            ctx.sweep_slice(ell, d, "blockfb", nb=4)
            for j, w in enumerate(ws):
                u = inputs.uniforms(seed, j, visit, 2 * N)
                w.sweep_slice(ell, d, "blockfb", u, nb=4)
                np.testing.assert_array_equal(ctx.fields(j), w.x)
                assert rel(ctx.G(j), w.G) < FP64_TOL
            if ws[0].pos % stab == 0:
                ctx.recompute_G()
                for j, w in enumerate(ws):
                    w.recompute()
                    assert rel(ctx.G(j), w.G) < FP64_TOL
