"""GPU parity at the code paths the 40 x 40 bench takes, against the FP64 oracle.

The cases of test_gpu_parity.py fit a slice into one window (block force bias) or give every
CTA of the local update a single row.  The bench runs neither: at N = 1600 a block force-bias
slice spans 13 windows (the next window's block comes from the pipelined flush), and each CTA of
the local update owns 10-11 rows.  These tests run those paths:

* block force bias over several windows per slice, FP64 free-running (decisions identical, G
  within 1e-10 after every slice, recomputes included), and FP32 replay at 40 x 40 (G within
  1e-5 after each slice);
* the local update with more rows than CTAs, FP64 free-running at 16 x 16 and 40 x 40, and FP32
  replay at 40 x 40;
* FP32 replay of a mixed-size walker population in one context.
"""
import numpy as np
import pytest

import oracle
from paper_2506_09611_gb300 import inputs

pytestmark = pytest.mark.gpu

afqmc = pytest.importorskip("paper_2506_09611_gb300.afqmc")

FP64_TOL = 1e-10
FP32_TOL = 1e-5


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _replay_bytes(N, mode, nb, dec, extra):
    rep = np.zeros(2 * N, np.uint8)
    if mode == "blockfb":
        nblocks = (N + nb - 1) // nb
        rep[:N] = (extra["xprop"] > 0)
        rep[N:N + nblocks] = dec
    else:
        rep[:N] = dec
    return rep


def _free_run(L, ns, M, stab, U, mode, k, nb, seed, steps=None):
    """FP64 free run of the walker through `steps` slice-steps of a forward + backward sweep."""
    N = L * L
    P = inputs.trial_state(L, L, ns)
    X = inputs.initial_fields(M, N, seed=seed)
    model = oracle.Model(L, L, 1.0, U, 0.05, M)
    w = oracle.Walker(model, P, P, X)
    order = [(ell, +1) for ell in range(1, M + 1)] + [(ell, -1) for ell in range(M, 0, -1)]
    if steps is not None:
        order = order[:steps]
    with afqmc.Context(M, U=U, precision="fp64", stab_every=stab, seed=seed) as ctx:
        ctx.init_walkers([L], [ns], [ns], np.concatenate([P.ravel(), P.ravel()]), X)
        for s in range(2):
            assert rel(ctx.G(0, s), w.G[s]) < FP64_TOL
        for visit, (ell, d) in enumerate(order):
            u = inputs.uniforms(seed, 0, visit, 2 * N)
            dec_o, _, extra = w.sweep_slice(ell, d, mode, u, k=k, nb=nb)
            st = ctx.sweep_slice(ell, d, mode, k=k, nb=nb, want_stats=True)
            dec_g = ctx.decisions(0)
            if mode == "blockfb":
                nblocks = (N + nb - 1) // nb
                np.testing.assert_array_equal(dec_g[:N], (extra["xprop"] > 0).astype(np.uint8),
                                              err_msg=f"proposals slice {ell} dir {d}")
                np.testing.assert_array_equal(dec_g[N:N + nblocks], dec_o, err_msg=f"blocks slice {ell} dir {d}")
                assert st[0].proposals == nblocks
            else:
                np.testing.assert_array_equal(dec_g[:N], dec_o, err_msg=f"decisions slice {ell} dir {d}")
                assert st[0].proposals == N and st[0].accepts == int(dec_o.sum())
            for s in range(2):
                r = rel(ctx.G(0, s), w.G[s])
                assert r < FP64_TOL, f"slice {ell} dir {d} spin {s}: rel err {r}"
            assert st[0].sign == w.sign
            if w.pos % stab == 0:
                ctx.recompute_G()
                w.recompute(stab)
                for s in range(2):
                    assert rel(ctx.G(0, s), w.G[s]) < FP64_TOL
        np.testing.assert_array_equal(ctx.fields(0), w.x)


@pytest.mark.parametrize("L,ns,nb", [(12, 63, 4), (12, 63, 16), (12, 63, 7), (16, 112, 16)])
def test_blockfb_several_windows_per_slice_fp64(L, ns, nb):
    """FP64 windows hold (64 // nb) nb sites: 12 x 12 gives windows of 64, 64, 16 (nb = 4, 16) and
    63, 63, 18 with a ragged last block (nb = 7); 16 x 16 gives four windows.  Every window after
    the first starts from the block the previous window's pipelined flush prepared."""
    M, stab = 6, 3
    _free_run(L, ns, M, stab, 4.0, "blockfb", 16, nb, seed=41 + nb, steps=None if L == 12 else 4)


@pytest.mark.parametrize("L,ns,M,stab,steps", [(16, 112, 4, 2, 8), (40, 700, 10, 10, 1)])
def test_local_update_with_several_rows_per_cta_fp64(L, ns, M, stab, steps):
    """N = 256 and N = 1600 sites over at most 152 CTAs: each CTA owns several rows, the path the
    bench's local baseline takes.  Decisions identical, G within 1e-10 after every slice."""
    U = 4.0 if L == 16 else 6.0
    _free_run(L, ns, M, stab, U, "local", 16, 4, seed=7, steps=steps)


def _replay_40x40(mode, k, nb, seed, slices):
    L, ns, M, stab = 40, 700, 10, 10
    N = L * L
    P = inputs.trial_state(L, L, ns)
    X = inputs.initial_fields(M, N, seed=seed)
    model = oracle.Model(L, L, 1.0, 6.0, 0.05, M)
    w = oracle.Walker(model, P, P, X)
    with afqmc.Context(M, U=6.0, precision="fp32", stab_every=stab, seed=seed) as ctx:
        ctx.init_walkers([L], [ns], [ns], np.concatenate([P.ravel(), P.ravel()]), X)
        for ell in range(1, slices + 1):
            u = inputs.uniforms(seed, 0, ell - 1, 2 * N)
            dec, _, extra = w.sweep_slice(ell, +1, mode, u, k=k, nb=nb)
            ctx.sweep_slice(ell, +1, mode, k=k, nb=nb, replay=_replay_bytes(N, mode, nb, dec, extra))
            for s in range(2):
                r = rel(ctx.G(0, s), w.G[s])
                assert r < FP32_TOL, (mode, ell, s, r)
        np.testing.assert_array_equal(ctx.fields(0), w.x)


def test_blockfb_40x40_fp32_replay_thirteen_windows():
    """The bench's block force-bias configuration (nb = 16, FP32 windows of 128 sites: 13 windows
    per slice) for three replayed slices."""
    _replay_40x40("blockfb", 64, 16, seed=3, slices=3)


def test_local_40x40_fp32_replay():
    """The bench's local baseline (FP32, 10-11 rows per CTA) for two replayed slices."""
    _replay_40x40("local", 64, 16, seed=4, slices=2)


@pytest.mark.parametrize("mode,k,nb", [("delayed", 64, 16), ("blockfb", 64, 16)])
def test_mixed_population_fp32_replay(mode, k, nb):
    """Walkers of the population's lattice sizes in one FP32 context (groups per size, launched
    together), each replaying its own oracle chain: G within 1e-5 after every slice of a forward
    run through a recompute."""
    Ls = [8, 12, 16, 8, 12, 24]
    M, stab, U, seed = 6, 3, 4.0, 13
    ns = [inputs.n_sigma_for(L, 0.875) for L in Ls]
    walkers, Ps, Xs = [], [], []
    for wi, L in enumerate(Ls):
        P = inputs.trial_state(L, L, ns[wi])
        X = inputs.initial_fields(M, L * L, seed=seed, walker=wi)
        Ps.append(np.concatenate([P.ravel(), P.ravel()]))
        Xs.append(X.ravel())
        walkers.append(oracle.Walker(oracle.Model(L, L, 1.0, U, 0.05, M), P, P, X))
    with afqmc.Context(M, U=U, precision="fp32", stab_every=stab, seed=seed) as ctx:
        ctx.init_walkers(Ls, ns, ns, np.concatenate(Ps), np.concatenate(Xs))
        for ell in range(1, M + 1):
            reps = []
            for wi, w in enumerate(walkers):
                N = Ls[wi] ** 2
                dec, _, extra = w.sweep_slice(ell, +1, mode, inputs.uniforms(seed, wi, ell - 1, 2 * N), k=k, nb=nb)
                reps.append(_replay_bytes(N, mode, nb, dec, extra))
            ctx.sweep_slice(ell, +1, mode, k=k, nb=nb, replay=np.concatenate(reps))
            for wi, w in enumerate(walkers):
                for s in range(2):
                    r = rel(ctx.G(wi, s), w.G[s])
                    assert r < FP32_TOL, f"walker {wi} (L={Ls[wi]}) slice {ell} spin {s}: {r}"
            if ell % stab == 0:
                ctx.recompute_G()
                for wi, w in enumerate(walkers):
                    w.recompute(stab)
                    for s in range(2):
                        assert rel(ctx.G(wi, s), w.G[s]) < 1e-6
        for wi, w in enumerate(walkers):
            np.testing.assert_array_equal(ctx.fields(wi), w.x)
