"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Both sides get the same seeded inputs: trial state P, initial fields and the
Philox uniforms of every slice visit (the device generator is checked bit for
bit against the input module's numpy Philox first).  FP64 runs free: the
decisions must be identical and G must agree to 1e-10 (relative Frobenius
norm) after every slice.  FP32 runs replay the oracle's decisions and G must
stay within 1e-5 between FP64 recomputes.
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


def make(L, ns, M, U=4.0, dtau=0.05, stab=4, precision="fp64", seed=11, hs=oracle.HS_SZ_REAL, wrap=None):
    P = inputs.trial_state(L, L, ns)
    X = inputs.initial_fields(M, L * L, seed=seed)
    ctx = afqmc.Context(M, dtau=dtau, U=U, precision=precision, hs=hs, stab_every=stab, seed=seed)
    ctx.init_walkers([L], [ns], [ns], np.concatenate([P.ravel(), P.ravel()]), X)
    if wrap is not None:
        ctx.set_wrap(wrap)
    model = oracle.Model(L, L, 1.0, U, dtau, M, hs)
    w = oracle.Walker(model, P, P, X)
    return ctx, w, P, X


def test_device_philox_matches_numpy():
    for (seed, walker, visit) in [(1, 0, 0), (11, 3, 17), (2**40 + 5, 7, 123456)]:
        dev = afqmc.afqmc_debug_uniforms(seed, walker, visit, 1000)
        ref = inputs.uniforms(seed, walker, visit, 1000)
        np.testing.assert_array_equal(dev, ref)


@pytest.mark.parametrize("L,ns,M,stab", [(4, 7, 8, 4), (6, 13, 12, 3)])
def test_init_G0_matches_oracle(L, ns, M, stab):
    ctx, w, P, X = make(L, ns, M, stab=stab)
    with ctx:
        for s in range(2):
            assert rel(ctx.G(0, s), w.G[s]) < FP64_TOL
        e, sg = ctx.measure_energy()
        assert abs(e[0] - w.m.energy(w.G[0], w.G[1])) < 1e-9 * max(1, abs(e[0]))
        assert sg[0] == w.sign


def _replay(N, nb, dec, extra):
    """Replay bytes of a block force-bias slice: the proposed fields (x' = +1) of the N sites, then
    the decision of each block."""
    rep = np.zeros(2 * N, np.uint8)
    rep[:N] = (extra["xprop"] > 0)
    rep[N:N + (N + nb - 1) // nb] = dec
    return rep


def _run_sweep(ctx, w, mode, k=16, nb=4, seed=11, slices=None, stab=4, tol=FP64_TOL, check_every=True):
    M = w.m.M
    N = w.m.N
    order = [(ell, +1) for ell in range(1, M + 1)] + [(ell, -1) for ell in range(M, 0, -1)]
    if slices is not None:
        order = order[:slices]
    visit = 0
    for (ell, d) in order:
        u = inputs.uniforms(seed, 0, visit, 2 * N)
        visit += 1
        dec_o, ratio_o, extra = w.sweep_slice(ell, d, mode, u, k=k, nb=nb)
        ctx.sweep_slice(ell, d, mode, k=k, nb=nb)
        dec_g = ctx.decisions(0)
        if mode == "blockfb":
            nblocks = (N + nb - 1) // nb
            np.testing.assert_array_equal(dec_g[N:N + nblocks], dec_o, err_msg=f"block decisions slice {ell} dir {d}")
            np.testing.assert_array_equal(dec_g[:N], (extra["xprop"] > 0).astype(np.uint8))
        else:
            np.testing.assert_array_equal(dec_g[:N], dec_o, err_msg=f"decisions slice {ell} dir {d}")
        if check_every:
            for s in range(2):
                r = rel(ctx.G(0, s), w.G[s])
                assert r < tol, f"slice {ell} dir {d} spin {s}: rel err {r}"
        if w.pos % stab == 0:
            ctx.recompute_G()
            w.recompute(stab)
            for s in range(2):
                assert rel(ctx.G(0, s), w.G[s]) < tol
    np.testing.assert_array_equal(ctx.fields(0), w.x)


@pytest.mark.parametrize("wrap", ["dense", "separable"])
@pytest.mark.parametrize("mode,k,nb", [("local", 16, 4), ("delayed", 1, 4), ("delayed", 5, 4), ("delayed", 16, 4),
                                       ("blockfb", 16, 1), ("blockfb", 16, 4), ("blockfb", 16, 7),
                                       ("blockfb", 16, 16)])
def test_sweep_fp64_free_running(mode, k, nb, wrap):
    """nb = 16 = N is the full force-bias update (Sec. II.D): one block holds the whole slice."""
    ctx, w, P, X = make(4, 7, 8, stab=4, wrap=wrap)
    with ctx:
        _run_sweep(ctx, w, mode, k=k, nb=nb)


@pytest.mark.parametrize("mode,k,nb", [("local", 16, 4), ("delayed", 16, 4), ("delayed", 64, 4),
                                       ("blockfb", 16, 5)])
def test_sweep_fp64_ragged_6x6(mode, k, nb):
    """N = 36: delayed windows of 16 leave a ragged tail of 4; blocks of 5 leave a tail of 1."""
    ctx, w, P, X = make(6, 15, 6, stab=3, U=6.0)
    with ctx:
        _run_sweep(ctx, w, mode, k=k, nb=nb, stab=3)


def test_delayed_matches_local_on_gpu_8x8():
    """Same uniforms: the GPU delayed and local updates take the same decisions (Sec. IV.C)."""
    L, ns, M = 8, 28, 6
    P = inputs.trial_state(L, L, ns)
    X = inputs.initial_fields(M, L * L, seed=3)
    out = {}
    for mode in ("local", "delayed"):
        with afqmc.Context(M, precision="fp64", stab_every=3, seed=3) as ctx:
            ctx.init_walkers([L], [ns], [ns], np.concatenate([P.ravel(), P.ravel()]), X)
            decs = []
            for ell in range(1, 4):
                ctx.sweep_slice(ell, +1, mode, k=32)
                decs.append(ctx.decisions(0)[:L * L].copy())
                if ell % 3 == 0:
                    ctx.recompute_G()
            out[mode] = (decs, ctx.G(0, 0), ctx.G(0, 1))
    for a, b in zip(out["local"][0], out["delayed"][0]):
        np.testing.assert_array_equal(a, b)
    assert rel(out["delayed"][1], out["local"][1]) < FP64_TOL
    assert rel(out["delayed"][2], out["local"][2]) < FP64_TOL


@pytest.mark.parametrize("wrap", ["dense", "separable"])
@pytest.mark.parametrize("mode,k,nb", [("local", 32, 4), ("delayed", 32, 4), ("delayed", 128, 4),
                                       ("blockfb", 32, 8)])
def test_sweep_fp32_replay(mode, k, nb, wrap):
    """FP32 bulk with the oracle's decisions forced: G within 1e-5 between FP64 recomputes, with the
    dense tensor-core wrap and with the separable wrap."""
    L, ns, M, stab = 8, 28, 10, 5
    P = inputs.trial_state(L, L, ns)
    X = inputs.initial_fields(M, L * L, seed=5)
    model = oracle.Model(L, L, 1.0, 4.0, 0.05, M)
    w = oracle.Walker(model, P, P, X)
    N = L * L
    with afqmc.Context(M, precision="fp32", stab_every=stab, seed=5) as ctx:
        ctx.init_walkers([L], [ns], [ns], np.concatenate([P.ravel(), P.ravel()]), X)
        ctx.set_wrap(wrap)
        for s in range(2):
            assert rel(ctx.G(0, s), w.G[s]) < 1e-6
        visit = 0
        for ell in range(1, M + 1):
            u = inputs.uniforms(5, 0, visit, 2 * N)
            visit += 1
            dec, ratio, extra = w.sweep_slice(ell, +1, mode, u, k=k, nb=nb)
            rep = np.zeros(2 * N, np.uint8)
            if mode == "blockfb":
                nblocks = (N + nb - 1) // nb
                rep[:N] = (extra["xprop"] > 0)
                rep[N:N + nblocks] = dec
            else:
                rep[:N] = dec
            ctx.sweep_slice(ell, +1, mode, k=k, nb=nb, replay=rep)
            for s in range(2):
                r = rel(ctx.G(0, s), w.G[s])
                assert r < FP32_TOL, f"slice {ell} spin {s}: {r}"
            if ell % stab == 0:
                drift = ctx.recompute_G()
                w.recompute(stab)
                assert drift[0] < FP32_TOL
                for s in range(2):
                    assert rel(ctx.G(0, s), w.G[s]) < 1e-6
        np.testing.assert_array_equal(ctx.fields(0), w.x)


def test_charge_channel_fp64():
    """Attractive U with the real charge decoupling (prefactor exp(-lam x) in the ratio)."""
    ctx, w, P, X = make(4, 5, 8, U=-4.0, stab=4, hs=oracle.HS_CHARGE_REAL)
    with ctx:
        _run_sweep(ctx, w, "delayed", k=8, slices=8)
        _run_sweep.__doc__  # keep flake quiet


def test_full_size_40x40_first_slices():
    """40x40 (N = 1600, 700 per spin) with the kernels and launch configuration of the bench
    (delayed windows of 64 sites; FP64 here, FP32 replay below).  M = 10 keeps the oracle's own
    FP64 G(0) cheap; the slice kernels do not depend on M.  G(0), the decisions of two forward
    slices and G after each are compared with the oracle; projector invariants hold."""
    L, ns, M, stab = 40, 700, 10, 10
    N = L * L
    P = inputs.trial_state(L, L, ns)
    X = inputs.initial_fields(M, N, seed=1)
    model = oracle.Model(L, L, 1.0, 6.0, 0.05, M)
    w = oracle.Walker(model, P, P, X)
    with afqmc.Context(M, U=6.0, precision="fp64", stab_every=stab, seed=1) as ctx:
        ctx.init_walkers([L], [ns], [ns], np.concatenate([P.ravel(), P.ravel()]), X)
        for s in range(2):
            G0 = ctx.G(0, s)
            assert rel(G0, w.G[s]) < FP64_TOL
            assert abs(np.trace(np.eye(N) - G0) - ns) < 1e-8
        for ell in (1, 2):
            u = inputs.uniforms(1, 0, ell - 1, 2 * N)
            dec, _, _ = w.sweep_slice(ell, +1, "delayed", u, k=64)
            ctx.sweep_slice(ell, +1, "delayed", k=64)
            np.testing.assert_array_equal(ctx.decisions(0)[:N], dec)
            for s in range(2):
                assert rel(ctx.G(0, s), w.G[s]) < FP64_TOL


def test_full_size_40x40_fp32_replay():
    L, ns, M, stab = 40, 700, 10, 10
    N = L * L
    P = inputs.trial_state(L, L, ns)
    X = inputs.initial_fields(M, N, seed=2)
    model = oracle.Model(L, L, 1.0, 6.0, 0.05, M)
    w = oracle.Walker(model, P, P, X)
    with afqmc.Context(M, U=6.0, precision="fp32", stab_every=stab, seed=2) as ctx:
        ctx.init_walkers([L], [ns], [ns], np.concatenate([P.ravel(), P.ravel()]), X)
        ctx.set_wrap("dense")  # the tensor-core wrap at full size (the separable one: its own file)
        for ell in (1, 2, 3):
            u = inputs.uniforms(2, 0, ell - 1, 2 * N)
            dec, _, _ = w.sweep_slice(ell, +1, "delayed", u, k=64)
            rep = np.zeros(2 * N, np.uint8)
            rep[:N] = dec
            ctx.sweep_slice(ell, +1, "delayed", k=64, replay=rep)
            for s in range(2):
                r = rel(ctx.G(0, s), w.G[s])
                assert r < FP32_TOL, (ell, s, r)


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("fp32", FP32_TOL)])
def test_apply_flips_matches_oracle(precision, tol):
    """afqmc_apply_flips (stateless Woodbury rank-m update) = the oracle's sequential rank-1
    updates with the same sites forced to accept; m = 0 is a no-op, and an out-of-range site is
    reported as AFQMC_ERR_ARG with G left unchanged."""
    torch = pytest.importorskip("torch")
    L, ns, M, ell = 6, 15, 6, 3
    N = L * L
    P = inputs.trial_state(L, L, ns)
    X = inputs.initial_fields(M, N, seed=9)
    model = oracle.Model(L, L, 1.0, 6.0, 0.05, M)
    G = [model.green_scratch(X, P, s, ell)[0] for s in range(2)]
    sites = np.array([2, 5, 11, 12, 30, 35], np.int32)
    rep = np.zeros(N, np.uint8)
    rep[sites] = 1
    Gu_ref, Gd_ref, _, _, _, _ = model.local_slice(G[0], G[1], X[ell - 1], np.zeros(N), replay=rep)
    x = X[ell - 1, sites].astype(np.float64)
    delta = np.concatenate([np.exp(-2.0 * model.c[s] * x) - 1.0 for s in range(2)])
    ld = N + 7
    dt = torch.float64 if precision == "fp64" else torch.float32
    Gd_dev = [torch.zeros((N, ld), dtype=dt, device="cuda") for _ in range(2)]
    for s in range(2):
        Gd_dev[s][:, :N] = torch.from_numpy(G[s]).to(dt)
    s_dev = torch.from_numpy(sites).cuda()
    d_dev = torch.from_numpy(delta).cuda()
    stream = torch.cuda.current_stream()
    afqmc.afqmc_apply_flips(precision, N, ld, Gd_dev[0].data_ptr(), Gd_dev[1].data_ptr(), s_dev.data_ptr(),
                            d_dev.data_ptr(), len(sites), stream)
    # no-ops
    afqmc.afqmc_apply_flips(precision, N, ld, Gd_dev[0].data_ptr(), Gd_dev[1].data_ptr(), s_dev.data_ptr(),
                            d_dev.data_ptr(), 0, stream)
    bad = torch.tensor([3, N + 4], dtype=torch.int32, device="cuda")
    with pytest.raises(afqmc.AfqmcError) as ex:  # found on the device, reported, G untouched
        afqmc.afqmc_apply_flips(precision, N, ld, Gd_dev[0].data_ptr(), Gd_dev[1].data_ptr(), bad.data_ptr(),
                                d_dev.data_ptr(), 2, stream)
    assert ex.value.code == -1
    torch.cuda.synchronize()
    for s, ref in enumerate((Gu_ref, Gd_ref)):
        got = Gd_dev[s][:, :N].double().cpu().numpy()
        assert rel(got, ref) < tol
        assert float(Gd_dev[s][:, N:].abs().max()) == 0.0  # padding untouched
    with pytest.raises(afqmc.AfqmcError):
        afqmc.afqmc_apply_flips(precision, N, N - 1, Gd_dev[0].data_ptr(), Gd_dev[1].data_ptr(), s_dev.data_ptr(),
                                d_dev.data_ptr(), len(sites), stream)


@pytest.mark.parametrize("mode,k,nb", [("delayed", 5, 4), ("local", 16, 4), ("blockfb", 16, 3)])
def test_mixed_walker_groups_fp64(mode, k, nb):
    """Walkers of mixed lattices in one context.  Walkers with the same lattice form a group
    whose every launch covers them all; each walker still takes its own oracle's decisions
    (its uniforms are keyed by its index in the context) and G agrees to 1e-10 after every
    slice of a forward and a backward sweep, recomputes included."""
    Ls = [4, 6, 4, 6, 4]
    M, stab, U, seed = 8, 4, 4.0, 21
    ns_of = {4: 7, 6: 16}
    walkers, Ps, Xs = [], [], []
    for wi, L in enumerate(Ls):
        P = inputs.trial_state(L, L, ns_of[L])
        X = inputs.initial_fields(M, L * L, seed=seed, walker=wi)
        Ps.append(np.concatenate([P.ravel(), P.ravel()]))
        Xs.append(X.ravel())
        walkers.append(oracle.Walker(oracle.Model(L, L, 1.0, U, 0.05, M), P, P, X))
    ns = [ns_of[L] for L in Ls]
    with afqmc.Context(M, U=U, precision="fp64", stab_every=stab, seed=seed) as ctx:
        ctx.init_walkers(Ls, ns, ns, np.concatenate(Ps), np.concatenate(Xs))
        for wi, w in enumerate(walkers):
            for s in range(2):
                assert rel(ctx.G(wi, s), w.G[s]) < FP64_TOL
        order = [(ell, +1) for ell in range(1, M + 1)] + [(ell, -1) for ell in range(M, 0, -1)]
        for visit, (ell, d) in enumerate(order):
            ctx.sweep_slice(ell, d, mode, k=k, nb=nb)
            for wi, w in enumerate(walkers):
                N = Ls[wi] ** 2
                dec_o, _, extra = w.sweep_slice(ell, d, mode, inputs.uniforms(seed, wi, visit, 2 * N), k=k, nb=nb)
                dec_g = ctx.decisions(wi)
                if mode == "blockfb":
                    nblocks = (N + nb - 1) // nb
                    np.testing.assert_array_equal(dec_g[N:N + nblocks], dec_o)
                else:
                    np.testing.assert_array_equal(dec_g[:N], dec_o, err_msg=f"walker {wi} slice {ell} dir {d}")
                for s in range(2):
                    r = rel(ctx.G(wi, s), w.G[s])
                    assert r < FP64_TOL, f"walker {wi} slice {ell} dir {d} spin {s}: {r}"
            if walkers[0].pos % stab == 0:
                ctx.recompute_G()
                for wi, w in enumerate(walkers):
                    w.recompute(stab)
                    for s in range(2):
                        assert rel(ctx.G(wi, s), w.G[s]) < FP64_TOL
        e, sg = ctx.measure_energy()
        for wi, w in enumerate(walkers):
            np.testing.assert_array_equal(ctx.fields(wi), w.x)
            assert abs(e[wi] - w.m.energy(w.G[0], w.G[1])) < 1e-9 * max(1.0, abs(e[wi]))
            assert sg[wi] == w.sign


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_replay_matches_direct_launches(precision):
    """With CUDA graphs on, every slice is captured on its first visit and replayed after that
    (the second sweep below is all replays); decisions and G are bit-identical to direct launches
    because the uniforms are keyed by a device-side visit counter."""
    Ls = [4, 6, 4]
    M, stab, seed = 4, 2, 9
    ns_of = {4: 7, 6: 16}
    P = np.concatenate([np.concatenate([inputs.trial_state(L, L, ns_of[L]).ravel()] * 2) for L in Ls])
    X = np.concatenate([inputs.initial_fields(M, L * L, seed=seed, walker=wi).ravel() for wi, L in enumerate(Ls)])
    ns = [ns_of[L] for L in Ls]
    ctxs = [afqmc.Context(M, U=4.0, precision=precision, stab_every=stab, seed=seed) for _ in range(2)]
    try:
        for c in ctxs:
            c.init_walkers(Ls, ns, ns, P, X)
        ctxs[1].set_graphs(True)
        order = [(ell, +1) for ell in range(1, M + 1)] + [(ell, -1) for ell in range(M, 0, -1)]
        for sweep in range(2):
            for (ell, d) in order:
                for c in ctxs:
                    c.sweep_slice(ell, d, "delayed", k=8)
                for wi in range(len(Ls)):
                    np.testing.assert_array_equal(ctxs[0].decisions(wi), ctxs[1].decisions(wi))
                    for s in range(2):
                        np.testing.assert_array_equal(ctxs[0].G(wi, s), ctxs[1].G(wi, s))
                pos = ell if d > 0 else ell - 1
                if pos % stab == 0:
                    for c in ctxs:
                        c.recompute_G()
        for wi in range(len(Ls)):
            np.testing.assert_array_equal(ctxs[0].fields(wi), ctxs[1].fields(wi))
    finally:
        for c in ctxs:
            c.close()


@pytest.mark.parametrize("precision,L,ns,nb", [("fp64", 5, 11, 25), ("fp32", 5, 11, 25)])
def test_full_force_bias_one_block_per_slice(precision, L, ns, nb):
    """The full force-bias update (Sec. II.D, Eqs. FullFrcbsPhiLPhiR, RatioApprox, AcceptRatio): block
    force bias with n_b = N, one proposal and one N-site determinant per slice, on the largest square
    lattice whose slice fits one block (n_b <= 32).  FP64 runs free against the oracle (identical
    decisions, G within 1e-10 per slice); FP32 replays the oracle's proposals and decisions (G within
    1e-5 per slice)."""
    M, stab = 4, 2
    N = L * L
    assert nb == N
    ctx, w, P, X = make(L, ns, M, stab=stab, precision=precision, U=4.0)
    with ctx:
        if precision == "fp64":
            _run_sweep(ctx, w, "blockfb", k=16, nb=nb, stab=stab)
            return
        for ell in range(1, M + 1):
            u = inputs.uniforms(11, 0, ell - 1, 2 * N)
            dec, _, extra = w.sweep_slice(ell, +1, "blockfb", u, k=16, nb=nb)
            ctx.sweep_slice(ell, +1, "blockfb", k=16, nb=nb, replay=_replay(N, nb, dec, extra))
            for s_ in range(2):
                assert rel(ctx.G(0, s_), w.G[s_]) < FP32_TOL, (ell, s_)
            if ell % stab == 0:
                ctx.recompute_G()
                w.recompute()
