"""GPU parity of the imaginary spin-z decoupling (Sec. II.B, Eqs. HSspinDecomp, BIOpForHubbard) in the
spin-coupled engine (afqmc_soc_params.hs = AFQMC_SOC_HS_SZ) against the FP64 oracle.

With lam = 0 and the spin-balanced trial state P_dn = conj(P_up) this is the paper's attractive
Hubbard model: the GPU's G must keep no spin-mixing block and G_dn = conj(G_up), every ratio is
real and positive, and FP64 free runs follow the oracle decision for decision with G within 1e-10
after every slice and recompute.  A run with lam = 0.5 covers the phases together with spin mixing.
FP32 replays stay within 1e-5.
"""
import numpy as np
import pytest

import oracle
from paper_2506_09611_gb300 import inputs
from tests.test_gpu_soc import FP32_TOL, FP64_TOL, _free_run, _replay, order, rel

pytestmark = pytest.mark.gpu

soc = pytest.importorskip("paper_2506_09611_gb300.soc")


def make_sz(L, ns, M, stab, precision="fp64", gemm="tc3", U=-4.0, dtau=0.05, lam=0.0, seed=21):
    P = inputs.sz_trial_state(L, ns) if lam == 0.0 else inputs.soc_trial_state(L, 2 * ns, lam=lam)
    X = inputs.initial_fields(M, L * L, seed=seed)
    ctx = soc.SocContext(L, M, 2 * ns, 1, precision, gemm, stab, 1.0, lam, U, dtau, seed, hs="sz")
    ctx.init(P, X)
    model = oracle.SocModel(L, 1.0, lam, U, dtau, M, hs="sz")
    w = oracle.SocWalker(model, P, X)
    return ctx, w


def _spin_structure(G, N, tol):
    assert np.abs(G[:N, N:]).max() < tol and np.abs(G[N:, :N]).max() < tol
    assert np.abs(G[N:, N:] - G[:N, :N].conj()).max() < tol


@pytest.mark.parametrize("L,ns,M,stab", [(3, 4, 8, 4), (4, 7, 6, 3), (6, 15, 8, 4)])
def test_init_G0_and_energy_match_oracle(L, ns, M, stab):
    ctx, w = make_sz(L, ns, M, stab)
    with ctx:
        G = ctx.G(0)
        assert rel(G, w.G) < FP64_TOL
        _spin_structure(G, L * L, 1e-12)
        e = ctx.measure_energy()[0]
        eo = w.m.energy(w.G)
        assert abs(e - eo) < 1e-9 * max(1.0, abs(eo))


@pytest.mark.parametrize("mode,k,nb", [("local", 1, 1), ("delayed", 5, 1), ("delayed", 16, 1),
                                       ("blockfb", 1, 1), ("blockfb", 1, 4), ("blockfb", 1, 7)])
def test_fp64_free_run_matches_oracle(mode, k, nb):
    L, ns, M, stab = 4, 7, 4, 2
    ctx, w = make_sz(L, ns, M, stab, seed=5)
    with ctx:
        _free_run(ctx, w, mode, k, nb, 5, 2 * M, stab, FP64_TOL)
        _spin_structure(ctx.G(0), L * L, 1e-11)
        r = ctx.ratios(0)
        r = r[:L * L] if mode != "blockfb" else r[L * L:L * L + (L * L + nb - 1) // nb]
        assert np.abs(r.imag).max() < 1e-9 * max(1.0, np.abs(r).max())


def test_fp64_ragged_lattice_and_spin_mixing():
    """3 x 3 (2N = 18, a padded row, ragged windows and blocks), and 4 x 4 with lam = 0.5: the
    spin-z phases together with the Rashba spin mixing."""
    for mode, k, nb in (("delayed", 4, 1), ("blockfb", 1, 4)):
        ctx, w = make_sz(3, 4, 4, 2, seed=9)
        with ctx:
            _free_run(ctx, w, mode, k, nb, 9, 8, 2, FP64_TOL)
    for mode, k, nb in (("delayed", 8, 1), ("blockfb", 1, 5)):
        ctx, w = make_sz(4, 8, 4, 2, lam=0.5, seed=11)
        with ctx:
            _free_run(ctx, w, mode, k, nb, 11, 8, 2, FP64_TOL)


@pytest.mark.parametrize("mode,k,nb", [("delayed", 16, 1), ("blockfb", 1, 8), ("local", 1, 1)])
def test_fp32_replay_within_tolerance(mode, k, nb):
    L, ns, M, stab = 6, 15, 6, 3
    ctx, w = make_sz(L, ns, M, stab, precision="fp32", seed=13)
    rng = np.random.default_rng(4321)
    N = L * L
    with ctx:
        for visit, (ell, d) in enumerate(order(M)[:5]):
            rep = _replay(rng, N, mode, nb)
            u = inputs.uniforms(13, 0, visit, 2 * N)
            w.sweep_slice(ell, d, mode, u, k=k, nb=nb, replay=rep)
            ctx.sweep_slice(ell, d, mode, k=k, nb=nb, replay=rep)
            r = rel(ctx.G(0), w.G)
            assert r < FP32_TOL, (mode, ell, d, r)
            if w.pos % stab == 0:
                ctx.recompute_G()
                w.recompute()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("L,ns", [(4, 7), (6, 15)])
def test_pairing_observables_match_oracle(precision, L, ns):
    """afqmc_soc_measure_pairing (Sec. IV's D, <Delta^2>, n_k and the pairing matrix, FP64 from the bulk
    G) against the oracle's soc_pairing evaluated on the same G read back from the device, for two
    walkers after a few free-running slices."""
    M, stab, nw = 4, 2, 2
    N = L * L
    P = inputs.sz_trial_state(L, ns)
    X = np.concatenate([inputs.initial_fields(M, N, seed=40 + w) for w in range(nw)])
    ctx = soc.SocContext(L, M, 2 * ns, nw, precision, "tc3", stab, 1.0, 0.0, -4.0, 0.05, 31, hs="sz")
    model = oracle.SocModel(L, 1.0, 0.0, -4.0, 0.05, M, hs="sz")
    with ctx:
        ctx.init(P, X)
        for ell in (1, 2):
            ctx.sweep_slice(ell, +1, "delayed", k=8)
        got = ctx.measure_pairing()
        for w in range(nw):
            ref = model.pairing(ctx.G(w))
            assert abs(got["D"][w] - ref["D"]) < 1e-11
            assert abs(got["Delta2"][w] - ref["Delta2"]) < 1e-11
            np.testing.assert_allclose(got["nk"][w], ref["nk"], atol=1e-11)
            np.testing.assert_allclose(got["Mk"][w], ref["Mk"], atol=1e-11)
            assert abs(ref["D"].imag) < 1e-6 and 0 < ref["D"].real < 1
        only = ctx.measure_pairing(want_k=False)  # the same sums (FP64 atomics: any order)
        np.testing.assert_allclose(only["D"], got["D"], rtol=1e-13, atol=1e-15)
