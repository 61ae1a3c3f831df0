"""GPU parity of constrained-path AFQMC (afqmc_cp_*, Sec. IV.D) against the FP64 oracle (oracle/cpqmc.py)
on the same seeded inputs: the trial determinant, the walkers' start and the Philox uniforms of
every step.  After every projection step the sampled fields are identical, the ln weight factors
agree to 1e-10, the walkers' determinants to 1e-10 (relative Frobenius norm) and the mixed local
energies to 1e-9; the comb selects the same walkers; after a re-orthonormalisation the basis
differs, so the mixed one-body matrices U_R (U_L U_R)^{-1} U_L are compared instead.  Local heat bath
(one site per window) and the delayed scheme (windows of k sites) give the same fields and weights;
block force bias (n_b = 1, 4, 7, ragged last blocks) draws the oracle's proposals and weights.
"""
import numpy as np
import pytest

import oracle
from oracle.cpqmc import CPEnsemble
from paper_2506_09611_gb300 import inputs

pytestmark = pytest.mark.gpu

afqmc = pytest.importorskip("paper_2506_09611_gb300.afqmc")


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def make(L, ns, nw, U, hs, dtau=0.05, seed=7):
    m = oracle.Model(L, L, 1.0, U, dtau, 1, hs=hs)
    P = inputs.trial_state(L, L, ns)
    rng = np.random.default_rng(100 + L)
    phi = P + 0.2 * rng.standard_normal(P.shape)
    phi0 = np.concatenate([np.concatenate([phi.ravel(), phi.ravel()]) for _ in range(nw)])
    ctx = afqmc.CPContext(L, ns, nw, P, phi0, dtau=dtau, U=U, t=1.0, hs=hs, seed=seed)
    ens = CPEnsemble(m, P, nw, phi0=phi)
    return ctx, ens, seed


def _oracle_step(ens, seed, visit, mode, nb=4):
    N, nw = ens.m.N, len(ens.w)
    u = np.stack([inputs.uniforms(seed, j, visit, 2 * N)[:N] for j in range(nw)])
    w0 = ens.w.copy()
    # the delayed scheme draws the local heat bath's fields
    out = ens.step("blockfb" if mode == "blockfb" else "local", u, nb=nb)
    with np.errstate(divide="ignore"):
        return np.log(ens.w) - np.log(w0), [o[0] for o in out]


def _compare(ctx, ens, lw_gpu, lw_o, x_o, basis=True):
    nw = len(ens.w)
    np.testing.assert_allclose(lw_gpu, lw_o, rtol=0, atol=1e-10)
    el, _ = ctx.energy()
    for j in range(nw):
        np.testing.assert_array_equal(ctx.fields(j), x_o[j])
        phi, _ = ctx.walker(j)
        for s in range(2):
            if basis:
                assert rel(phi[s], ens.UR[j][s]) < 1e-10
            else:
                A = phi[s] @ np.linalg.solve(ens.UL @ phi[s], ens.UL)
                assert rel(A, ens.A(j, s)) < 1e-10
        assert abs(el[j] - ens.local_energy(j)) < 1e-9 * max(1.0, abs(el[j]))


@pytest.mark.parametrize("mode,k,nb", [("local", 1, 1), ("delayed", 4, 1), ("delayed", 16, 1), ("blockfb", 1, 1),
                                       ("blockfb", 1, 4), ("blockfb", 1, 7)])
@pytest.mark.parametrize("L,ns,U,hs", [(4, 7, 4.0, oracle.HS_SZ_REAL), (3, 4, -4.0, oracle.HS_CHARGE_REAL)])
def test_steps_match_the_oracle(mode, k, nb, L, ns, U, hs):
    nw = 3
    ctx, ens, seed = make(L, ns, nw, U, hs)
    with ctx:
        for v in range(4):
            lw_o, x_o = _oracle_step(ens, seed, v, mode, nb)
            lw_g = ctx.step(mode, k, nb)
            _compare(ctx, ens, lw_g, lw_o, x_o)


def test_comb_and_reorthonormalisation_match_the_oracle():
    L, ns, nw = 4, 7, 5
    ctx, ens, seed = make(L, ns, nw, 4.0, oracle.HS_SZ_REAL)
    with ctx:
        v = 0
        for _ in range(3):
            lw_o, x_o = _oracle_step(ens, seed, v, "delayed")
            lw_g = ctx.step("delayed", 8)
            v += 1
        _compare(ctx, ens, lw_g, lw_o, x_o)
        idx_g = ctx.comb(0.41)
        idx_o = ens.comb(0.41)
        np.testing.assert_array_equal(idx_g, idx_o)
        ctx.reorth()
        ens.reorthonormalise()
        for _ in range(2):
            lw_o, x_o = _oracle_step(ens, seed, v, "delayed")
            lw_g = ctx.step("delayed", 8)
            v += 1
            _compare(ctx, ens, lw_g, lw_o, x_o, basis=False)
        _, emean = ctx.energy()
        assert abs(emean - ens.energy()) < 1e-9 * abs(ens.energy())


def test_state_rules():
    L, ns = 3, 4
    P = inputs.trial_state(L, L, ns)
    with afqmc.Context(1, precision="fp32", form="T", stab_every=1) as c32:
        c32.init_walkers([L], [ns], [ns], np.concatenate([P.ravel(), P.ravel()]), np.ones((1, 1, L * L), np.int8))
        with pytest.raises(afqmc.AfqmcError):
            afqmc.afqmc_cp_init(c32.h, P)  # FP64 only
    ctx, ens, seed = make(L, ns, 2, 4.0, oracle.HS_SZ_REAL)
    with ctx:
        with pytest.raises(afqmc.AfqmcError):
            ctx.step("blockfb", 1, 33)  # blocks of at most 32 sites
        with pytest.raises(afqmc.AfqmcError):
            ctx.comb(1.0)  # u0 in [0, 1)
