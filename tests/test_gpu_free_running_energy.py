"""Free-running energies: independent Markov chains of the GPU path (FP64 and FP32 bulk) and of the
FP64 oracle give the same ground-state energy within their statistical errors.

Workload: the 4 x 4 Hubbard lattice of the first configuration (U/t = 4, 7 particles per spin,
dtau = 0.05, M = 40 slices, the free-electron trial state).  Each ensemble is a set of walkers
with their own seeds (so the three ensembles are statistically independent): the oracle runs the
plain local update, the GPU the delayed update (the same Markov chain, Sec. III.A).  The energy
(Eqs. 2DHubbard, Oxformula) is measured at the middle slice l = M/2 on every forward pass, after
the first sweeps are discarded; the estimate is sum(s E) / sum(s) and its error is the standard
jackknife error over walkers.  Replay parity pins single chains element by element; this test
checks what replay cannot: that chains which the FP32 rounding has made diverge still sample the
same distribution.
"""
import numpy as np
import pytest

import oracle
from paper_2506_09611_gb300 import inputs

pytestmark = pytest.mark.gpu

afqmc = pytest.importorskip("paper_2506_09611_gb300.afqmc")

L, NS, U, DTAU, M, STAB = 4, 7, 4.0, 0.05, 40, 10
N = L * L
SWEEPS, BURN = 60, 10


def _order():
    return [(ell, +1) for ell in range(1, M + 1)] + [(ell, -1) for ell in range(M, 0, -1)]


def _estimate(E, S):
    """E, S: [walker][sweep] energies and signs; returns sum(s E) / sum(s) and its jackknife error
    over walkers (a walker's sweeps are correlated; different walkers are independent)."""
    A, B = (E * S).sum(axis=1), S.sum(axis=1)
    n = len(A)
    mean = float(A.sum() / B.sum())
    loo = (A.sum() - A) / (B.sum() - B)
    return mean, float(np.sqrt((n - 1) / n * ((loo - loo.mean()) ** 2).sum()))


def _gpu_ensemble(precision, n_walkers, seed):
    P = inputs.trial_state(L, L, NS)
    X = np.concatenate([inputs.initial_fields(M, N, seed=seed, walker=w).ravel() for w in range(n_walkers)])
    Pcat = np.concatenate([np.concatenate([P.ravel(), P.ravel()])] * n_walkers)
    E = np.zeros((n_walkers, SWEEPS))
    S = np.zeros((n_walkers, SWEEPS))
    decs = []
    with afqmc.Context(M, dtau=DTAU, U=U, precision=precision, stab_every=STAB, seed=seed) as ctx:
        ctx.init_walkers([L] * n_walkers, [NS] * n_walkers, [NS] * n_walkers, Pcat, X)
        for sw in range(SWEEPS):
            for (ell, d) in _order():
                ctx.sweep_slice(ell, d, "delayed", k=16)
                if sw < 2:
                    decs.append(ctx.decisions(0)[:N].copy())
                if d > 0 and ell == M // 2:
                    E[:, sw], S[:, sw] = ctx.measure_energy()
                pos = ell if d > 0 else ell - 1
                if pos % STAB == 0:
                    ctx.recompute_G()
    return E[:, BURN:], S[:, BURN:], decs


def _oracle_ensemble(n_walkers, seed):
    P = inputs.trial_state(L, L, NS)
    model = oracle.Model(L, L, 1.0, U, DTAU, M)
    E = np.zeros((n_walkers, SWEEPS))
    S = np.zeros((n_walkers, SWEEPS))
    for wi in range(n_walkers):
        w = oracle.Walker(model, P, P, inputs.initial_fields(M, N, seed=seed, walker=wi))
        visit = 0
        for sw in range(SWEEPS):
            for (ell, d) in _order():
                w.sweep_slice(ell, d, "local", inputs.uniforms(seed, wi, visit, 2 * N))
                visit += 1
                if d > 0 and ell == M // 2:
                    E[wi, sw] = model.energy(w.G[0], w.G[1])
                    S[wi, sw] = w.sign
                if w.pos % STAB == 0:
                    w.recompute(STAB)
    return E[:, BURN:], S[:, BURN:]


def test_free_running_energies_agree_within_two_sigma():
    e64, s64, d64 = _gpu_ensemble("fp64", 32, seed=101)
    e32, s32, d32 = _gpu_ensemble("fp32", 32, seed=202)
    eor, sor = _oracle_ensemble(16, seed=303)
    est = {"gpu_fp64": _estimate(e64, s64), "gpu_fp32": _estimate(e32, s32), "oracle": _estimate(eor, sor)}
    # the ensembles are independent chains: their decision sequences differ from the first slice
    assert any(not np.array_equal(a, b) for a, b in zip(d64, d32))
    for a, b in (("gpu_fp64", "oracle"), ("gpu_fp32", "oracle"), ("gpu_fp32", "gpu_fp64")):
        (ma, sa), (mb, sb) = est[a], est[b]
        assert sa > 0 and sb > 0
        assert abs(ma - mb) < 2.0 * np.hypot(sa, sb), (a, b, est)
    for m, s in est.values():  # errors small enough for the comparison to mean something
        assert s < 0.02 * abs(m)
