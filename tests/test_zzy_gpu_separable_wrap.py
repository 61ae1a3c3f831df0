"""GPU parity of the wrap through the separable lattice propagator (afqmc_set_wrap with
AFQMC_WRAP_SEPARABLE: E = Ex (x) Ex, two L-point passes per product) against the FP64 oracle, in
both of its forms (tile width 0: four line passes, one lattice coordinate each; width > 0: two
tile passes): free-running FP64 sweeps with identical decisions and G within 1e-10 after every
slice, forward and backward, ragged tiles (N = 36 against 16-wide tiles) and a lattice side that
is not a multiple of 4 (the line passes' scalar path); FP32 replay at 16 x 16 and at the bench's
40 x 40 within 1e-5.  The file sorts after the rest of the GPU suite."""
import numpy as np
import pytest

import oracle
from paper_2506_09611_gb300 import inputs
from tests.test_gpu_parity import FP32_TOL, _run_sweep, make, rel

pytestmark = pytest.mark.gpu

afqmc = pytest.importorskip("paper_2506_09611_gb300.afqmc")


@pytest.mark.parametrize("tile", [0, 16])
@pytest.mark.parametrize("L,ns,mode,k,nb", [(4, 7, "delayed", 8, 4), (6, 15, "delayed", 16, 4),
                                            (6, 15, "blockfb", 16, 5), (6, 15, "local", 16, 4)])
def test_separable_wrap_fp64_free_running(L, ns, mode, k, nb, tile):
    ctx, w, P, X = make(L, ns, 6, stab=3, U=6.0)
    with ctx:
        ctx.set_wrap("separable")
        ctx.set_wrap_tile(tile)
        _run_sweep(ctx, w, mode, k=k, nb=nb, stab=3)


@pytest.mark.parametrize("tile", [0, 4])
@pytest.mark.parametrize("L,ns,M,stab,k", [(16, 112, 10, 5, 32), (40, 700, 10, 10, 64)])
def test_separable_wrap_fp32_replay(L, ns, M, stab, k, tile):
    N = L * L
    P = inputs.trial_state(L, L, ns)
    X = inputs.initial_fields(M, N, seed=3)
    model = oracle.Model(L, L, 1.0, 6.0, 0.05, M)
    w = oracle.Walker(model, P, P, X)
    with afqmc.Context(M, U=6.0, precision="fp32", stab_every=stab, seed=3) as ctx:
        ctx.init_walkers([L], [ns], [ns], np.concatenate([P.ravel(), P.ravel()]), X)
        ctx.set_wrap("separable")
        ctx.set_wrap_tile(tile)
        for ell in (1, 2, 3):
            u = inputs.uniforms(3, 0, ell - 1, 2 * N)
            dec, _, _ = w.sweep_slice(ell, +1, "delayed", u, k=k)
            rep = np.zeros(2 * N, np.uint8)
            rep[:N] = dec
            ctx.sweep_slice(ell, +1, "delayed", k=k, replay=rep)
            for s in range(2):
                r = rel(ctx.G(0, s), w.G[s])
                assert r < FP32_TOL, (ell, s, r)


def test_set_wrap_rejects_an_unknown_mode():
    ctx, w, P, X = make(4, 7, 4, stab=2)
    with ctx:
        with pytest.raises(afqmc.AfqmcError) as e:
            ctx.set_wrap(7)
        assert e.value.code == -1
