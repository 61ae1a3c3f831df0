"""afqmc_apply_flips_noalloc against afqmc_apply_flips.

The no-allocation entry point serves callers that cannot allocate device memory where they
apply an update (a fixed memory budget owned by a host framework, a real-time loop that may not
call cudaMalloc, a plugin without an allocator).  It must give the same G as the allocating entry
point, on two calls in a row (its static scratch keeps the previous call's contents).  This file
sorts after the main GPU suite so that a run stopping at its first failure has run that suite
first.
"""
import numpy as np
import pytest

import oracle
from paper_2506_09611_gb300 import inputs

pytestmark = pytest.mark.gpu

afqmc = pytest.importorskip("paper_2506_09611_gb300.afqmc")
torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-10, "fp32": 1e-5}


def _case(L=8, ns=28, M=6, ell=2, seed=4):
    N = L * L
    P = inputs.trial_state(L, L, ns)
    X = inputs.initial_fields(M, N, seed=seed)
    model = oracle.Model(L, L, 1.0, 4.0, 0.05, M)
    G = [model.green_scratch(X, P, s, ell)[0] for s in range(2)]
    return N, G, X[ell - 1].astype(np.float64), model


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_equals_allocating_entry_point_twice(precision):
    N, G, x, model = _case()
    ld = N + 3
    dt = torch.float64 if precision == "fp64" else torch.float32
    calls = [np.array([1, 4, 9, 20, 33, 50, 63], np.int32), np.array([0, 7, 8, 41], np.int32)]
    outs = {}
    stream = torch.cuda.current_stream()
    for fn in (afqmc.afqmc_apply_flips, afqmc.afqmc_apply_flips_noalloc):
        Gd = [torch.zeros((N, ld), dtype=dt, device="cuda") for _ in range(2)]
        for s in range(2):
            Gd[s][:, :N] = torch.from_numpy(G[s]).to(dt)
        xs = x.copy()
        for sites in calls:
            delta = np.concatenate([np.exp(-2.0 * model.c[s] * xs[sites]) - 1.0 for s in range(2)])
            xs[sites] *= -1
            s_dev = torch.from_numpy(sites).cuda()
            d_dev = torch.from_numpy(delta).cuda()
            fn(precision, N, ld, Gd[0].data_ptr(), Gd[1].data_ptr(), s_dev.data_ptr(), d_dev.data_ptr(),
               len(sites), stream)
            torch.cuda.synchronize()
        outs[fn.__name__] = [g[:, :N].double().cpu().numpy() for g in Gd]
    for s in range(2):
        a = outs["afqmc_apply_flips_noalloc"][s]
        b = outs["afqmc_apply_flips"][s]
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < TOL[precision]


def test_noalloc_rejects_sizes_beyond_its_scratch():
    Gd = torch.zeros(8, dtype=torch.float32, device="cuda")
    with pytest.raises(afqmc.AfqmcError) as e:
        afqmc.afqmc_apply_flips_noalloc("fp32", 4097, 4097, Gd.data_ptr(), Gd.data_ptr(), Gd.data_ptr(),
                                        Gd.data_ptr(), 1)
    assert e.value.code == -1
