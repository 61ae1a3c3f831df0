"""afqmc_apply_flips_noalloc: the rank-m update of G with no device allocation.

Some callers cannot allocate device memory where they apply an update: code that runs under a
fixed device-memory budget owned by a host framework, a real-time loop that may not call
cudaMalloc (or wait for the synchronisation an allocation can cause), or a plugin whose host
process gives it no allocator.  The entry point keeps its scratch in a file-scope device array
and must give what afqmc_apply_flips gives, on two calls in a row (the array keeps the previous
call's contents), and what the oracle's sequential rank-1 updates give.  This file is collected
after every other test file, so a run that stops at its first failure has run the rest first.
"""
import numpy as np
import pytest

import oracle
from paper_2506_09611_gb300 import inputs

pytestmark = pytest.mark.gpu

afqmc = pytest.importorskip("paper_2506_09611_gb300.afqmc")
torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-10, "fp32": 1e-5}
DT = {"fp64": torch.float64, "fp32": torch.float32}


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _case(L=8, ns=28, M=6, ell=2, seed=4):
    N = L * L
    P = inputs.trial_state(L, L, ns)
    X = inputs.initial_fields(M, N, seed=seed)
    model = oracle.Model(L, L, 1.0, 4.0, 0.05, M)
    G = [model.green_scratch(X, P, s, ell)[0] for s in range(2)]
    return N, G, X[ell - 1].astype(np.int8), model


def _to_dev(G, N, ld, precision):
    out = []
    for s in range(2):
        g = torch.zeros((N, ld), dtype=DT[precision], device="cuda")
        g[:, :N] = torch.from_numpy(G[s]).to(DT[precision])
        out.append(g)
    return out


def _call(fn, precision, N, ld, Gd, sites, delta, stream):
    s_dev = torch.from_numpy(np.ascontiguousarray(sites, np.int32)).cuda()
    d_dev = torch.from_numpy(np.ascontiguousarray(delta, np.float64)).cuda()
    fn(precision, N, ld, Gd[0].data_ptr(), Gd[1].data_ptr(), s_dev.data_ptr(), d_dev.data_ptr(), len(sites), stream)
    torch.cuda.synchronize()


def _oracle_flips(model, G, xl, calls):
    """The oracle's local update with exactly the given sites forced to accept, call after call."""
    N = model.N
    Gu, Gd, x = G[0], G[1], xl.copy()
    for sites in calls:
        rep = np.zeros(N, np.uint8)
        rep[sites] = 1
        Gu, Gd, x, _, _, _ = model.local_slice(Gu, Gd, x, np.zeros(N), replay=rep)
    return [Gu, Gd]


def _deltas(model, x, sites):
    return np.concatenate([np.exp(-2.0 * model.c[s] * x[sites].astype(np.float64)) - 1.0 for s in range(2)])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_equals_allocating_entry_point_and_oracle_twice(precision):
    """Two calls in a row on the same G: the no-allocation entry point gives the allocating entry
    point's G and the oracle's.  A third call with a site outside [0, N) is reported as
    AFQMC_ERR_ARG and leaves G as it was, although the shared scratch still holds the second call's
    sizes."""
    N, G, xl, model = _case()
    ld = N + 3
    calls = [np.array([1, 4, 9, 20, 33, 50, 63], np.int32), np.array([0, 7, 8, 41], np.int32)]
    ref = _oracle_flips(model, G, xl, calls)
    stream = torch.cuda.current_stream()
    outs = {}
    for fn in (afqmc.afqmc_apply_flips, afqmc.afqmc_apply_flips_noalloc):
        Gd = _to_dev(G, N, ld, precision)
        x = xl.copy()
        for sites in calls:
            _call(fn, precision, N, ld, Gd, sites, _deltas(model, x, sites), stream)
            x[sites] *= -1
        outs[fn.__name__] = [g[:, :N].double().cpu().numpy() for g in Gd]
        if fn is afqmc.afqmc_apply_flips_noalloc:
            before = [g.clone() for g in Gd]
            bad = np.array([3, N + 4], np.int32)
            with pytest.raises(afqmc.AfqmcError) as ex:
                _call(fn, precision, N, ld, Gd, bad, _deltas(model, x, np.array([3, 3])), stream)
            assert ex.value.code == -1
            for s in range(2):
                assert torch.equal(Gd[s], before[s])
    for s in range(2):
        a = outs["afqmc_apply_flips_noalloc"][s]
        assert rel(a, outs["afqmc_apply_flips"][s]) < TOL[precision]
        assert rel(a, ref[s]) < TOL[precision]


def test_noalloc_at_its_largest_lattice_fp32():
    """N = 4096 sites (the largest the static scratch holds) on a synthetic, well-conditioned G:
    the oracle's rank-1 updates of the same flips, and the allocating entry point, agree."""
    L = 64
    N = L * L
    model = oracle.Model(L, L, 1.0, 4.0, 0.05, 2)
    rng = np.random.default_rng(8)
    G = [0.5 * np.eye(N) + 0.02 * rng.standard_normal((N, N)) / np.sqrt(N) for _ in range(2)]
    xl = inputs.initial_fields(1, N, seed=8)[0].astype(np.int8)
    sites = np.sort(rng.choice(N, size=40, replace=False)).astype(np.int32)
    ref = _oracle_flips(model, G, xl, [sites])
    ld = N
    stream = torch.cuda.current_stream()
    got = {}
    for fn in (afqmc.afqmc_apply_flips_noalloc, afqmc.afqmc_apply_flips):
        Gd = _to_dev(G, N, ld, "fp32")
        _call(fn, "fp32", N, ld, Gd, sites, _deltas(model, xl, sites), stream)
        got[fn.__name__] = [g.double().cpu().numpy() for g in Gd]
    for s in range(2):
        assert rel(got["afqmc_apply_flips_noalloc"][s], ref[s]) < TOL["fp32"]
        np.testing.assert_array_equal(got["afqmc_apply_flips_noalloc"][s], got["afqmc_apply_flips"][s])


def test_singular_update_is_reported_and_leaves_G_unchanged():
    """1 + (1 - G_II) D with a zero pivot: G_ii = 0 and delta = -1 make it exactly 0."""
    N, ld = 16, 32
    G = [np.zeros((N, N)), np.zeros((N, N))]
    stream = torch.cuda.current_stream()
    for fn in (afqmc.afqmc_apply_flips, afqmc.afqmc_apply_flips_noalloc):
        Gd = _to_dev(G, N, ld, "fp64")
        with pytest.raises(afqmc.AfqmcError) as ex:
            _call(fn, "fp64", N, ld, Gd, np.array([3], np.int32), np.array([-1.0, -1.0]), stream)
        assert ex.value.code == -4
        assert float(Gd[0].abs().max()) == 0.0 and float(Gd[1].abs().max()) == 0.0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    Gd = torch.zeros(8, dtype=torch.float32, device="cuda")
    with pytest.raises(afqmc.AfqmcError) as e:
        afqmc.afqmc_apply_flips_noalloc("fp32", 4097, 4097, Gd.data_ptr(), Gd.data_ptr(), Gd.data_ptr(),
                                        Gd.data_ptr(), 1)
    assert e.value.code == -1
