"""The N > 1 path of bench.py on the CPU: two gloo ranks agree on the slowest rank's time and the
whole-job throughput counts every rank's updates (weak scaling, one walker per rank)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = 100.0 + 25.0 * rank  # rank 1 is the slow one
        out[rank] = (bench.max_over_ranks(dist, ms, "cpu"),
                     bench.job_throughput(world, 1000, 2, bench.max_over_ranks(dist, ms, "cpu")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_sum_the_work():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as mgr:  # no fork of a process that already runs threads
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == 125.0
        assert value == pytest.approx(world * 1000 * 2 / 0.125)


def test_single_rank_throughput():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_throughput(1, 256000, 3, 1500.0) == pytest.approx(256000 * 3 / 1.5)


def test_an_auxiliary_leg_that_fails_is_reported_in_the_line(capsys):
    sys.path.insert(0, ROOT)
    import bench

    assert bench.optional_leg("soc", lambda: {"value": 1.0}) == {"value": 1.0}

    def boom():
        raise RuntimeError("afqmc_soc_sweep_slice failed: -3")

    assert bench.optional_leg("soc", boom) == {"error": "RuntimeError: afqmc_soc_sweep_slice failed: -3"}
    assert "soc leg failed" in capsys.readouterr().err


def test_dense_wrap_leg_times_whole_sweeps_with_that_wrap():
    """bench.dense_wrap_leg on a fake device: it switches the context from the default separable
    wrap to the dense wrap before the first slice, times whole sweeps (2M slice-steps), reports the
    tensor-core product's roofline from the profile, and closes the context."""
    import types

    sys.path.insert(0, ROOT)
    import bench

    clock = {"t": 0.0}
    made = []

    class Ev:
        def __init__(self, enable_timing=True):
            self.t = 0.0

        def record(self, stream=None):
            self.t = clock["t"]

        def elapsed_time(self, other):
            return other.t - self.t

    class Ctx:
        def __init__(self, M, **kw):
            self.h, self.wrap, self.closed, self.slices = object(), "separable", False, 0
            made.append(self)

        def init_walkers(self, *a, **kw):
            pass

        def set_wrap(self, mode):
            self.wrap = mode

        def sweep_slice(self, ell, d, mode, k=32, nb=4, stream=None):
            assert self.wrap == "dense" and mode == "delayed"
            self.slices += 1
            clock["t"] += 2.0

        def set_profiling(self, on):
            pass

        def profile(self):
            return {"wrap": {"ms": 7.5}, "wrap_gemm": {"ms": 7.0, "intervals": 320}}

        def close(self):
            self.closed = True

    fake_torch = types.SimpleNamespace(
        cuda=types.SimpleNamespace(Event=Ev, synchronize=lambda: None),
        empty=lambda *a, **k: types.SimpleNamespace(zero_=lambda: None), float32=None)
    fake_afqmc = types.SimpleNamespace(Context=Ctx, afqmc_recompute_G=lambda h, n, s: None)
    args = types.SimpleNamespace(gemm="tc3", steps=2, k=64, nb=16)
    r = bench.dense_wrap_leg(fake_afqmc, fake_torch, None, args, 1, 52.0)
    assert r["ms_per_step"] == 2.0 * 2 * bench.M
    assert r["value"] == bench.N * bench.M * 2 / (r["ms_per_step"] / 1e3)
    assert r["wrap_ms_per_step"] == 7.5 and r["separable_wrap_ms_per_step"] == 52.0
    roof = r["wrap_gemm_roofline"]
    assert roof["bound"] == "tensor" and roof["work_per_launch"] == 2 * 2 * bench.N ** 3
    assert made[-1].closed and made[-1].slices == (1 + 2 + 1) * 2 * bench.M  # warm-up, timed, profiled


def test_kernel_rooflines_use_the_documented_work_per_launch():
    """bench.kernel_rooflines on a synthetic profile: the algorithmic work per launch is the
    documented figure (wrap: 2 x 2 N^3 flop for both spins; flush: read + write of both spins' FP32
    G; solve: 2 x 2 Nsigma^2 N), achieved = work x launches / summed time, frac = achieved / peak,
    and the list is sorted by time per step (the dominant kernel first)."""
    sys.path.insert(0, ROOT)
    import bench

    N, NS = bench.N, bench.NS
    assert (N, NS) == (1600, 700)
    pk = {"hbm_gbs": 6789.6, "bf16_tflops": 1911.7, "sm_max_mhz": 2070.0}
    prof = {"wrap_gemm": {"ms": 52.0, "intervals": 320}, "flush_gemm": {"ms": 160.0, "intervals": 4000},
            "solve": {"ms": 13.0, "intervals": 16}, "elim": {"ms": 0.0, "intervals": 0}}
    out = bench.kernel_rooflines(prof, "tc3", pk, "measured", steps=1, wrap="dense")
    by = {r["kernel"].split(" ")[0]: r for r in out}
    wrap = by["wrap"]
    assert wrap["work_per_launch"] == 2 * 2 * 1600 ** 3 == 1.6384e10
    assert wrap["achieved"] == pytest.approx(1.6384e10 * 320 / 0.052 / 1e12)
    assert wrap["peak"] == pytest.approx(1911.7 * 1.1 / 2.25) and wrap["bound"] == "tensor"
    assert wrap["frac"] == pytest.approx(wrap["achieved"] / wrap["peak"])
    flush = by["rankm_kernel:"]
    assert flush["work_per_launch"] == 2 * 2 * 1600 * 1600 * 4 == 40960000
    assert flush["achieved"] == pytest.approx(40960000 * 4000 / 0.160 / 1e9) and flush["unit"] == "GB/s"
    solve = by["lu_solve_kernel"]
    assert solve["work_per_launch"] == pytest.approx(2 * 2.0 * 700 ** 2 * 1600)
    assert "elim" not in {r["kernel"] for r in out} and len(out) == 3
    assert [r["ms_per_step"] for r in out] == sorted((r["ms_per_step"] for r in out), reverse=True)
    assert out[0] is flush  # 160 ms per step: the dominant entry
    # the separable wrap: one interval is one wrap, four L-point passes over both spins' G, each
    # pass a kernel launch that reads and writes G (line passes) or two tile launches
    sep = {r["kernel"].split(" ")[0]: r for r in bench.kernel_rooflines(prof, "tc3", pk, "measured", steps=1)}
    s = sep["sep_line_kernel"]
    assert s["work_per_launch"] == 2 * 2 * 4 * 40 * 1600 ** 2 and s["bound"] == "alu"
    assert s["bytes_per_launch"] == 4 * 2 * 2 * 1600 ** 2 * 4 and s["launches_per_interval"] == 4
    assert s["peak"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    t = {r["kernel"].split(" ")[0]: r for r in
         bench.kernel_rooflines(prof, "tc3", pk, "measured", steps=1, wrap_tile=8)}["sep_kernel"]
    assert t["work_per_launch"] == s["work_per_launch"] and t["bytes_per_launch"] == s["bytes_per_launch"] / 2


def _fake_clock_torch(clock):
    import types

    class Ev:
        def __init__(self, enable_timing=True):
            self.t = 0.0

        def record(self, stream=None):
            self.t = clock["t"]

        def elapsed_time(self, other):
            return other.t - self.t

    return types.SimpleNamespace(cuda=types.SimpleNamespace(Event=Ev, synchronize=lambda: None))


def test_walkers_leg_times_one_sweep_of_n_walkers_with_graphs():
    """bench.walkers_40x40_leg on a fake device: per walker count one context with n walkers of the
    headline lattice, graphs on before the untimed sweep, one timed sweep (2M slice-steps with a
    recompute at every multiple of the period), rate = n N 2M / time, and the context closed."""
    import types

    sys.path.insert(0, ROOT)
    import bench

    clock = {"t": 0.0}
    made = []

    class Ctx:
        def __init__(self, M, **kw):
            self.h, self.graphs, self.closed, self.slices, self.n = object(), False, False, 0, 0
            assert kw["stab_every"] == bench.STAB and kw["precision"] == "fp32"
            made.append(self)

        def init_walkers(self, Ls, nu, nd, P, X, stream=None):
            self.n = len(Ls)
            assert Ls == [bench.L] * self.n and len(X) == self.n * bench.M * bench.N

        def set_graphs(self, on):
            self.graphs = on

        def sweep_slice(self, ell, d, mode, k=32, nb=4, stream=None):
            assert self.graphs and mode == "delayed"
            self.slices += 1
            clock["t"] += 1.0 + 0.25 * self.n

        def close(self):
            self.closed = True

    recs = []
    fake_afqmc = types.SimpleNamespace(Context=Ctx, afqmc_recompute_G=lambda h, n, s: recs.append(h))
    args = types.SimpleNamespace(gemm="tc3", k=64, nb=16)
    r = bench.walkers_40x40_leg(fake_afqmc, _fake_clock_torch(clock), None, args, 1, counts=(2, 4))
    for n, ctx in zip((2, 4), made):
        ms = 2 * bench.M * (1.0 + 0.25 * n)
        assert r[f"walkers_{n}"]["ms_per_step"] == ms
        assert r[f"walkers_{n}"]["value"] == n * bench.N * bench.M * 2 / (ms / 1e3)
        assert ctx.closed and ctx.slices == 2 * 2 * bench.M  # capture sweep + timed sweep
    # one recompute at every multiple of the period, both directions, in both sweeps of both counts
    per_sweep = 2 * (bench.M // bench.STAB)
    assert len(recs) == 2 * 2 * per_sweep


def test_cpqmc_leg_reports_each_scheme_and_its_speedup():
    """bench.cpqmc_leg on a fake device: every scheme (local heat bath, delayed k = 16 and 32, block
    force bias n_b = 8) gets its own ensemble, two untimed steps, CP_STEPS timed steps with the comb
    and a re-orthonormalisation every CP_EVERY steps, rate = walkers N steps / time, and the
    speed-ups are relative to the local scheme."""
    import types

    sys.path.insert(0, ROOT)
    import bench

    clock = {"t": 0.0}
    cost = {"local": 10.0, "delayed": 1.0, "blockfb": 0.5}
    made = []

    class CP:
        def __init__(self, L, ns, n, P, **kw):
            self.steps, self.combs, self.reorths, self.closed = [], 0, 0, False
            assert (L, n) == (bench.CP_L, bench.CP_WALKERS)
            made.append(self)

        def step(self, mode, k, nb, stream=None):
            self.steps.append((mode, k, nb))
            clock["t"] += cost[mode] * (32.0 / k if mode == "delayed" else 1.0)

        def comb(self, u0, stream=None):
            assert 0.0 <= u0 < 1.0
            self.combs += 1

        def reorth(self, stream=None):
            self.reorths += 1

        def energy(self, stream=None):
            return [0.0], -1.0

        def close(self):
            self.closed = True

    fake_afqmc = types.SimpleNamespace(CPContext=CP)
    r = bench.cpqmc_leg(fake_afqmc, _fake_clock_torch(clock), None, 1)
    n = bench.CP_L * bench.CP_L
    expect = {"local": 10.0, "delayed_k16": 2.0, "delayed_k32": 1.0, "blockfb_nb8": 0.5}
    for key, c in expect.items():
        assert r[key]["ms_per_step"] == pytest.approx(c)
        assert r[key]["value"] == pytest.approx(bench.CP_WALKERS * n * bench.CP_STEPS / (c * bench.CP_STEPS / 1e3))
        assert r["speedup_vs_local"][key] == pytest.approx(10.0 / c)
    for cp in made:
        assert cp.closed and len(cp.steps) == 2 + bench.CP_STEPS
        assert cp.combs == cp.reorths == bench.CP_STEPS // bench.CP_EVERY
