"""Choice of the delay rank and the block size (host logic, no GPU): the paper's rules on
synthetic cost and acceptance curves, the trial bookkeeping and the JSON cache."""
import math

import pytest

from paper_2506_09611_gb300 import tune


def test_trials_keep_the_best_time_and_the_mean_acceptance():
    calls = []
    samples = {4: [(3.0, 0.8), (2.0, 0.6)], 8: [(1.5, 0.4), (1.7, 0.2)]}

    def measure(nb):
        calls.append(nb)
        return samples[nb][sum(1 for c in calls if c == nb) - 1]

    tr = tune.run_trials([4, 8], measure, repeats=2)
    assert calls == [4, 4, 8, 8]  # in the order given, every repeat
    assert tr[0] == tune.Trial(4, 2.0, pytest.approx(0.7))
    assert tr[1] == tune.Trial(8, 1.5, pytest.approx(0.3))


@pytest.mark.parametrize("bad", [0.0, -1.0, math.inf, math.nan])
def test_trials_reject_a_time_that_is_not_positive_and_finite(bad):
    with pytest.raises(ValueError):
        tune.run_trials([16], lambda k: bad)


def test_trials_reject_duplicates_bad_acceptance_and_mixed_reports():
    with pytest.raises(ValueError):
        tune.run_trials([16, 16], lambda k: 1.0)
    with pytest.raises(ValueError):
        tune.run_trials([4], lambda nb: (1.0, 1.5))
    flip = iter([(1.0, 0.5), 1.0])
    with pytest.raises(ValueError):
        tune.run_trials([4], lambda nb: next(flip), repeats=2)
    with pytest.raises(ValueError):
        tune.run_trials([], lambda k: 1.0)


def test_delay_rank_is_the_fastest_on_a_time_curve_with_an_interior_minimum():
    """Sec. IV.A: the time per sweep first falls with k (fewer, larger rank-k products), then rises
    (the per-accept corrections grow with k).  The rule picks the minimum; a tie goes to the
    smaller k."""
    n_sigma = 700

    def ms(k):  # the rank-k product's overhead per site falls as 1/k; the per-accept corrections grow with k
        return 1e-3 * (4.0 * n_sigma ** 2 / k + 0.5 * k * n_sigma)

    tr = tune.run_trials(tune.delay_ranks(128), ms)
    best = tune.fastest(tr)
    assert best.value == min(tune.delay_ranks(128), key=ms)
    assert best.value not in (8, 128)  # interior
    assert tune.fastest([tune.Trial(64, 1.0), tune.Trial(32, 1.0)]).value == 32


def test_block_size_is_the_fastest_admissible_one():
    """Sec. IV.B.2: larger blocks are cheaper per site but accepted less often.  With the fastest
    block below the 0.5 floor, the choice is the fastest block at or above it."""
    def measure(nb):
        return 200.0 / nb + nb / 4.0, math.exp(-nb / 20.0)

    tr = tune.run_trials(tune.block_sizes(), measure)
    assert tune.fastest(tr).value == 32  # fastest overall, acceptance 0.20
    choice = tune.block_size(tr)
    assert choice.value == 8  # acceptance exp(-0.4) = 0.67 >= 0.5; 16 gives 0.45
    assert tune.block_size(tr, floor=0.4).value == 16
    assert tune.block_size(tr, floor=0.0).value == 32


def test_block_size_without_an_admissible_candidate_takes_the_highest_acceptance():
    tr = [tune.Trial(4, 9.0, 0.30), tune.Trial(8, 5.0, 0.20), tune.Trial(16, 3.0, 0.10)]
    assert tune.block_size(tr).value == 4
    tied = [tune.Trial(4, 9.0, 0.30), tune.Trial(2, 7.0, 0.30)]
    assert tune.block_size(tied).value == 2
    with pytest.raises(ValueError):
        tune.block_size([tune.Trial(4, 1.0)])


def test_candidate_lists_follow_the_window_limits():
    assert tune.delay_ranks(128) == [8, 16, 32, 64, 128]
    assert tune.delay_ranks(64, 16) == [16, 32, 64]
    assert tune.delay_ranks(100) == [8, 16, 32, 64]
    assert tune.block_sizes() == [2, 4, 8, 16, 32]
    with pytest.raises(ValueError):
        tune.delay_ranks(4)


def test_workload_key_is_canonical():
    a = tune.workload_key(L=40, n_up=700, U=6.0, precision="fp32")
    b = tune.workload_key(precision="fp32", U=6.0, n_up=700, L=40)
    assert a == b
    assert a != tune.workload_key(L=40, n_up=700, U=4.0, precision="fp32")
    with pytest.raises(ValueError):
        tune.workload_key(U=math.nan)
    with pytest.raises(ValueError):
        tune.workload_key(shape=[40, 40])


def test_cache_round_trip_and_a_hit_skips_the_measurement(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    key = tune.workload_key(L=16, n_up=112, U=4.0, precision="fp32")
    cache = tune.TuneCache(path)
    choice, trials = tune.tune(cache, key, "k", [16, 32], lambda k: {16: 2.0, 32: 1.0}[k])
    assert choice == tune.Trial(32, 1.0) and len(trials) == 2

    def boom(k):
        raise AssertionError("measured despite a cached choice")

    again = tune.TuneCache(path)  # a new process reads the file
    choice2, trials2 = tune.tune(again, key, "k", [16, 32], boom)
    assert choice2 == choice and trials2 == []
    # another knob or another workload is measured
    nb, _ = tune.tune(again, key, "nb", [4, 8], lambda nb: (1.0 / nb, 0.9 - nb / 20), rule=tune.block_size)
    assert nb.value == 8
    other = tune.workload_key(L=24, n_up=252, U=4.0, precision="fp32")
    assert tune.tune(again, other, "k", [16], lambda k: 3.0)[0].value == 16
    assert sorted(tune.TuneCache(path)._d) == sorted([key, other])
    assert [p.name for p in (tmp_path / "sub").iterdir()] == ["tune.json"]  # no temporary left


def test_cache_rejects_a_file_that_is_not_an_object(tmp_path):
    p = tmp_path / "t.json"
    p.write_text("[1, 2]")
    with pytest.raises(ValueError):
        tune.TuneCache(str(p))


def test_time_on_stream_brackets_n_calls_with_events_on_the_given_stream():
    log = []

    class FakeEvent:
        def __init__(self, enable_timing):
            assert enable_timing
            self.t = None

        def record(self, stream):
            log.append(("record", stream))
            self.t = sum(1 for e in log if e[0] == "call")

        def elapsed_time(self, other):
            return 10.0 * (other.t - self.t)  # 10 ms per call

    class Cuda:
        Event = FakeEvent

        @staticmethod
        def synchronize():
            log.append(("sync",))

    class Torch:
        cuda = Cuda

    ms = tune.time_on_stream(Torch, "s1", lambda: log.append(("call",)), n=3)
    assert ms == pytest.approx(10.0)
    assert log[0] == ("sync",) and log[-1] == ("sync",)
    assert log[1] == ("record", "s1") and log[-2] == ("record", "s1")
    assert sum(1 for e in log if e[0] == "call") == 3


class _FakeContext:
    """The sequencing rules of afqmc_sweep_slice / afqmc_recompute_G (slice order, direction, a
    recompute owed at every multiple of stab_every, the k and n_b limits) on a fake clock."""

    def __init__(self, M, stab, n_walkers=2):
        self.M, self.stab, self.n = M, stab, n_walkers
        self.pos, self.owed, self.clock, self.calls = 0, False, 0.0, 0

    def sweep_slice(self, ell, direction, mode, k=32, nb=4, want_stats=False, stream=None):
        self.calls += 1
        assert not self.owed, "recompute owed"
        assert 1 <= ell <= self.M
        assert self.pos == (ell - 1 if direction > 0 else ell)
        if mode == "delayed":
            assert 1 <= k <= 128
            self.clock += 40.0 / k + 0.1 * k  # minimum at k = 20 -> 16 of {16, 32, 64, 128}
        else:
            assert mode == "blockfb" and 1 <= nb <= 32
            self.clock += 30.0 / nb
        self.pos = ell if direction > 0 else ell - 1
        self.owed = self.pos % self.stab == 0
        if not want_stats:
            return None
        acc = round(100 * math.exp(-nb / 20.0))
        return [type("S", (), {"proposals": 100, "accepts": acc})() for _ in range(self.n)]

    def recompute(self, stream):
        assert self.pos % self.stab == 0
        self.owed = False


class _ClockTorch:
    def __init__(self, ctx):
        ctx_ = ctx

        class Ev:
            def __init__(self, enable_timing):
                self.t = 0.0

            def record(self, stream):
                self.t = ctx_.clock

            def elapsed_time(self, other):
                return other.t - self.t

        self.cuda = type("C", (), {"Event": Ev, "synchronize": staticmethod(lambda: None)})


@pytest.mark.parametrize("slices,stab", [(20, 10), (15, 10), (3, 1)])
def test_autotune_walker_follows_the_sweep_rules_and_returns_to_slice_zero(slices, stab, tmp_path):
    ctx = _FakeContext(M=40, stab=stab)
    cache = tune.TuneCache(str(tmp_path / "t.json"))
    key = tune.workload_key(L=40, n_up=700, U=6.0, precision="fp32")
    r = tune.autotune_walker(ctx, _ClockTorch(ctx), None, ctx.recompute, slices, stab, cache=cache, key=key)
    assert ctx.pos == 0 and not ctx.owed  # back at slice 0, nothing owed
    assert r["k"].value == 16
    assert [t.value for t in r["k_trials"]] == [16, 32, 64, 128]
    # time falls with n_b, acceptance exp(-n_b / 20): 8 is the largest block with >= 0.5
    assert r["nb"].value == 8 and r["nb"].acceptance == pytest.approx(0.67)
    assert [t.value for t in r["nb_trials"]] == [2, 4, 8, 16, 32]
    assert r["nb_trials"][0].ms == pytest.approx(slices * 15.0)  # the timed forward walk only
    calls = ctx.calls
    r2 = tune.autotune_walker(ctx, _ClockTorch(ctx), None, ctx.recompute, slices, stab, cache=cache, key=key)
    assert ctx.calls == calls and r2["k"] == r["k"] and r2["nb"] == r["nb"]  # cached: no sweeps


def test_autotune_walker_times_the_wrap_tile_widths_and_leaves_the_fastest_set(tmp_path):
    class TiledContext(_FakeContext):
        tile = 0

        def set_wrap_tile(self, w):
            assert w in (4, 8, 16)
            self.tile = w

        def sweep_slice(self, ell, direction, mode, k=32, nb=4, want_stats=False, stream=None):
            if mode == "delayed":
                self.clock += {0: 0.0, 4: 0.5, 8: 0.2, 16: 0.9}[self.tile]  # 8 is the fastest width
            return super().sweep_slice(ell, direction, mode, k, nb, want_stats, stream)

    ctx = TiledContext(M=20, stab=10)
    cache = tune.TuneCache(str(tmp_path / "t.json"))
    r = tune.autotune_walker(ctx, _ClockTorch(ctx), None, ctx.recompute, 10, 10, k_candidates=[16, 32],
                             nb_candidates=[4], cache=cache, key="w", tile_candidates=(4, 8, 16))
    assert r["tile"].value == 8 and ctx.tile == 8
    assert [t.value for t in r["tile_trials"]] == [4, 8, 16]
    assert ctx.pos == 0 and not ctx.owed
    ctx.tile = 0
    r2 = tune.autotune_walker(ctx, _ClockTorch(ctx), None, ctx.recompute, 10, 10, k_candidates=[16, 32],
                              nb_candidates=[4], cache=cache, key="w", tile_candidates=(4, 8, 16))
    assert r2["tile"].value == 8 and ctx.tile == 8 and r2["tile_trials"] == []  # from the cache


def test_autotune_walker_with_a_lower_floor_takes_larger_blocks():
    ctx = _FakeContext(M=10, stab=5)
    r = tune.autotune_walker(ctx, _ClockTorch(ctx), None, ctx.recompute, 5, 5, k_candidates=[32],
                             nb_candidates=[4, 16, 32], floor=0.3)
    assert r["k"].value == 32 and r["nb"].value == 16


def test_run_cli_tunes_then_walks_with_the_choice(tmp_path, monkeypatch, capsys):
    """`python -m paper_2506_09611_gb300.run --tune CACHE`: the trials run once, the walk uses the
    chosen k and n_b, and a second run reads the cache without trial walks (fake device)."""
    import json

    import numpy as np

    torch = pytest.importorskip("torch")
    from paper_2506_09611_gb300 import afqmc, run

    made = []

    class Ctx(_FakeContext):
        def __init__(self, M, **kw):
            super().__init__(M=M, stab=kw["stab_every"], n_walkers=1)
            self.h = object()
            self.modes = []
            made.append(self)

        def init_walkers(self, *a, **kw):
            pass

        def sweep_slice(self, ell, direction, mode, k=32, nb=4, want_stats=False, stream=None):
            self.modes.append((mode, k, nb))
            return super().sweep_slice(ell, direction, mode, k, nb, want_stats, stream)

        def measure_energy(self, stream=None):
            return np.array([-1.0]), np.array([1.0])

        def set_wrap(self, mode):
            self.wrap = mode

        def set_wrap_tile(self, w):
            self.tile = w

        def close(self):
            pass

    class Ev:
        def __init__(self, enable_timing=True):
            self.t = 0.0

        def record(self, stream=None):
            self.t = made[-1].clock

        def elapsed_time(self, other):
            return other.t - self.t

    monkeypatch.setattr(afqmc, "load", lambda *a: None)
    monkeypatch.setattr(afqmc, "Context", Ctx)
    monkeypatch.setattr(afqmc, "afqmc_recompute_G", lambda h, n, st: made[-1].recompute(st))
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "Event", Ev)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "fake")
    cache = str(tmp_path / "tune.json")
    argv = ["--L", "4", "--M", "10", "--stab", "5", "--slices", "4", "--mode", "blockfb", "--tune", cache,
            "--tune-slices", "5", "--wrap", "dense"]
    run.main(argv)
    out = json.loads(capsys.readouterr().out)
    assert (out["k"], out["nb"]) == (16, 8) and out["tuned"]["cached"] is False
    assert made[-1].modes[-4:] == [("blockfb", 16, 8)] * 4  # the walk itself
    run.main(argv)
    out2 = json.loads(capsys.readouterr().out)
    assert (out2["k"], out2["nb"]) == (16, 8) and out2["tuned"]["cached"] is True
    assert made[-1].modes == [("blockfb", 16, 8)] * 4  # no trial walks with a cached choice
    run.main(argv[:-1] + ["separable"])
    out3 = json.loads(capsys.readouterr().out)
    assert out3["wrap"] == "separable" and made[-1].wrap == "separable"
    # the separable wrap's walk is keyed apart from the dense one and tunes its tile width too
    assert out3["tuned"]["cached"] is False and out3["tuned"]["wrap_tile"] in (0, 4, 8, 16)
    assert made[-1].tile == out3["tuned"]["wrap_tile"]
    with pytest.raises(SystemExit):
        run.main(["--soc", "--wrap", "separable"])


def test_run_cli_tunes_the_soc_walker_from_its_decisions(tmp_path, monkeypatch, capsys):
    """`run --soc --tune CACHE`: the spin-orbit-coupled context reports no slice statistics, so
    the block acceptance comes from its decisions (replay layout: N proposals, then the blocks)."""
    import json

    import numpy as np

    torch = pytest.importorskip("torch")
    from paper_2506_09611_gb300 import afqmc, run, soc

    made = []

    class SocCtx:
        def __init__(self, L, M, n_e, n_walkers, precision, gemm, stab, t, lam, U, dtau, seed):
            self.inner = _FakeContext(M=M, stab=stab, n_walkers=n_walkers)
            self.N, self.h, self.last_nb, self.modes = L * L, object(), None, []
            made.append(self)

        def init(self, P, X, stream=None):
            pass

        def sweep_slice(self, ell, direction, mode, k=32, nb=16, replay=None, stream=None):
            self.modes.append((mode, k, nb))
            self.last_nb = nb
            self.inner.sweep_slice(ell, direction, mode, k, min(nb, 32), False, stream)

        def decisions(self, walker=0):
            nb = self.last_nb
            nblk = (self.N + nb - 1) // nb
            d = np.zeros(2 * self.N, np.uint8)
            d[self.N:self.N + round(nblk * math.exp(-nb / 20.0))] = 1
            return d

        def measure_energy(self, stream=None):
            return np.array([-1.0 + 0.0j])

        def close(self):
            pass

    class Ev:
        def __init__(self, enable_timing=True):
            self.t = 0.0

        def record(self, stream=None):
            self.t = made[-1].inner.clock

        def elapsed_time(self, other):
            return other.t - self.t

    monkeypatch.setattr(afqmc, "load", lambda *a: None)
    monkeypatch.setattr(soc, "SocContext", SocCtx)
    monkeypatch.setattr(soc, "afqmc_soc_recompute_G", lambda h, n, st: made[-1].inner.recompute(st))
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "Event", Ev)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "fake")
    argv = ["--soc", "--L", "4", "--M", "10", "--stab", "5", "--slices", "3", "--mode", "blockfb", "--tune",
            str(tmp_path / "t.json"), "--tune-slices", "5"]
    run.main(argv)
    out = json.loads(capsys.readouterr().out)
    # k from {16, 32, 64} (FP32 window limit 64); n_b from {2, ..., 64}: 8 is the largest block whose
    # acceptance (1 of 2 blocks) reaches 0.5
    assert out["model"] == "soc" and (out["k"], out["nb"]) == (16, 8)
    assert out["tuned"]["nb_acceptance"] == 0.5 and out["tuned"]["cached"] is False
    assert {nb for m, _, nb in made[-1].modes if m == "blockfb"} >= {2, 4, 8, 16, 32, 64}
    assert made[-1].inner.pos == 3 and made[-1].modes[-3:] == [("blockfb", 16, 8)] * 3
