"""Choice of the delay rank k and the block size n_b from timed trial runs.

* Delayed update (Sec. III.A).  The accepted fields and G do not depend on the delay rank: every k
  gives the same Markov chain, so k only trades the rank-k product's efficiency against the
  per-accept panel corrections (Sec. IV.A: time first falls, then rises with k).  The choice is
  the candidate with the least time.
* Block force-bias update (Sec. III.B).  The block size sets both the cost and the acceptance
  ratio, which falls as n_b grows (Sec. IV.B.2).  The paper settles n_b by trial runs that keep
  the time low while the acceptance stays above a chosen floor (0.5 in its example).  The rule
  here: the fastest candidate whose measured acceptance reaches the floor; when none does, the
  candidate with the highest acceptance.

The measurement belongs to the caller: a function of the candidate that runs it through the
public API on the device and returns its time in milliseconds (and, for n_b, its acceptance).
This module orders the candidates, applies the rule, and keeps a JSON cache of the choices per
workload (device, lattice, particle numbers, interaction, precision), so that a production run
tunes once.  `time_on_stream` is the CUDA-event timer the measurements use.
"""
from __future__ import annotations

import json
import math
import os
import tempfile
from dataclasses import asdict, dataclass
from typing import Callable, Iterable, Optional, Sequence, Tuple, Union

# the paper's example floor for the block force-bias acceptance ratio (Sec. IV.B.2)
ACCEPTANCE_FLOOR = 0.5

Measurement = Union[float, Tuple[float, float]]


@dataclass(frozen=True)
class Trial:
    """One candidate's measurement: ms is the best of its repeats, acceptance their mean."""
    value: int
    ms: float
    acceptance: Optional[float] = None


def _split(m: Measurement) -> Tuple[float, Optional[float]]:
    if isinstance(m, tuple):
        ms, acc = float(m[0]), float(m[1])
        if not 0.0 <= acc <= 1.0:
            raise ValueError(f"acceptance {acc} outside [0, 1]")
        return ms, acc
    return float(m), None


def run_trials(candidates: Iterable[int], measure: Callable[[int], Measurement], repeats: int = 1) -> list:
    """measure(c) for every candidate, `repeats` times each, in the order given.  A measurement is
    a time in ms, or (ms, acceptance).  Times must be finite and positive."""
    if repeats < 1:
        raise ValueError("repeats must be >= 1")
    out = []
    seen = set()
    for c in candidates:
        c = int(c)
        if c in seen:
            raise ValueError(f"candidate {c} listed twice")
        seen.add(c)
        times, accs = [], []
        for _ in range(repeats):
            ms, acc = _split(measure(c))
            if not (math.isfinite(ms) and ms > 0.0):
                raise ValueError(f"candidate {c}: time {ms} ms is not a positive finite number")
            times.append(ms)
            if acc is not None:
                accs.append(acc)
        if accs and len(accs) != repeats:
            raise ValueError(f"candidate {c}: acceptance reported by some repeats only")
        out.append(Trial(c, min(times), sum(accs) / len(accs) if accs else None))
    if not out:
        raise ValueError("no candidates")
    return out


def fastest(trials: Sequence[Trial]) -> Trial:
    """The trial with the least time; ties go to the smaller value (less buffer memory)."""
    if not trials:
        raise ValueError("no trials")
    return min(trials, key=lambda t: (t.ms, t.value))


def block_size(trials: Sequence[Trial], floor: float = ACCEPTANCE_FLOOR) -> Trial:
    """The fastest trial whose acceptance is at least `floor`; when none reaches it, the one with
    the highest acceptance (ties: the faster, then the smaller n_b)."""
    if not trials:
        raise ValueError("no trials")
    if any(t.acceptance is None for t in trials):
        raise ValueError("block-size trials need an acceptance")
    ok = [t for t in trials if t.acceptance >= floor]
    if ok:
        return fastest(ok)
    return min(trials, key=lambda t: (-t.acceptance, t.ms, t.value))


def delay_ranks(k_max: int, k_min: int = 8) -> list:
    """Powers of two from k_min up to the largest delay rank the window kernel holds (128 sites
    for an FP32 bulk G, 64 for FP64)."""
    if k_min < 1 or k_max < k_min:
        raise ValueError("need 1 <= k_min <= k_max")
    out, k = [], k_min
    while k <= k_max:
        out.append(k)
        k *= 2
    return out


def block_sizes(nb_max: int = 32, nb_min: int = 2) -> list:
    """Powers of two from nb_min up to the largest block the window kernel holds (32 sites)."""
    return delay_ranks(nb_max, nb_min)


def workload_key(**params) -> str:
    """A canonical key for the cache: the parameters sorted by name, floats in repr form."""
    for k, v in params.items():
        if not isinstance(v, (int, float, str, bool)) or isinstance(v, float) and not math.isfinite(v):
            raise ValueError(f"workload parameter {k}={v!r} is not a finite scalar or a string")
    return json.dumps(params, sort_keys=True, separators=(",", ":"))


class TuneCache:
    """Choices per workload key in a JSON file (written atomically: a temporary file, then a rename)."""

    def __init__(self, path: str):
        self.path = path
        self._d = {}
        if os.path.exists(path):
            with open(path) as f:
                d = json.load(f)
            if not isinstance(d, dict):
                raise ValueError(f"{path}: not a JSON object")
            self._d = d

    def get(self, key: str, knob: str) -> Optional[dict]:
        return self._d.get(key, {}).get(knob)

    def put(self, key: str, knob: str, choice: Trial, trials: Sequence[Trial]) -> None:
        self._d.setdefault(key, {})[knob] = {"choice": asdict(choice), "trials": [asdict(t) for t in trials]}
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".tune.", suffix=".json")
        try:
            with os.fdopen(fd, "w") as f:
                json.dump(self._d, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
        except BaseException:
            if os.path.exists(tmp):
                os.unlink(tmp)
            raise


def tune(cache: Optional[TuneCache], key: str, knob: str, candidates: Iterable[int],
         measure: Callable[[int], Measurement], rule: Callable[[Sequence[Trial]], Trial] = fastest,
         repeats: int = 1) -> Tuple[Trial, list]:
    """The cached choice for (key, knob) when there is one (no measurement then, and an empty
    trial list), else run the trials, apply `rule`, store and return (choice, trials)."""
    if cache is not None:
        hit = cache.get(key, knob)
        if hit is not None:
            return Trial(**hit["choice"]), []
    trials = run_trials(candidates, measure, repeats)
    choice = rule(trials)
    if cache is not None:
        cache.put(key, knob, choice, trials)
    return choice, trials


def time_on_stream(torch, stream, fn: Callable[[], None], n: int = 1) -> float:
    """Milliseconds per call of fn(), between CUDA events recorded on `stream` (the stream the
    library launches on), with a device synchronisation on both sides."""
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(n):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / n


def _walk(ctx, stream, mode, k, nb, slices, stab_every, recompute, direction, want_stats, counted=None):
    """Slices 1..slices forward (direction +1) or slices..1 backward, with the FP64 recompute at
    every multiple of stab_every the walker reaches; returns (accepts, proposals) summed over the
    context's walkers when want_stats, else (0, 0).  counted (nullable) runs one counted slice
    itself, counted(ell, direction, nb) -> (accepts, proposals), for contexts whose sweep_slice
    returns no statistics."""
    acc = prop = 0
    ells = range(1, slices + 1) if direction > 0 else range(slices, 0, -1)
    for ell in ells:
        if want_stats and counted is not None:
            a, p = counted(ell, direction, nb)
            acc += a
            prop += p
        elif want_stats:
            st = ctx.sweep_slice(ell, direction, mode, k=k, nb=nb, want_stats=True, stream=stream)
            acc += sum(s.accepts for s in st)
            prop += sum(s.proposals for s in st)
        else:
            ctx.sweep_slice(ell, direction, mode, k=k, nb=nb, stream=stream)
        pos = ell if direction > 0 else ell - 1
        if pos % stab_every == 0:
            recompute(stream)
    return acc, prop


def autotune_walker(ctx, torch, stream, recompute, slices: int, stab_every: int, k_candidates=None,
                    nb_candidates=None, floor: float = ACCEPTANCE_FLOOR, cache: Optional[TuneCache] = None,
                    key: str = "", k_max: int = 128, nb_max: int = 32, counted=None,
                    tile_candidates=None) -> dict:
    """Delay rank and block size for the walkers of an afqmc Context that sit at slice 0.

    Each candidate walks slices 1..`slices` forward and back down to slice 0, so the context
    ends where it began (its fields have moved on: the walks are Markov-chain steps).  k: one
    untimed walk, then the time of one delayed walk there and back.  n_b: the time of the
    block force-bias walk forward, and its acceptance (accepted over proposed blocks, all
    walkers) on the block force-bias walk back.  `recompute(stream)` runs the FP64 recompute
    the context requires at every multiple of `stab_every` (afqmc_recompute_G).  Contexts whose
    sweep_slice reports no statistics (the spin-orbit-coupled one) pass `counted` (see _walk).
    With tile_candidates (tile widths of the separable wrap, ctx.set_wrap_tile), the width is
    chosen last, by the time of the delayed walk with the chosen k, and left set on the context.
    Returns {"k": Trial, "nb": Trial, "k_trials": [...], "nb_trials": [...]} (plus "tile" and
    "tile_trials" when widths were given); cached choices skip their trials."""
    if not 1 <= slices:
        raise ValueError("slices must be >= 1")
    ks = list(k_candidates) if k_candidates is not None else delay_ranks(k_max, 16)
    nbs = list(nb_candidates) if nb_candidates is not None else block_sizes(nb_max)

    def delayed_round_trip(k):
        _walk(ctx, stream, "delayed", k, 1, slices, stab_every, recompute, +1, False)
        _walk(ctx, stream, "delayed", k, 1, slices, stab_every, recompute, -1, False)

    def measure_k(k):
        delayed_round_trip(k)  # warm-up (first use of this window size)
        return time_on_stream(torch, stream, lambda: delayed_round_trip(k))

    def measure_nb(nb):
        ms = time_on_stream(torch, stream,
                            lambda: _walk(ctx, stream, "blockfb", 1, nb, slices, stab_every, recompute, +1, False))
        acc, prop = _walk(ctx, stream, "blockfb", 1, nb, slices, stab_every, recompute, -1, True, counted)
        if prop <= 0:
            raise RuntimeError(f"block size {nb}: no proposals counted")
        return ms, acc / prop

    k, k_trials = tune(cache, key, "k", ks, measure_k)
    nb, nb_trials = tune(cache, key, "nb", nbs, measure_nb, rule=lambda t: block_size(t, floor))
    out = {"k": k, "nb": nb, "k_trials": k_trials, "nb_trials": nb_trials}
    if tile_candidates is not None:
        def measure_tile(w):
            ctx.set_wrap_tile(w)
            delayed_round_trip(k.value)  # warm-up with this width
            return time_on_stream(torch, stream, lambda: delayed_round_trip(k.value))

        tile, tile_trials = tune(cache, key, "wrap_tile", tile_candidates, measure_tile)
        ctx.set_wrap_tile(tile.value)
        out.update({"tile": tile, "tile_trials": tile_trials})
    return out
