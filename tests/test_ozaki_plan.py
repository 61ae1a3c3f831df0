"""The digit-split plan behind the FP64-accurate products (host code, no GPU needed).

The tensor cores compute a group of digit-plane products exactly only if every partial sum is an
integer below 2^24; the FP64 result is complete only if every digit pair (p, q) with
p + q <= s + 1 is summed once and the digits carry at least 54 bits.  These invariants are
checked on the plan the library builds for the recompute's shapes and for the edge of each
digit width's exact range."""
import itertools

import pytest

afqmc = pytest.importorskip("paper_2506_09611_gb300.afqmc")

SHAPES = [(700, 700, 1600, 2), (1600, 1600, 700, 2), (1152, 1152, 2304, 1), (2304, 1152, 1152, 1),
          (252, 252, 576, 140), (576, 576, 252, 140), (33, 70, 13, 1), (128, 128, 1040, 1), (128, 128, 1041, 1),
          (128, 128, 4227, 1), (128, 128, 4228, 1), (64, 64, 17458, 1)]


@pytest.mark.parametrize("M,N,K,batch", SHAPES)
def test_plan_is_exact_and_complete(M, N, K, batch):
    b, s, groups = afqmc.afqmc_debug_ozaki_plan(M, N, K, batch)
    assert b in (5, 6, 7) and b * s >= 54
    seen = []
    for grp in groups:
        assert 1 <= len(grp) <= 16
        levels = {p + q for p, q in grp}
        assert len(levels) == 1  # one power-of-two scale per accumulator
        assert len(grp) * K * (2 ** b - 1) ** 2 < 2 ** 24  # every partial sum exact in FP32
        seen.extend(grp)
    want = [(p, q) for p, q in itertools.product(range(1, s + 1), repeat=2) if p + q <= s + 1]
    assert sorted(seen) == sorted(want)  # every kept pair exactly once


def test_recompute_shapes_use_six_bit_digits():
    """At 40 x 40 both recompute products split into 6-bit digits: 45 pairs."""
    for shape in ((700, 700, 1600, 2), (1600, 1600, 700, 2)):
        b, s, groups = afqmc.afqmc_debug_ozaki_plan(*shape)
        assert (b, s, sum(len(g) for g in groups)) == (6, 9, 45)


def test_plan_rejects_k_beyond_the_exact_range():
    with pytest.raises(afqmc.AfqmcError):
        afqmc.afqmc_debug_ozaki_plan(64, 64, 17459, 1)  # 17459 * 31^2 >= 2^24 even for one pair
    with pytest.raises(afqmc.AfqmcError):
        afqmc.afqmc_debug_ozaki_plan(0, 64, 64, 1)
