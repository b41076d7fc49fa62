"""Rank decisions of the oracle's rounding that the GPU must reproduce.

The oracle records, for every bond of every rounding, the relative distance `gap` between the
truncation threshold delta and the discarded tail at the chosen rank (and one rank before).  A
rank is unique only when that distance is above the round-off of the two implementations; every
seeded parity case here is chosen so that it is, and the tests assert it instead of skipping a
case that would land on a tie."""

TIE = 1e-9


def gaps(info, keys=None):
    """Every bond gap of one rounding's info (keys=None) or of a step's roundings."""
    if keys is None:
        return [b["gap"] for b in info["bonds"]]
    return [b["gap"] for k in keys for b in info[k]["bonds"]]


STEP_KEYS = ("transport_round", "source_round")


def assert_tie_free(info, keys=None, tie=TIE, where=""):
    g = gaps(info, keys)
    assert min(g) > tie, f"seeded case lands within {tie:g} of the truncation threshold ({where}): {min(g):.3g}"
