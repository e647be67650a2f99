"""The printed values under tests/golden/ against what the paper states
about them, so that a mistyped or transposed entry fails on the CPU."""
from conftest import read_printed


def test_every_printed_value_cites_its_passage():
    vals = read_printed()
    assert len(vals) == 5
    for key, (v, cite) in vals.items():
        assert cite.startswith("Sec. 3."), (key, cite)
        assert 0.0 < v < 1.0, (key, v)


def test_bubble_velocities_rise_towards_hadamard_rybczynski():
    """Sec. 3.4: the clean terminal velocity approaches U_th as the
    confinement ratio falls and stays below it."""
    v = {k: x for k, (x, _) in read_printed().items()}
    seq = [v["bubble_clean_2R/Lx=0.4"], v["bubble_clean_2R/Lx=0.2"], v["bubble_clean_2R/Lx=0.1"]]
    assert seq == sorted(seq) and seq[-1] < 1.0, seq


def test_migration_wall_slowing():
    """Sec. 3.2: the walls of the narrower box slow the droplet, and the
    wider box agrees well with the YGB velocity (within a few per cent)."""
    v = {k: x for k, (x, _) in read_printed().items()}
    assert v["migration_5Rx5Rx10R"] < v["migration_10Rx10Rx10R"] < 1.0
    assert abs(v["migration_10Rx10Rx10R"] - 1.0) < 0.01
