"""The schedule comparison itself, on the CPU: equal traces pass, a difference
at an oracle tie is excused (and says so), any other difference fails."""
import pytest

from oracle import params
from schedule_parity import compare

PRM = params.ihs_params("srht")


def _base():
    return [("gd", 1, 1, 0.5 * PRM.c_gd), ("double", 2, 1, 3 * PRM.c_gd), ("gd", 2, 2, 0.2 * PRM.c_gd),
            ("stop", 3, 2, 0.4)]


def test_equal_traces():
    assert compare(_base(), _base(), "srht") == (True, "equal")


def test_difference_away_from_a_tie_fails():
    gpu = _base()
    gpu[1] = ("gd", 2, 1, 0.99 * PRM.c_gd)          # GPU accepted where the oracle doubled at 3 c_gd
    ok, note = compare(gpu, _base(), "srht")
    assert not ok and "decision 1" in note


def test_difference_at_a_tie_is_excused():
    ref = _base()
    ref[1] = ("double", 2, 1, PRM.c_gd * (1 + 2e-4))   # oracle's ratio just above the threshold
    gpu = _base()
    gpu[1] = ("gd", 2, 1, PRM.c_gd * (1 - 1e-5))
    ok, note = compare(gpu, ref, "srht")
    assert ok and note.startswith("tie at decision 1")


def test_a_later_tie_does_not_excuse_an_earlier_difference():
    ref = _base()
    ref[2] = ("gd", 2, 2, PRM.c_gd * (1 - 1e-4))       # a near-tie, but after the first difference
    gpu = list(ref)
    gpu[0] = ("double", 1, 1, 2 * PRM.c_gd)
    ok, _ = compare(gpu, ref, "srht")
    assert not ok


def test_stop_tie_on_either_side():
    ref = _base()
    ref[3] = ("stop", 3, 2, 1.0 - 1e-4)
    gpu = _base()[:3] + [("gd", 3, 2, 0.5 * PRM.c_gd), ("stop", 4, 2, 0.3)]
    assert compare(gpu, ref, "srht")[0]
    ok, note = compare(_base()[:3] + [("stop", 3, 2, 0.9995)], _base()[:3] + [("gd", 3, 2, 0.3 * PRM.c_gd)], "srht")
    assert ok and "GPU stop" in note
    ok, _ = compare(_base()[:3] + [("stop", 3, 2, 0.5)], _base()[:3] + [("gd", 3, 2, 0.3 * PRM.c_gd)], "srht")
    assert not ok


def test_truncated_trace_fails():
    ok, _ = compare(_base()[:2], _base(), "srht")
    assert not ok


@pytest.mark.parametrize("name,thr", [("polyak", PRM.c_p), ("polyak_reject", PRM.c_p), ("gd", PRM.c_gd)])
def test_threshold_by_event(name, thr):
    ref = [(name, 1, 1, thr * (1 + 5e-4))]
    gpu = [("other", 1, 1, 0.0)]
    assert compare(gpu, ref, "srht")[0]
