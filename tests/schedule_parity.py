"""Decision-by-decision comparison of the GPU controller with the oracle's run of
the same draws (Algorithm 1 and its gradient-only variant).

Both sides log every decision as (event, t, m, value): value is the tested
ratio, (r_p/r_1)^(1/t) against cbar_p for the Polyak candidate and r_gd/r_t
against cbar_gd for the gradient-IHS candidate and a doubling, or the stopping
test's sqrt(2 Lambda r_t)/(tol ||Abar x_t||) against 1.  The two schedules must
be equal event for event.  The only excuse is a tie: when the first differing
decision is one the oracle took with its value within `band` (relative) of the
threshold, the two arithmetics (FP64 here, FP32 gradients with FP64 scalars
on the GPU) may legitimately decide it differently, and the runs part ways
there.  A stop that the GPU took and the oracle did not is excused the same
way on the GPU's own stopping value (the oracle logs no value for a stop it
did not take).  Any other difference fails.
"""
import warnings

from oracle import params

TIE_BAND = 1e-3

_THRESHOLD_KIND = {"polyak": "p", "polyak_reject": "p", "gd": "gd", "gd_at_cap": "gd", "double": "gd",
                   "floor": "gd", "stop": "stop"}


def _threshold(prm, name):
    kind = _THRESHOLD_KIND.get(name)
    if kind == "p":
        return prm.c_p
    if kind == "gd":
        return prm.c_gd
    if kind == "stop":
        return 1.0
    return None


def _near(value, thr, band):
    return thr is not None and abs(value - thr) <= band * thr


def compare(gpu_events, ref_trace, kind, band=TIE_BAND):
    """(ok, note): note is "equal", "tie at decision k: ..." or the mismatch."""
    prm = params.ihs_params(kind)
    gpu = [tuple(e) for e in gpu_events]
    ref = [tuple(e) for e in ref_trace]
    for k, (a, b) in enumerate(zip(gpu, ref)):
        if a[:3] == b[:3]:
            continue
        thr = _threshold(prm, b[0])
        if _near(b[3], thr, band):
            return True, "tie at decision %d: oracle %s (value %.6g, threshold %.6g), GPU %s" % (k, b, b[3], thr, a)
        if a[0] == "stop" and _near(a[3], 1.0, band):
            return True, "tie at decision %d: GPU stop (value %.6g), oracle %s" % (k, a[3], b)
        return False, "decision %d differs: GPU %s, oracle %s" % (k, a, b)
    if len(gpu) != len(ref):
        return False, "one run ended early: %d GPU decisions, %d oracle decisions" % (len(gpu), len(ref))
    return True, "equal"


def assert_same_schedule(gpu_events, ref_trace, kind, band=TIE_BAND):
    ok, note = compare(gpu_events, ref_trace, kind, band)
    assert ok, note
    if note != "equal":
        warnings.warn("schedule parity excused a tie: " + note)
    return note
