"""Pins of the counting-scalar operation counter (oracle/opcount.py) and of the stored counts the
benchmark's rooflines use (profiles/oracle_op_counts.json).

The counter is checked on expressions whose operation counts are known by construction, on the
selection rules (an unselected np.where branch costs nothing, the compared values of the decision
count when the selected value is used), on integer powers, and on consistency: the whole
right-hand side's reconstruction and Riemann work per face equals ten single-stencil WENO5-Z calls
and one single-face HLLC call.  The stored file must equal a fresh count."""
import json
import math
import os

import numpy as np
import pytest

from conftest import ROOT
from oracle import ns_fv as nf
from oracle import opcount as oc


def _count(expr, *vals):
    xs = [oc.counted_array(np.array([v])) for v in vals]
    out = oc._counting(lambda: expr(*xs))
    outs = out if isinstance(out, (list, tuple)) else [out]
    return oc.tally([np.asarray(o).reshape(-1)[0] for o in outs])


def test_counts_of_known_expressions():
    t = _count(lambda a, b, c: (2.0 * a - 7.0 * b + 11.0 * c) / 6.0, 1.0, 2.0, 3.0)["other"]
    assert (t["mul"], t["add"], t["div"]) == (3, 2, 1)
    t = _count(lambda a, b: -a * b + abs(a - b), 1.0, 3.0)["other"]
    assert (t["neg"], t["mul"], t["add"], t["misc"]) == (1, 1, 2, 1)
    t = _count(lambda a: np.sqrt(a * a + 1.0), 2.0)["other"]
    assert (t["mul"], t["add"], t["sqrt"]) == (1, 1, 1)


def test_shared_values_count_once():
    def f(a, b):
        s = a + b                 # one addition, used three times
        return s * s + s
    t = _count(f, 1.0, 2.0)["other"]
    assert (t["add"], t["mul"]) == (2, 1)


def test_integer_powers_and_pow():
    for n, muls in ((2, 1), (3, 2), (4, 2), (6, 3), (8, 3)):
        t = _count(lambda a: a ** n, 1.1)["other"]
        assert t["mul"] == muls and t["pow"] == 0, n
    t = _count(lambda a: a ** 0.7, 1.1)["other"]
    assert t["pow"] == 1 and t["mul"] == 0


def test_selections_count_the_taken_branch_and_the_decision():
    pnp = oc._NumpyProxy()             # what the oracle's modules see while counting

    def f(a, b):
        x = a * b                 # compared
        y = a + b                 # compared
        return pnp.where(x > y, x * 2.0, y / 3.0)
    t = _count(f, 3.0, 4.0)["other"]          # x = 12 > y = 7: the multiplication branch
    assert (t["mul"], t["add"], t["div"]) == (2, 1, 0)
    t = _count(f, 0.5, 0.5)["other"]          # x = 0.25 < y = 1: the division branch
    assert (t["mul"], t["add"], t["div"]) == (1, 1, 1)

    def nested(a, b):
        # a branch test that is never reached costs nothing: the second test applies only where
        # the first failed
        first = a - b
        second = a * b
        return pnp.where(first > 0.0, a, pnp.where(second > 1.0, b, a + 1.0))
    t = _count(nested, 2.0, 1.0)["other"]     # first > 0: only the first test is needed
    assert (t["add"], t["mul"]) == (1, 0)
    t = _count(nested, 1.0, 2.0)["other"]     # first < 0, second = 2 > 1: both tests
    assert (t["add"], t["mul"]) == (1, 1)


def test_rhs_counts_equal_single_calls():
    """Per face of a whole right-hand side: ten WENO5-Z reconstructions and one HLLC call, as the
    same functions count on one stencil and one face (no work lost or shared between faces)."""
    from paper_2406_19494_gb300 import workloads as wl
    P = ("periodic", "periodic")
    c = wl.random_box(3, (6, 5, 4), bc=(P, P, P), lo=(0, 0, 0), hi=(2 * math.pi,) * 3, visc="none",
                      weno="z")
    per = oc.count_rhs(c)
    one = _count(lambda *q: nf.weno5(*q, "z", 1e-40), 1.0, 1.1, 1.3, 1.2, 1.25)["recon"]
    for k in oc.CLASSES:
        assert per["recon"][k] == pytest.approx(10 * one[k]), k
    WL = (1.0, 0.3, 0.1, -0.2, 1.0)
    WR = (1.05, 0.25, 0.12, -0.18, 0.98)
    h = _count(lambda *w: nf.hllc_flux(list(w[:5]), list(w[5:]), 0, 1.4), *(WL + WR))["riemann"]
    assert sum(per["riemann"][k] for k in ("add", "mul", "div", "sqrt")) == pytest.approx(
        h["add"] + h["mul"] + h["div"] + h["sqrt"])
    assert per["div"]["add"] + per["div"]["div"] == 15          # F+ - F-, / dx, accumulate: 5 x 3


@pytest.mark.slow
def test_stored_counts_are_current():
    path = os.path.join(ROOT, "profiles", "oracle_op_counts.json")
    stored = json.load(open(path))["workloads"]
    fresh = oc.counts_for(oc.workloads_to_count()["weno5z_power"])
    for unit in ("face", "cell_axis", "cell_update", "recon", "riemann", "visc", "prim", "stage_per_step"):
        for k, v in fresh[unit].items():
            assert stored["weno5z_power"][unit][k] == pytest.approx(v, rel=1e-12), (unit, k)
