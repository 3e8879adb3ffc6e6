"""Values printed in the paper (fixtures under tests/golden/, each citing its
source) against the oracle and the workload definitions."""
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2410_11129_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name, sep=None):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [[c.strip() for c in (l.split(sep) if sep else l.split())]
                for l in fh if l.strip() and not l.startswith("#")]


def test_weights_match_eq17(orc):
    w = orc.tables()[0]
    for a0, a1, num, den in _rows("eq17_weights.txt"):
        for a in range(int(a0), int(a1) + 1):
            assert w[a] == float(Fraction(int(num), int(den)))


def _table2():
    return {case: (float(r23), float(r13))
            for case, r23, r13 in _rows("table2_surface_tension_ratios.txt", "|")}


def test_table2_transcription():
    assert _table2() == W.TABLE2


@pytest.mark.parametrize("case", list(W.TABLE2))
def test_table2_topologies_and_spreading_signs(orc, case):
    """Sec. 3.8 defines each topology by inequalities of the ratios; with
    gamma_i of Eq. 27 each one is the sign of one spreading coefficient
    (S_i = -gamma_i > 0: phase i spreads): complete engulfing-type 1 is
    gamma_2 < 0, type 2 gamma_1 < 0, non-engulfing gamma_3 < 0, partial
    engulfing all gamma_i > 0. A transposed index in Eq. 27 fails here."""
    r23, r13 = _table2()[case]
    cond = {"partial engulfing": abs(r13 - r23) < 1 and r13 + r23 > 1,
            "non-engulfing": r13 + r23 < 1,
            "complete engulfing-type 1": r13 > r23 + 1,
            "complete engulfing-type 2": r23 > r13 + 1}
    assert cond[case] and sum(cond.values()) == 1
    cfg = W.topology(case, 0.005, nx=32, ny=16, r1=3.0, r2=6.0)
    g = np.array([orc.derive(cfg).gamma[i] for i in range(3)])
    negative = {"partial engulfing": None, "non-engulfing": 2,
                "complete engulfing-type 1": 1, "complete engulfing-type 2": 0}[case]
    for i in range(3):
        assert (g[i] < 0) == (i == negative), (case, g)
