"""The oracle's pins catch plausible mistakes (CPU only).

Each mutant is the oracle rebuilt with one planted mistake (ORC_MUTANT in
oracle/pic_oracle.c): a wrong shape piece, a missing staggering offset, a
dropped Boris half kick, an Esirkepov window off by one node, 1/2 for 1/3 in
Esirkepov's W, a flipped curl sign, a flipped current sign, momentum used as
velocity, an energy-conserving gather that keeps order p for one component,
a Vay pusher without its explicit magnetic half, CKC with the wrong
transverse weights, a field energy without the cell volume, a kinetic
energy of gamma m instead of (gamma - 1) m, a charge density without 1/dV, a
z filter whose compensation pass has the wrong sign, a deposit that takes the
previous particle's weight (invisible with equal weights).  Every mutant must
fail at least one pin.
"""
import pytest

import pins_lib
from oracle import Oracle

MUTANTS = {
    1: "cubic shape inner piece",
    2: "Ex gathered without staggering",
    3: "Boris second half kick dropped",
    4: "Esirkepov window start off by one",
    5: "Esirkepov 1/2 for 1/3",
    6: "curl sign in the B update",
    7: "current sign in the E update",
    8: "momentum used as velocity",
    9: "energy-conserving gather keeps order p for E_y",
    10: "Vay without the explicit half of v x B",
    11: "CKC with box-average weights",
    12: "field energy without the cell volume",
    13: "kinetic energy gamma m in place of (gamma - 1) m",
    14: "charge density without 1/dV",
    15: "z filter compensation with the wrong sign",
    16: "deposit with the previous particle's weight",
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS), ids=lambda k: MUTANTS[k])
def test_mutant_is_caught(mutant):
    O = Oracle(mutant=mutant)
    failed = []
    for pin in pins_lib.ALL_PINS:
        try:
            pin(O)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"no pin catches mutant {mutant} ({MUTANTS[mutant]})"
