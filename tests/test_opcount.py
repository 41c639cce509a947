"""The operation-counting build of the oracle computes the oracle's own values
and counts the simple stages exactly as their formulas read -- no GPU."""
import numpy as np

import synth
from oracle import opcount as OC
from oracle import oracle as O


def test_counting_build_is_the_oracle_and_counts_closed_forms():
    pr = synth.blast(16, seed=3)
    prm = O.params(gamma=5.0 / 3.0, cfl=0.4, limiter=0, emf=1)
    a, b = pr.state.copy(), pr.state.copy()
    counts, h = OC.count_step(a, pr.n, pr.g, pr.dx, prm)
    P = O.patch(b, pr.n, pr.g, pr.dx)
    O.fill_periodic(P)
    assert O.cfl_dt(P, prm) == h
    O.advance(P, prm, h, 0)
    assert np.array_equal(a, b)
    pu = OC.per_unit(counts, pr.n)
    # edge E^n and the arithmetic edge EMF: the mean of four values (3 adds, 1 multiply)
    for s in (3, 6):
        assert (pu[s]["add"], pu[s]["mul"], pu[s]["div"], pu[s]["sqrt"]) == (3.0, 1.0, 0.0, 0.0)
    # CT half step of a face: B - hdt/dx_b (E_c(+b) - E_c) + hdt/dx_c (E_b(+c) - E_b)
    assert (pu[4]["add"], pu[4]["mul"]) == (4.0, 2.0)
    # every HLLD face evaluation takes square roots (fast speeds, Alfven speeds)
    assert pu[5]["sqrt"] >= 4.0 and pu[5]["div"] >= 10.0
    assert OC.units(pr.n)[7] == 16 ** 3 and OC.units(pr.n)[1] == 20 ** 3
