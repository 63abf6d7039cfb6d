"""The oracle's operation count (the algorithmic flops of one ray interaction).

The counting build compiles the oracle's own sources as C++ with a double that counts the
operations it executes, so it must trace exactly what the oracle traces; the stored count that the
benchmark divides by must be the one a fresh count gives.
"""
import json

import numpy as np
import pytest


@pytest.fixture(scope="module")
def opc(oracle_mod):
    from oracle import opcount

    opcount.build()
    return opcount


def test_counting_build_traces_what_the_oracle_traces(oracle_mod, opc):
    o, xy, pmax = opc.ellipsoid_sample(stride=160)
    inter, cnt, rec = opc.count_trace(o.params, xy, pmax, records=True)
    ref = o.trace_rays(xy, pmax)
    assert inter == xy.shape[0] * (pmax + 1)
    assert np.array_equal(rec[..., oracle_mod.VALID], ref[..., oracle_mod.VALID])
    v = ref[..., oracle_mod.VALID] != 0
    for lo, hi in ((oracle_mod.S, oracle_mod.S + 3), (oracle_mod.F, oracle_mod.F + 6), (oracle_mod.PSI, oracle_mod.PSI + 1)):
        r, g = ref[..., lo:hi][v], rec[..., lo:hi][v]
        assert np.abs(g - r).max() <= 1e-12 * np.abs(r).max()
    assert all(c > 0 for c in cnt.values())


def test_counts_add_over_rays(oracle_mod, opc):
    o, xy, pmax = opc.ellipsoid_sample(stride=200)
    i1, c1, _ = opc.count_trace(o.params, xy, pmax)
    i2, c2, _ = opc.count_trace(o.params, np.concatenate([xy, xy]), pmax)
    assert i2 == 2 * i1 and all(c2[k] == 2 * c1[k] for k in c1)


def test_stored_count_is_current(oracle_mod, opc):
    with open(opc.GOLDEN) as f:
        stored = json.load(f)
    fresh = opc.measure()
    assert stored["interactions"] == fresh["interactions"]
    assert stored["counts"] == fresh["counts"]
