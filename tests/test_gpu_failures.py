"""Failure detection of the library, driven from the host with inputs that
make the device code take its own error paths (no GPU fault, trap or hang).

* Cell-list capacity: a walker whose particles crowd one cell beyond the
  cell's fixed capacity (all pairs still outside the hard-core guard, so the
  configuration is legal).  Uploading it works -- the from-scratch energy
  falls back to all pairs -- but the sweep's cell build cannot hold it: the
  handle's status becomes REGC_ECAPACITY, sticky on every later call, while a
  second handle on the same device keeps working and matches the oracle.
* Numeric: an MD segment with a time step far too long for the forces drives
  pairs inside the hard-core guard; the energy recompute at the end of the
  segment reports it as REGC_ENUMERIC (positions are kept inside the box by
  construction, so nothing is read or written out of range).
* Timeout: the sweep's bounded mbarrier wait on the bulk copy of a walker's
  positions is made to run out by the test hook regc_test_expire_waits (the
  next sweep's walkers issue no copy, so the barrier phase they wait for never
  completes and each wait ends by its own budget of about 1 s of clock
  cycles).  The handle reports REGC_ETIMEOUT, sticky; the context stays
  usable and a fresh handle matches the oracle.
"""
import time

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from paper_1908_11118_gb300 import Regc, RegcError
from paper_1908_11118_gb300 import build as B

pytestmark = pytest.mark.gpu

ETIMEOUT, ECAPACITY, ENUMERIC = -4, -5, -6


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    O.build()


def crowded_walkers(p, n_crowd, spacing=0.6):
    """Walker 0: n_crowd particles on a lattice of the given spacing (0.55 in
    z) inside the first cell of the sweep's cell grid (cells of the fcc(111)
    workload are about 2.68 x 2.71 x 3.0), at least 1.0 above the top surface
    layer; the other walkers a few particles."""
    pos, n = W.initial_walkers(p, [0] + [5] * (p.S - 1), seed=3)
    g = np.arange(4) * spacing + 0.15
    gz = np.arange(4) * 0.55 + 1.0
    sites = np.array([(x, y, p.z_lo + z) for z in gz for y in g for x in g])
    pos[0, :n_crowd] = W.f32(sites[:n_crowd])
    n[0] = n_crowd
    return pos, n


def test_cell_capacity_overflow_is_sticky():
    p = W.fcc111_paper_scale(L=2, M=2, nmax=64)
    # the sweep's cells hold ceil(1.6 V_cell) + 8 = 43 particles here
    pos, n = crowded_walkers(p, 60)
    g = Regc(p)
    g.set_walkers(pos, n)                       # legal: every pair beyond the guard
    assert np.isfinite(g.get_walkers()[2]).all()
    g.sweep(1)
    with pytest.raises(RegcError) as err:
        g.get_walkers()
    assert err.value.status == ECAPACITY
    for call in (lambda: g.sweep(1), g.exchange, g.histograms, g.check_energy):
        with pytest.raises(RegcError) as err:
            call()
        assert err.value.status == ECAPACITY
    g.close()
    # the device and a fresh handle are unaffected: a lock-step check against the oracle
    pos, n = crowded_walkers(p, 20)              # within capacity
    h = Regc(p)
    h.set_walkers(pos, n)
    tr = h.sweep_traced(2)
    o = O.Oracle(p, pos=pos, n=n)
    to = o.sweeps(2, trace=True)
    assert np.array_equal(tr["accepted"], to["accepted"]) and np.array_equal(tr["index"], to["index"])
    assert h.check_energy() == 0.0
    h.close()


def test_md_with_a_runaway_time_step_reports_numeric():
    p = W.fcc100_small(L=8, M=8)                  # cells hold nmax: no capacity error possible
    pos, n = W.initial_walkers(p, [p.nmax] * p.S, seed=2, min_dist=0.9)
    g = Regc(p)
    g.set_walkers(pos, n)
    g.md(20, 0.02, 0.5)                           # a sane step first: no error
    g.check_energy()
    with pytest.raises(RegcError) as err:
        g.md(20, 0.8, 0.5)                        # forty times too long
        g.get_walkers()
    assert err.value.status == ENUMERIC
    with pytest.raises(RegcError) as err:
        g.sweep(1)
    assert err.value.status == ENUMERIC
    g.close()


def test_expired_wait_reports_timeout_and_the_context_stays_usable():
    p = W.fcc100_small()
    pos, n = W.initial_walkers(p, [6] * p.S, seed=4)
    g = Regc(p)
    g.set_walkers(pos, n)
    g.test_expire_waits()
    t0 = time.perf_counter()
    g.sweep(1)
    with pytest.raises(RegcError) as err:
        g.histograms()
    waited = time.perf_counter() - t0
    assert err.value.status == ETIMEOUT
    assert 0.3 < waited < 30.0, waited             # the waits ended by their own budget
    for call in (lambda: g.sweep(1), g.exchange, g.check_energy):
        with pytest.raises(RegcError) as err:
            call()
        assert err.value.status == ETIMEOUT
    g.close()
    # the hook is one-shot and per handle: a fresh handle samples as the oracle does
    h = Regc(p)
    h.set_walkers(pos, n)
    tr = h.sweep_traced(2)
    o = O.Oracle(p, pos=pos, n=n)
    to = o.sweeps(2, trace=True)
    assert np.array_equal(tr["accepted"], to["accepted"]) and np.array_equal(tr["index"], to["index"])
    h.sweep(3)
    assert h.check_energy() == 0.0
    h.close()
