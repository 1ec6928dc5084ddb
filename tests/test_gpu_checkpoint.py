"""Checkpoint and restore: a run continued from a checkpoint -- in the same
handle or a new one -- is bit-identical to the run that was never
interrupted, for plain, delayed-acceptance and cluster systems; a corrupted or
foreign checkpoint is refused and changes nothing."""
import numpy as np
import pytest

import workloads as W
from paper_1908_11118_gb300 import Regc
from paper_1908_11118_gb300 import build as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def state(g):
    pos, n, e, sow = g.get_walkers()
    h = g.histograms()
    return [pos, n, e, sow] + [h[k] for k in sorted(h)] + list(g.counters())


def same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def steps(g, k):
    for _ in range(k):
        g.sweep(5)
        g.exchange()


def make(kind):
    if kind == "cluster":
        p = W.cluster_in_gas(L=2, M=2, nmax_b=32, seed=2)
        pos, n = W.cluster_initial(p, 8, seed=1)
    else:
        p = W.fcc100_small(seed=3)
        pos, n = W.initial_walkers(p, 12, seed=2)
    g = Regc(p)
    g.set_walkers(pos, n)
    if kind == "delayed":
        g.surrogate_init(seed=4)
        g.set_mode(True)
    return p, g


@pytest.mark.parametrize("kind", ["plain", "delayed", "cluster"])
def test_resume_is_bit_identical(kind):
    p, g = make(kind)
    steps(g, 3)
    ck = g.checkpoint()
    steps(g, 4)
    want = state(g)
    # a new handle of the same problem continues the saved run exactly
    _, h = make(kind)
    steps(h, 1)                       # whatever it did before is overwritten
    h.restore(ck)
    steps(h, 4)
    same(state(h), want)
    # and so does the original handle, rolled back
    g.restore(ck)
    steps(g, 4)
    same(state(g), want)
    if kind == "delayed":
        assert np.array_equal(g.surrogate_get(), h.surrogate_get())


def test_bad_checkpoints_are_refused():
    p, g = make("plain")
    steps(g, 2)
    ck = bytearray(g.checkpoint())
    before = state(g)
    bad = bytearray(ck)
    bad[len(bad) // 2] ^= 0xFF            # payload corrupted: checksum
    with pytest.raises(Exception):
        g.restore(bytes(bad))
    with pytest.raises(Exception):
        g.restore(bytes(ck[:-8]))          # truncated
    other = Regc(W.fcc100_small(seed=99))  # another seed: another Philox key
    with pytest.raises(Exception):
        other.restore(bytes(ck))
    same(state(g), before)
