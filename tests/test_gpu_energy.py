"""From-scratch walker energies on the GPU (the kernel behind
regc_set_walkers, regc_check_energy and every MD segment) against the FP64
oracle, through both of its pair enumerations:

* all pairs in circulant order (a periodic box with fewer than three cells
  along an axis: the 6.25 x 6.25 fcc(100) box), for odd and even N from 0 to
  Nmax, where the offset N / 2 of an even N must be counted once;
* the forward half of the 27-cell stencil (the 1024-replica fcc(111)
  workload's box), up to N = Nmax = 512, and a walker whose particles crowd one
  cell past its capacity (the kernel falls back to all pairs).

After sweeps the running energy of every walker equals the from-scratch one
exactly (regc_check_energy returns 0), which holds only if both enumerations
list each pair within rc once with the sweep's rounded displacement.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from paper_1908_11118_gb300 import Regc
from paper_1908_11118_gb300 import build as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    O.build()


def energies_match(p, pos, n):
    g = Regc(p)
    g.set_walkers(pos, n)
    e = g.get_walkers()[2]
    o = O.Oracle(p, pos=pos, n=n)
    np.testing.assert_allclose(e, o.energy, rtol=1e-5, atol=1e-4)
    return g


def test_all_pairs_path_odd_and_even_n():
    p = W.fcc100_small(seed=1)                  # 6.25 x 6.25 box: two cells along x and y
    n_init = [0, 1, 2, 3, 4, 5, 6, 7, 8, 15, 16, 17, 30, 31, 32, 32]
    pos, n = W.initial_walkers(p, n_init, seed=2)
    assert list(n) == n_init
    g = energies_match(p, pos, n)
    g.run(20, exchange_every=10)
    assert g.check_energy() == 0.0


def test_cell_path_up_to_nmax():
    p = W.fcc111_paper_scale(L=2, M=2, seed=3)
    pos, n = W.lattice_walkers(p, [1, 255, 511, 512], seed=4)
    g = energies_match(p, pos, n)
    g.run(20, exchange_every=10)
    assert g.check_energy() == 0.0


def test_crowded_cell_falls_back_to_all_pairs():
    p = W.fcc111_paper_scale(L=2, M=2, seed=5)
    # cells of the box: 7 x 6 x 4 (2.68 x 2.71 x 3.0), capacity 43 particles
    ncx, ncy = int(p.Lx // 2.5), int(p.Ly // 2.5)
    hx, hy = p.Lx / ncx, p.Ly / ncy
    g1 = np.arange(4) * 0.62
    cube = np.stack(np.meshgrid(g1, g1, g1, indexing="ij"), -1).reshape(-1, 3)
    cube = cube + np.array([2 * hx + 0.4, 2 * hy + 0.4, p.z_lo + 6.4])   # 64 particles inside cell (2, 2, 2)
    pos, n = W.lattice_walkers(p, [0, 200, 64, 300], seed=6)
    pos[0, :64] = W.f32(cube)
    n[0] = 64
    pos[2, :64] = W.f32(cube + np.array([0.0, 0.0, -3.0]))               # the same in cell (2, 2, 1)
    energies_match(p, pos, n)


def test_page_locked_walker_buffers_are_read_and_written_in_place():
    """A page-locked position buffer is read by the repacking kernel itself
    and a page-locked output buffer written by the unpacking kernel (no staged
    copy): the walkers, energies and the run that follows are those of the
    copied path, and entries beyond N of the output are left as they were."""
    torch = pytest.importorskip("torch")
    p = W.fcc111_paper_scale(L=4, M=4, nmax=64)
    rng = np.random.default_rng(3)
    pos, n = W.lattice_walkers(p, rng.integers(0, 33, p.S), seed=3)
    pinned_in = torch.empty(pos.shape, dtype=torch.float32, pin_memory=True).numpy()
    pinned_in[:] = pos
    a, b = Regc(p), Regc(p)
    a.set_walkers(pos.astype(np.float32), n)
    b.set_walkers(pinned_in, n)
    for h in (a, b):
        h.sweep(4)
        h.exchange()
    pa, na, ea, sa = a.get_walkers()
    out = (torch.full(pos.shape, -7.0, dtype=torch.float32, pin_memory=True).numpy(),
           torch.empty(p.S, dtype=torch.int32, pin_memory=True).numpy(),
           torch.empty(p.S, dtype=torch.float64, pin_memory=True).numpy(),
           torch.empty(p.S, dtype=torch.int32, pin_memory=True).numpy())
    pb, nb_, eb, sb = b.get_walkers(out=out)
    assert np.array_equal(na, nb_) and np.array_equal(ea, eb) and np.array_equal(sa, sb)
    for w in range(p.S):
        assert np.array_equal(pa[w, :na[w]], pb[w, :nb_[w]])
        assert np.all(pb[w, nb_[w]:] == -7.0)
    assert b.check_energy() == 0.0
