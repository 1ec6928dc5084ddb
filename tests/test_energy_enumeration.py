"""Host checks of the two pair enumerations of the from-scratch energy kernel
(its index arithmetic restated in Python; no GPU).

* Circulant order: a walker's team of T threads takes items k = (d - 1) N + i,
  d = 1 .. floor(N / 2), thread t starting at k = t and stepping by T with
  (i, d) advanced incrementally; for even N the offset N / 2 only from
  i < N / 2.  Every unordered pair {i, j} must appear exactly once, for odd and
  even N, N below and above T.
* Forward half stencil: particle i against its own cell (partners j > i) and
  the 13 neighbour offsets after (0, 0, 0) in (z, y, x) order, periodic in x
  and y (and z when the box is), clipped at the ends of a non-periodic z.  With
  at least three cells along every periodic axis, every pair of particles in
  the same or neighbouring cells must appear exactly once, and no other pair.

The GPU tests then check that the kernel's energies equal the oracle's and the
sweep's running totals; these checks cover many more sizes than a GPU run can.
"""
import itertools

import numpy as np
import pytest

TEAM = 4 * 256   # CTAs per walker x threads per CTA


def circulant_pairs(N, T=TEAM):
    seen = {}
    D = N >> 1
    if N < 2 or D == 0:
        return seen
    even = N % 2 == 0
    qT, rT = T // N, T % N
    for t in range(T):
        i, d = t % N, t // N + 1
        while d <= D:
            if not (even and d == D and i >= D):
                j = (i + d) % N
                key = (min(i, j), max(i, j))
                seen[key] = seen.get(key, 0) + 1
            i += rT
            d += qT
            if i >= N:
                i -= N
                d += 1
    return seen


@pytest.mark.parametrize("N", list(range(0, 40)) + [63, 64, 65, 511, 512, 513, 1023, 1024, 1025, 2048, 2049])
def test_circulant_lists_every_pair_once(N):
    seen = circulant_pairs(N)
    assert len(seen) == N * (N - 1) // 2
    assert all(c == 1 for c in seen.values())


def stencil_pairs(cells, nc, periodic_z, T=TEAM):
    """cells: [N, 3] cell coordinates of the particles; nc = (ncx, ncy, ncz)."""
    ncx, ncy, ncz = nc
    N = len(cells)
    members = {}
    for p, c in enumerate(map(tuple, cells)):
        members.setdefault(c, []).append(p)
    seen = {}
    qT, rT = T // 14, T % 14
    for t in range(T):
        i, o = t // 14, t % 14
        while i < N:
            cx, cy, cz = cells[i]
            idx = 13 + o
            nx, ny, nz = cx + idx % 3 - 1, cy + (idx // 3) % 3 - 1, cz + idx // 9 - 1
            nx %= ncx
            ny %= ncy
            ok = True
            if nz >= ncz:
                if periodic_z:
                    nz -= ncz
                else:
                    ok = False
            if ok:
                for j in members.get((nx, ny, nz), []):
                    if o == 0 and j <= i:
                        continue
                    key = (min(i, j), max(i, j))
                    seen[key] = seen.get(key, 0) + 1
            o += rT
            i += qT
            if o >= 14:
                o -= 14
                i += 1
    return seen


def neighbours(a, b, nc, periodic_z):
    for ax in range(3):
        d = abs(int(a[ax]) - int(b[ax]))
        if ax < 2 or periodic_z:
            d = min(d, nc[ax] - d)
        if d > 1:
            return False
    return True


@pytest.mark.parametrize("nc,periodic_z,N", [
    ((3, 3, 1), False, 60), ((3, 3, 3), True, 80), ((4, 3, 5), False, 150), ((7, 6, 4), False, 512),
    ((5, 5, 5), True, 300), ((3, 4, 3), True, 40), ((6, 3, 2), False, 1),
])
def test_half_stencil_lists_every_neighbour_pair_once(nc, periodic_z, N):
    rng = np.random.default_rng(sum(nc) * 1000 + N)
    cells = np.stack([rng.integers(0, n, N) for n in nc], axis=1)
    seen = stencil_pairs(cells, nc, periodic_z)
    assert all(c == 1 for c in seen.values())
    want = {(i, j) for i, j in itertools.combinations(range(N), 2)
            if neighbours(cells[i], cells[j], nc, periodic_z)}
    assert set(seen) == want


def test_two_cells_along_an_axis_would_double_count():
    """Why the kernel takes the circulant order below three cells: with two
    cells along x, offsets -1 and +1 name the same cell and a pair of
    particles in the two cells is listed twice."""
    cells = np.array([[0, 0, 0], [1, 0, 0]])
    seen = stencil_pairs(cells, (2, 3, 3), True)
    assert seen[(0, 1)] == 2
