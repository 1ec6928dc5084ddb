"""One replica grid split over several processes, one GPU each.

The replicas of the (T, mu) grid only meet at the collective replica exchange
(Sec. II.A.2, Eq. Pacc; the paper gives each replica its own group of cores,
Sec. II.A.4).  Every process creates the same grid with the same walkers and
steps only its own contiguous range of walkers (regc_set_shard).  Before each
exchange attempt the processes all-gather their walkers' N (N_B) and exact
energies; each process writes the other ranges into its handle
(regc_set_walker_ne) and runs the same exchange on the same Philox stream, so
every process reaches the same state labels and configurations never move.
Each process's histograms count its own walkers' observations only; their sum
over the processes is the grid's (reduce_histograms).

The functions take an `engine` with the methods of `Regc` used here:
`shard` (w_begin, w_end), `walker_ne(b, e)`, `set_walker_ne(b, n, nb, efix)`
and `exchange()`; and a `gather(item)` that returns the list of every rank's
item in rank order (torch_gather for a torch.distributed process group).
Only argument marshalling and communication happen here; the exchange itself
runs in the library.
"""
from __future__ import annotations

import numpy as np


def shard_range(S: int, rank: int, world: int):
    """Walkers [w_begin, w_end) of process `rank` out of `world`: contiguous
    ranges, as even as possible, in rank order."""
    if world < 1 or not 0 <= rank < world or S < world:
        raise ValueError("need 0 <= rank < world <= S")
    return S * rank // world, S * (rank + 1) // world


def torch_gather(group=None):
    """A gather over a torch.distributed process group (gloo or NCCL): every
    rank's picklable item, in rank order."""
    import torch.distributed as dist

    def gather(item):
        out = [None] * dist.get_world_size(group)
        dist.all_gather_object(out, item, group=group)
        return out
    return gather


def exchange(engine, gather):
    """One replica-exchange attempt of a grid split over processes: the
    all-gather of (N, N_B, exact energy) by walker range, then the library's
    exchange on every process.  Returns the walkers written from other ranges."""
    b, e = engine.shard
    n, nb, efix = engine.walker_ne(b, e)
    written = 0
    for (rb, re_), (rn, rnb, refix) in gather(((b, e), (n, nb, efix))):
        if (rb, re_) == (b, e):
            continue
        if len(rn) != re_ - rb:
            raise ValueError("a rank sent %d walkers for the range [%d, %d)" % (len(rn), rb, re_))
        engine.set_walker_ne(rb, rn, rnb, refix)
        written += re_ - rb
    engine.exchange()
    return written


def run(engine, gather, n_sweeps: int, exchange_every: int = 10):
    """Alternate blocks of exchange_every sweeps of the process's walkers with
    a sharded exchange attempt (the schedule of Regc.run)."""
    done = 0
    while done < n_sweeps:
        k = min(exchange_every, n_sweeps - done) if exchange_every > 0 else n_sweeps - done
        engine.sweep(k)
        done += k
        if exchange_every > 0 and k == exchange_every:
            exchange(engine, gather)


def reduce_histograms(hists: dict, gather) -> dict:
    """The grid's histograms: every process's integer and float arrays summed
    over the processes (integers exactly)."""
    parts = gather({k: np.asarray(v) for k, v in hists.items()})
    return {k: np.sum([p[k] for p in parts], axis=0) for k in hists}
