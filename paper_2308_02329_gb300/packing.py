"""Independent small graphs packed into one context as the blocks of a block-diagonal
coupling matrix, so that the 128 lanes of the small-N tensor-core tile (one lane per
spin) carry several graphs at once.

A block-diagonal J couples no spin of one graph to another, so every graph of a pack
follows its own equations of motion; the per-spin coupling weights
(chym_set_coupling_weights) give each graph its own eps_i = eps_hat / lambda_max(J_i),
so all graphs share the pump grid h = h_th (1 + dh) with h_th = 1 - eps_hat.  A run of
the packed context is one run of every member graph (same pump, same seed; the noise
counters of a member use its spins' indices in the packed J, so members draw
independent noise).  Energies and ground-state hits are read per member with
chym_energy_segments.
"""
from dataclasses import dataclass, field

import numpy as np

CAPACITY = 128  # spins of one tensor-core tile


@dataclass
class Pack:
    members: list                 # indices into the graph list, in block order
    seg_begin: np.ndarray         # block b holds spins [seg_begin[b], seg_begin[b+1])
    J: np.ndarray = field(repr=False, default=None)

    @property
    def N(self):
        return int(self.seg_begin[-1])


def plan(sizes, capacity=CAPACITY):
    """First-fit decreasing packing of graphs of the given sizes into bins of at most
    `capacity` spins (graphs larger than `capacity` get a bin of their own).  Returns
    lists of graph indices, each list in block order (larger graphs first, ties by index)."""
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    bins, room = [], []
    for i in order:
        n = int(sizes[i])
        for b in range(len(bins)):
            if n <= room[b]:
                bins[b].append(i)
                room[b] -= n
                break
        else:
            bins.append([i])
            room.append(capacity - n)
    return bins


def build(Js, members):
    """The block-diagonal coupling matrix of the member graphs (in order) and the
    segment table of their spins."""
    sizes = [np.asarray(Js[i]).shape[0] for i in members]
    seg = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    J = np.zeros((int(seg[-1]), int(seg[-1])), dtype=np.float64)
    for b, i in enumerate(members):
        J[seg[b]:seg[b + 1], seg[b]:seg[b + 1]] = Js[i]
    return Pack(list(members), seg, J)


def spin_weights(pack, per_graph):
    """Per-spin weights of a pack from one value per member graph (in block order)."""
    sizes = np.diff(pack.seg_begin)
    return np.repeat(np.asarray(per_graph, dtype=np.float64), sizes)
