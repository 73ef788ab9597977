"""Ghost-atom domain decomposition for the attention family (host side).

The paper runs its deep potential on one rank and gathers every domain's atoms
there, and names domain-decomposed inference as future work (Sec. III, Sec.
V-B, Sec. VII).  The attention family is atom-local: an atom's energy depends
on its neighbours within rc only.  So a system splits into slabs along one axis,
one per rank; a rank

1. owns the atoms whose wrapped coordinate lies in its slab;
2. receives as ghosts every other atom within rc (along the axis, periodic) of
   its slab: every neighbour of an owned atom is then present exactly once, so
   each owned atom's environment, energy and pair gradients equal the whole
   system's;
3. evaluates its owned atoms as centres over owned + ghost atoms, giving
   partial forces on owned and ghost atoms: F_i = sum_p g_ip over its own slots
   minus g_kp for every slot p of a centre k whose neighbour is i;
4. sends each ghost's partial force back to the ghost's owner (reverse
   communication) and sums what it receives.

E is the sum over ranks of the owned energies.  One halo exchange of
positions and one reverse exchange of forces per evaluation.

Layer-coupled models (the attention family with message passing, the graph
family) reach L neighbour hops: an owned atom's energy depends on atoms up to
L x rc away, which is why the paper broadens the ghost area to L x rc (Sec.
III).  With `hops = L` the halo is L x rc; every atom then evaluates as a
centre (ghosts included, since their features feed the owned atoms') and the
energy counted is the owned atoms' only (seed 1 for owned, 0 for ghosts), so
the adjoint gives each local atom its partial force; the reverse exchange is
the same.  A ghost within L - 1 hops of an owned atom keeps its whole
neighbour list inside the halo; the outermost ghosts' lists are cut, but
only their species reach the owned atoms.

The evaluation of a subdomain is a callback (on a GPU, a context over owned +
ghost atoms whose centres mask, dp_set_centres, marks the owned ones, or for
a layer-coupled model whose energy seed, dp_set_energy_seed, does; in the
CPU tests the FP64 oracle), so this module holds the partitioning and the
communication only.
Exchanges use torch.distributed object collectives (gloo or NCCL); the design
sends to every rank for simplicity, where a production layout would talk to
the two slab neighbours only.
"""
from __future__ import annotations

import numpy as np


def slab_owner(coords, box, n_ranks, axis=0):
    """Rank owning each atom: slab floor(wrapped x_axis / (L / n_ranks))."""
    L = float(box[axis])
    w = np.mod(np.asarray(coords, dtype=np.float64)[:, axis], L)
    return np.minimum((w * n_ranks / L).astype(np.int64), n_ranks - 1)


def slab_distance(coords, box, rank, n_ranks, axis=0):
    """Periodic distance along the axis from each atom to slab `rank` (0 inside)."""
    L = float(box[axis])
    lo, hi = rank * L / n_ranks, (rank + 1) * L / n_ranks
    w = np.mod(np.asarray(coords, dtype=np.float64)[:, axis], L)
    inside = (w >= lo) & (w < hi)
    return np.where(inside, 0.0, np.minimum(np.mod(lo - w, L), np.mod(w - hi, L)))


class SlabDecomposition:
    """Slabs along `axis`; ghost halo of width hops x rc."""

    def __init__(self, box, n_ranks, rank, rc, axis=0, hops=1):
        box = np.asarray(box, dtype=np.float64)
        halo = hops * rc
        if n_ranks > 1 and box[axis] / n_ranks < halo:
            # a ghost two slabs away would need a second hop of the exchange
            raise ValueError("slabs must be at least as wide as the halo (hops x rc)")
        self.box, self.n_ranks, self.rank, self.rc, self.axis = box, n_ranks, rank, rc, axis
        self.halo = halo

    def gather_local(self, dist, ids, coords, types):
        """Owned atoms (global ids, positions, species) in; owned + ghosts out.

        Returns (local_ids, local_coords, local_types, n_owned): the owned atoms
        first, in the given order, then the ghosts by increasing global id."""
        ids = np.asarray(ids, dtype=np.int64)
        coords = np.asarray(coords, dtype=np.float64)
        types = np.asarray(types, dtype=np.int32)
        mine = (ids, coords, types)
        parts = [None] * self.n_ranks
        if dist is not None and self.n_ranks > 1:
            dist.all_gather_object(parts, mine)
        else:
            parts = [mine]
        g_ids, g_x, g_t = [], [], []
        for r, (pi, px, pt) in enumerate(parts):
            if r == self.rank:
                continue
            near = slab_distance(px, self.box, self.rank, self.n_ranks, self.axis) < self.halo
            g_ids.append(pi[near])
            g_x.append(px[near])
            g_t.append(pt[near])
        if g_ids:
            gi = np.concatenate(g_ids)
            order = np.argsort(gi, kind="stable")
            gi, gx, gt = gi[order], np.concatenate(g_x)[order], np.concatenate(g_t)[order]
        else:
            gi, gx, gt = np.zeros(0, np.int64), np.zeros((0, 3)), np.zeros(0, np.int32)
        return (np.concatenate([ids, gi]), np.concatenate([coords, gx]),
                np.concatenate([types, gt]), len(ids))

    def reduce_forces(self, dist, local_ids, local_forces, n_owned):
        """Partial forces on owned + ghost atoms in; total forces on the owned
        atoms out (the ghosts' partial forces go back to their owners)."""
        local_ids = np.asarray(local_ids, dtype=np.int64)
        F = np.array(local_forces[:n_owned], dtype=np.float64)
        sent = (local_ids[n_owned:], np.asarray(local_forces[n_owned:], dtype=np.float64))
        parts = [None] * self.n_ranks
        if dist is not None and self.n_ranks > 1:
            dist.all_gather_object(parts, sent)
        else:
            return F
        pos = {int(g): k for k, g in enumerate(local_ids[:n_owned])}
        for r, (gi, gf) in enumerate(parts):
            if r == self.rank:
                continue
            for g, f in zip(gi, gf):
                k = pos.get(int(g))
                if k is not None:
                    F[k] += f
        return F

    def total(self, dist, value):
        """Sum of a per-rank scalar over the ranks (FP64)."""
        if dist is None or self.n_ranks == 1:
            return float(value)
        parts = [None] * self.n_ranks
        dist.all_gather_object(parts, float(value))
        return float(sum(parts[r] for r in range(self.n_ranks)))   # fixed order


def local_system(coords, types, box, rank, n_ranks, rc, hops=1, axis=0):
    """Rank `rank`'s local atoms computed from the whole system in one process
    (what gather_local returns after its exchange): (global ids, positions,
    species, n_owned), owned atoms first by increasing id, then the ghosts
    within hops x rc of the slab by increasing id.  Neighbours at exactly
    equal distances are ranked by atom index; an evaluator that must rank
    them as the whole system does numbers the local atoms by global id."""
    coords = np.asarray(coords, dtype=np.float64)
    types = np.asarray(types, dtype=np.int32)
    owner = slab_owner(coords, box, n_ranks, axis)
    own = np.nonzero(owner == rank)[0]
    near = slab_distance(coords, box, rank, n_ranks, axis) < hops * rc
    ghost = np.nonzero(near & (owner != rank))[0]
    ids = np.concatenate([own, ghost])
    return ids, coords[ids], types[ids], len(own)


def partial_forces(n_local, centres, pair_j, pair_g):
    """Forces on local atoms from the pair gradients of the given centres:
    F_i += sum_p g_ip for centre i, F_j -= g_ip for its neighbour j."""
    F = np.zeros((n_local, 3))
    for q, i in enumerate(centres):
        for p in range(pair_j.shape[1]):
            j = int(pair_j[q, p])
            if j < 0:
                continue
            F[i] += pair_g[q, p]
            F[j] -= pair_g[q, p]
    return F
