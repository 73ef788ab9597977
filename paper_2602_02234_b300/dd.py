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
The halo exchange and the reverse force exchange are point to point with the
two slab neighbours (torch.distributed isend/irecv, gloo or NCCL): since the
halo is no wider than a slab, every ghost comes from one of them.  The total
energy is the one global reduction.
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

    def peers(self):
        """The slab neighbours (rank - 1 and rank + 1, periodic): with a halo
        no wider than a slab, every ghost lives in one of them."""
        if self.n_ranks == 1:
            return []
        return sorted({(self.rank - 1) % self.n_ranks, (self.rank + 1) % self.n_ranks})

    def gather_local(self, dist, ids, coords, types):
        """Owned atoms (global ids, positions, species) in; owned + ghosts out.

        Each rank sends its slab neighbours the owned atoms within the halo of
        their slabs (point to point) and receives theirs.  Returns
        (local_ids, local_coords, local_types, n_owned): the owned atoms
        first, in the given order, then the ghosts by increasing global id;
        `ghost_from` keeps the rank each ghost came from."""
        ids = np.asarray(ids, dtype=np.int64)
        coords = np.asarray(coords, dtype=np.float64)
        types = np.asarray(types, dtype=np.int32)
        out = {}
        for q in self.peers():
            near = slab_distance(coords, self.box, q, self.n_ranks, self.axis) < self.halo
            out[q] = np.concatenate([ids[near, None].astype(np.float64), coords[near],
                                     types[near, None].astype(np.float64)], axis=1)
        got = _exchange(dist, out, 5) if out and dist is not None else {}
        g_ids, g_x, g_t, g_src = [], [], [], []
        for q, rows in sorted(got.items()):
            g_ids.append(rows[:, 0].astype(np.int64))
            g_x.append(rows[:, 1:4])
            g_t.append(rows[:, 4].astype(np.int32))
            g_src.append(np.full(len(rows), q, np.int64))
        if g_ids:
            gi = np.concatenate(g_ids)
            order = np.argsort(gi, kind="stable")
            gi, gx = gi[order], np.concatenate(g_x)[order]
            gt, gs = np.concatenate(g_t)[order], np.concatenate(g_src)[order]
        else:
            gi, gx, gt, gs = np.zeros(0, np.int64), np.zeros((0, 3)), np.zeros(0, np.int32), np.zeros(0, np.int64)
        self.ghost_from = gs
        return (np.concatenate([ids, gi]), np.concatenate([coords, gx]),
                np.concatenate([types, gt]), len(ids))

    def reduce_forces(self, dist, local_ids, local_forces, n_owned):
        """Partial forces on owned + ghost atoms in; total forces on the owned
        atoms out: each ghost's partial force goes back to the neighbour it
        came from (point to point), which adds it to its owned atom."""
        local_ids = np.asarray(local_ids, dtype=np.int64)
        local_forces = np.asarray(local_forces, dtype=np.float64)
        F = np.array(local_forces[:n_owned], dtype=np.float64)
        if dist is None or self.n_ranks == 1:
            return F
        gids, gF = local_ids[n_owned:], local_forces[n_owned:]
        out = {}
        for q in self.peers():
            sel = self.ghost_from == q
            out[q] = np.concatenate([gids[sel, None].astype(np.float64), gF[sel]], axis=1)
        got = _exchange(dist, out, 4)
        pos = {int(g): k for k, g in enumerate(local_ids[:n_owned])}
        for q in sorted(got):                       # fixed order: by rank, then as sent
            for row in got[q]:
                F[pos[int(row[0])]] += row[1:4]
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


def _exchange(dist, out, width):
    """Point-to-point exchange of float64 row blocks with the peers in `out`
    ({rank: (k, width) array}): sizes first, then the rows, with non-blocking
    sends and receives so that no ordering between the ranks is needed.
    Returns {rank: the rows that rank sent here}."""
    import torch
    peers = sorted(out)
    n_out = {q: torch.tensor([len(out[q])], dtype=torch.int64) for q in peers}
    n_in = {q: torch.zeros(1, dtype=torch.int64) for q in peers}
    reqs = [dist.isend(n_out[q], q) for q in peers] + [dist.irecv(n_in[q], q) for q in peers]
    for r in reqs:
        r.wait()
    t_out = {q: torch.from_numpy(np.ascontiguousarray(out[q], dtype=np.float64).reshape(-1)) for q in peers}
    t_in = {q: torch.zeros(int(n_in[q].item()) * width, dtype=torch.float64) for q in peers}
    reqs = [dist.isend(t_out[q], q) for q in peers if t_out[q].numel()]
    reqs += [dist.irecv(t_in[q], q) for q in peers if t_in[q].numel()]
    for r in reqs:
        r.wait()
    return {q: t_in[q].numpy().reshape(-1, width) for q in peers}

