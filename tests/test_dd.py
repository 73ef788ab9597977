"""Ghost-atom domain decomposition on CPU ranks (gloo), with the FP64 oracle
evaluating each subdomain: energies and forces must equal the whole system's.
No GPU is involved (one-GPU machines cannot run a multi-GPU decomposition)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2602_02234_b300 import dd
from synth import configs as C, normal_blob, protein_in_water

MODEL = C.AttnModel(n_species=5, e1=8, e2=12, m1=16, m2=4, n_layers=2, hidden=16, heads=2,
                    f1=20, f2=16, f3=12, nmax=120, rc=6.0, rs=0.5)


def _system():
    return protein_in_water(900, 90, (26.0, 19.0, 19.0), 21)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = _system()
        w = normal_blob(oracle.af_weight_count(MODEL), 5, 0.1)
        owner = dd.slab_owner(s.coords, s.box, world)
        mine = np.nonzero(owner == rank)[0]
        dec = dd.SlabDecomposition(s.box, world, rank, MODEL.rc)
        ids, x, t, n_own = dec.gather_local(dist, mine, s.coords[mine], s.types[mine])
        res = oracle.af_atoms(MODEL, w, t, x, s.box, np.arange(n_own), nthreads=1)
        Fl = dd.partial_forces(len(ids), np.arange(n_own), res["pair_j"], res["pair_g"])
        F = dec.reduce_forces(dist, ids, Fl, n_own)
        E = dec.total(dist, res["atom_e"].sum())
        out[rank] = (mine, F, E, len(ids) - n_own)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_decomposition_reproduces_the_whole_system(world):
    s = _system()
    w = normal_blob(oracle.af_weight_count(MODEL), 5, 0.1)
    E, ae, F, V = oracle.af_compute(MODEL, w, s.types, s.coords, s.box)
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    rms = np.sqrt(np.mean(F ** 2))
    seen = np.zeros(s.n, bool)
    for r in range(world):
        mine, Fr, Er, n_ghost = res[r]
        assert n_ghost > 0
        assert not seen[mine].any()
        seen[mine] = True
        assert np.max(np.abs(Fr - F[mine])) <= 1e-11 * rms
        assert Er == pytest.approx(E, rel=1e-12)
    assert seen.all()                                    # every atom owned once


def test_halo_contains_every_neighbour_of_owned_atoms():
    s = _system()
    world = 3
    owner = dd.slab_owner(s.coords, s.box, world)
    cnt, nj, _, _ = oracle.neighbours(s.coords, s.box, MODEL.rc, 4096)
    for rank in range(world):
        near = dd.slab_distance(s.coords, s.box, rank, world) < MODEL.rc
        for i in np.nonzero(owner == rank)[0]:
            for j in nj[i, :cnt[i]]:
                assert owner[j] == rank or near[j]


def test_slabs_narrower_than_the_cutoff_are_refused():
    with pytest.raises(ValueError):
        dd.SlabDecomposition(np.array([10.0, 20.0, 20.0]), 2, 0, 6.0)


# ------------------------------------------------------------- layer-coupled models
from dataclasses import replace  # noqa: E402

MP_MODEL = replace(MODEL, message_passing=1)          # 2 layers: 2 hops
GF_MODEL = C.GraphModel(n_species=5, node=16, edge=8, n_layers=2, f1=20, f2=16, f3=12,
                        nmax=120, na=12)


def _layered_system():
    return protein_in_water(1290, 90, (37.0, 19.0, 19.0), 23)


def _layered(kind):
    m = MP_MODEL if kind == "mp" else GF_MODEL
    n = oracle.af_weight_count(m) if kind == "mp" else oracle.gf_weight_count(m)
    return m, normal_blob(n, 5, 0.1)


def _rank_layered(rank, world, port, kind, hops, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = _layered_system()
        m, w = _layered(kind)
        owner = dd.slab_owner(s.coords, s.box, world)
        mine = np.nonzero(owner == rank)[0]
        dec = dd.SlabDecomposition(s.box, world, rank, m.rc, hops=hops)
        ids, x, t, n_own = dec.gather_local(dist, mine, s.coords[mine], s.types[mine])
        seed = np.zeros(len(ids))
        seed[:n_own] = 1.0                       # ghosts evaluate, their energy is not counted
        E_loc, _, F_loc, _ = oracle.compute_seeded(m, w, t, x, s.box, seed, nthreads=1)
        F = dec.reduce_forces(dist, ids, F_loc, n_own)
        E = dec.total(dist, E_loc)
        out[rank] = (mine, F, E)
    finally:
        dist.destroy_process_group()


def _run_layered(kind, hops, world=3):
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_layered, args=(world, port, kind, hops, out), nprocs=world, join=True)
        return dict(out)


@pytest.mark.parametrize("kind", ["mp", "gf"])
def test_layer_coupled_models_need_an_L_hop_halo(kind):
    """Attention family with message passing and the graph family, 2 layers, 3
    ranks: with a halo of L x rc (the paper's broadened ghost area) every
    owned atom's force and the total energy equal the whole system's; with a
    halo of rc they do not."""
    s = _layered_system()
    m, w = _layered(kind)
    if kind == "mp":
        E, _, F, _ = oracle.af_compute(m, w, s.types, s.coords, s.box)
    else:
        E, _, F, _ = oracle.gf_compute(m, w, s.types, s.coords, s.box)
    rms = np.sqrt(np.mean(F ** 2))
    res = _run_layered(kind, hops=m.n_layers)
    seen = np.zeros(s.n, bool)
    for r in range(3):
        mine, Fr, Er = res[r]
        seen[mine] = True
        assert np.max(np.abs(Fr - F[mine])) <= 1e-11 * rms
        assert Er == pytest.approx(E, rel=1e-12)
    assert seen.all()
    res1 = _run_layered(kind, hops=1)
    worst = max(np.max(np.abs(res1[r][1] - F[res1[r][0]])) for r in range(3))
    # far above FP64 rounding: the second hop is missing
    assert worst > 1e-4 * rms and abs(res1[0][2] - E) > 1e-12 * abs(E)


def test_seeded_oracle_counts_only_seeded_atoms():
    """Seeds 1 everywhere give the plain whole-system result; the seeded
    energy is the seeded atoms' sum of atomic energies."""
    s = _layered_system()
    for kind in ("mp", "gf"):
        m, w = _layered(kind)
        full = oracle.af_compute(m, w, s.types, s.coords, s.box) if kind == "mp" else \
            oracle.gf_compute(m, w, s.types, s.coords, s.box)
        E1, ae1, F1, V1 = oracle.compute_seeded(m, w, s.types, s.coords, s.box, np.ones(s.n))
        assert E1 == full[0] and np.array_equal(F1, full[2]) and np.array_equal(ae1, full[1])
        seed = (np.arange(s.n) % 3 == 0).astype(float)
        E2, ae2, F2, _ = oracle.compute_seeded(m, w, s.types, s.coords, s.box, seed)
        assert E2 == pytest.approx(float(np.sum(ae1[seed > 0])), rel=1e-13)
        assert np.array_equal(ae2, ae1)
        assert np.max(np.abs(F2.sum(0))) <= 1e-10 * np.max(np.abs(F2))


def test_exchange_partners_are_the_slab_neighbours():
    """Halo and force exchanges are point to point with the two slab
    neighbours (one for two ranks, none for one)."""
    box = np.array([40.0, 20.0, 20.0])
    assert dd.SlabDecomposition(box, 4, 0, 6.0).peers() == [1, 3]
    assert dd.SlabDecomposition(box, 4, 2, 6.0).peers() == [1, 3]
    assert dd.SlabDecomposition(box, 2, 1, 6.0).peers() == [0]
    assert dd.SlabDecomposition(box, 1, 0, 6.0).peers() == []
