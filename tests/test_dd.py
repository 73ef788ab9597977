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
