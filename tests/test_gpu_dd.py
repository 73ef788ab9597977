"""GPU subdomain evaluation of the slab decomposition: every rank's local
system (owned atoms and their ghosts within rc) evaluated on the GPU with the
owned atoms as the only centres (dp_set_centres); the partial forces summed
over ranks, the owned energies and the virials must equal the whole system's
evaluation in the same precision.  The local atoms are numbered in the order
of their global ids, so neighbours at exactly equal distances (a water's two
hydrogens seen from its oxygen) are ranked as in the whole system; the owned
centres then see the same neighbour lists in the same order and give the
same pair gradients, and only the grouping of the final sums differs
(tolerance 1e-12 of the force RMS in every precision).

Layer-coupled models (message passing, the graph family) are evaluated with
an n_layers x rc halo and an energy seed instead (dp_set_energy_seed)."""
import numpy as np
import pytest

import oracle
import paper_2602_02234_b300 as dp
from paper_2602_02234_b300 import dd
from synth import configs as C, normal_blob, protein_in_water

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [dp.PREC_PLAIN_F64, dp.PREC_PLAIN_F32, dp.PREC_FUSED])
@pytest.mark.parametrize("world", [2, 3])
def test_subdomains_on_the_gpu_reproduce_the_whole_system(prec, world):
    m = C.ATTN_MODEL
    s = protein_in_water(900, 90, (26.0, 19.0, 19.0), 21)
    w = normal_blob(oracle.af_weight_count(m), C.WEIGHT_SEED)
    desc = dp.model_desc(m, prec)
    whole = dp.DeepPotential(desc, s.types, s.box, w)
    E, F, V = whole.compute(s.coords)
    whole.close()
    Fs, Es, Vs = np.zeros_like(F), 0.0, np.zeros((3, 3))
    seen = np.zeros(s.n, bool)
    for rank in range(world):
        ids, x, t, n_own = dd.local_system(s.coords, s.types, s.box, rank, world, m.rc)
        assert len(ids) > n_own                       # there are ghosts
        seen[ids[:n_own]] = True
        owned = np.arange(len(ids)) < n_own
        order = np.argsort(ids, kind="stable")        # global-id order
        ids, x, t, owned = ids[order], x[order], t[order], owned[order]
        pot = dp.DeepPotential(desc, t, s.box, w)
        pot.set_centres(owned)
        El, Fl, Vl = pot.compute(x)
        ae = pot.atom_energies()
        assert np.all(ae[~owned] == 0.0)               # ghosts carry no energy
        pot.close()
        np.add.at(Fs, ids, Fl)
        Es += El
        Vs += Vl
    assert seen.all()
    rms = float(np.sqrt(np.mean(F ** 2)))
    assert np.max(np.abs(Fs - F)) <= 1e-12 * rms
    assert Es == pytest.approx(E, rel=1e-12)
    assert np.max(np.abs(Vs - V)) <= 1e-12 * np.max(np.abs(V))


def test_centres_mask_refused_for_layer_coupled_models():
    from dataclasses import replace
    m = replace(C.ATTN_MODEL, message_passing=1)
    s = protein_in_water(900, 90, (26.0, 19.0, 19.0), 21)
    w = normal_blob(oracle.af_weight_count(m), C.WEIGHT_SEED)
    pot = dp.DeepPotential(dp.model_desc(m, dp.PREC_PLAIN_F32), s.types, s.box, w)
    with pytest.raises(dp.DPError) as e:
        pot.set_centres(np.arange(s.n) < 100)
    assert e.value.code == dp.DP_ERR_UNSUPPORTED


# ------------------------------------------------------------- layer-coupled models
# The attention family with message passing and the graph family reach
# n_layers neighbour hops: the halo is n_layers x rc, every local atom is a
# centre and only the owned atoms' energies are counted and seed the adjoint
# (dp_set_energy_seed).  The owned energies are the whole system's, evaluated
# in the same order (equal bits seen in every precision); each rank's partial
# forces carry only part of every adjoint, so their sum over ranks equals the
# whole system's up to the rounding of the path's arithmetic (seen: FP64
# 2e-15 of the force RMS, FP32 7e-7, the 16-bit tensor-core forms 5.5e-4).
LAYERED_TOL = {dp.PREC_PLAIN_F64: (1e-12, 1e-12), dp.PREC_PLAIN_F32: (1e-10, 1e-5),
               dp.PREC_FUSED: (1e-6, 3e-3)}


def _layered_model(kind):
    from dataclasses import replace
    if kind == "attention_mp":
        m = replace(C.ATTN_MODEL, message_passing=1, n_layers=2)
        return m, normal_blob(oracle.af_weight_count(m), C.WEIGHT_SEED)
    m = replace(C.GRAPH_MODEL, n_layers=2)
    return m, normal_blob(oracle.gf_weight_count(m), C.WEIGHT_SEED)


@pytest.mark.parametrize("prec", [dp.PREC_PLAIN_F64, dp.PREC_PLAIN_F32, dp.PREC_FUSED])
@pytest.mark.parametrize("kind", ["attention_mp", "graph"])
def test_seeded_subdomains_of_layer_coupled_models(kind, prec):
    m, w = _layered_model(kind)
    world, hops = 3, m.n_layers
    s = protein_in_water(1290, 90, (37.0, 19.0, 19.0), 23)
    desc = dp.model_desc(m, prec)
    whole = dp.DeepPotential(desc, s.types, s.box, w)
    E, F, V = whole.compute(s.coords)
    ae_whole = whole.atom_energies()
    whole.close()
    Fs, Es, Vs = np.zeros_like(F), 0.0, np.zeros((3, 3))
    seen = np.zeros(s.n, bool)
    etol, ftol = LAYERED_TOL[prec]
    for rank in range(world):
        ids, x, t, n_own = dd.local_system(s.coords, s.types, s.box, rank, world, m.rc, hops=hops)
        seen[ids[:n_own]] = True
        owned = np.arange(len(ids)) < n_own
        order = np.argsort(ids, kind="stable")        # global-id order
        ids, x, t, owned = ids[order], x[order], t[order], owned[order]
        pot = dp.DeepPotential(desc, t, s.box, w)
        pot.set_energy_seed(owned)
        El, Fl, Vl = pot.compute(x)
        ae = pot.atom_energies()
        pot.close()
        assert np.all(ae[~owned] == 0.0)               # ghosts carry no energy
        own_ids = ids[owned]
        assert np.max(np.abs(ae[owned] - ae_whole[own_ids])) <= etol * np.max(np.abs(ae_whole))
        np.add.at(Fs, ids, Fl)
        Es += El
        Vs += Vl
    assert seen.all()
    rms = float(np.sqrt(np.mean(F ** 2)))
    err_f = np.max(np.abs(Fs - F)) / rms
    err_v = np.max(np.abs(Vs - V)) / np.max(np.abs(V))
    print(f"{kind} prec {prec}: dE/E {abs(Es - E) / abs(E):.2e} dF/rms {err_f:.2e} dV {err_v:.2e}")
    assert Es == pytest.approx(E, rel=etol)
    assert err_f <= ftol
    assert err_v <= ftol


def test_energy_seed_with_a_one_hop_halo_misses_the_second_hop():
    """The L x rc halo is needed: with a one-hop halo the owned atoms' energies
    differ from the whole system's (the second hop's atoms are missing)."""
    m, w = _layered_model("attention_mp")
    s = protein_in_water(1290, 90, (37.0, 19.0, 19.0), 23)
    desc = dp.model_desc(m, dp.PREC_PLAIN_F64)
    whole = dp.DeepPotential(desc, s.types, s.box, w)
    whole.compute(s.coords)
    ae_whole = whole.atom_energies()
    whole.close()
    ids, x, t, n_own = dd.local_system(s.coords, s.types, s.box, 0, 3, m.rc, hops=1)
    owned = np.arange(len(ids)) < n_own
    order = np.argsort(ids, kind="stable")
    ids, x, t, owned = ids[order], x[order], t[order], owned[order]
    pot = dp.DeepPotential(desc, t, s.box, w)
    pot.set_energy_seed(owned)
    pot.compute(x)
    ae = pot.atom_energies()
    pot.close()
    assert np.max(np.abs(ae[owned] - ae_whole[ids[owned]])) > 1e-8 * np.max(np.abs(ae_whole))
