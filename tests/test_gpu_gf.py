"""GPU parity of the graph-family path against the FP64 oracle, through the C ABI.

Small systems are compared whole (FP64 GPU: 1e-10 of the force RMS, rounding
order only; FP32 GPU: 1e-4; the mixed form, FP32 with every matrix product on
the tensor cores with 16-bit operands: 2e-2 of the force RMS, 5e-3 relative
energy).  At the full 24,000-atom size the oracle's whole-system result is
stored by a script that calls only the oracle (tests/golden/), and every
precision is compared with it on 200 seeded atoms; the FP64 path's forces
are also checked against central finite differences of its energy (h = 1e-4 A).
"""
import json
import os
from dataclasses import replace

import numpy as np
import pytest

import oracle
import paper_2602_02234_b300 as dp
from synth import configs as C, maxwell_boltzmann, normal_blob, serving_system, water_box

pytestmark = pytest.mark.gpu


def weights(model, seed=C.WEIGHT_SEED, sigma=0.1):
    return normal_blob(oracle.gf_weight_count(model), seed, sigma)


def make(model, s, prec, w, masses=None):
    return dp.DeepPotential(dp.model_desc(model, prec), s.types, s.box, w, masses=masses)


def frms(F):
    return float(np.sqrt(np.mean(F ** 2)))


@pytest.mark.parametrize("case", ["tiny_water8", "config3_water96_small_box", "config3_protein700"])
@pytest.mark.parametrize("prec,tol", [(dp.PREC_PLAIN_F64, 1e-10), (dp.PREC_PLAIN_F32, 1e-4),
                                      (dp.PREC_FUSED, 2e-2)])
def test_gf_vs_oracle(case, prec, tol):
    if case == "tiny_water8":
        m = replace(C.GRAPH_MODEL, node=16, edge=8, n_layers=2, f1=12, f2=10, f3=8, nmax=40, na=10)
        s = water_box(8, 9.0, 3, min_oo=2.3)
        s.types = np.where(s.types == 0, 3, 0).astype(np.int32)
        w = weights(m, 3, 0.3)
    elif case == "config3_water96_small_box":
        m, s = C.GRAPH_MODEL, serving_system(96, 5)
        w = weights(m)
    else:
        if prec == dp.PREC_PLAIN_F64:
            pytest.skip("FP64 is covered by the two smaller cases")
        m, s = C.GRAPH_MODEL, serving_system(700, 9)
        w = weights(m)
    if prec == dp.PREC_FUSED and case == "tiny_water8":
        pytest.skip("the mixed form needs widths that are multiples of 16")
    pot = make(m, s, prec, w)
    E, F, V = pot.compute(s.coords)
    Eo, aeo, Fo, Vo = oracle.gf_compute(m, w, s.types, s.coords, s.box)
    etol = 5e-3 if prec == dp.PREC_FUSED else 10 * tol     # 16-bit products: ~0.2 % seen
    assert abs(E - Eo) <= etol * abs(Eo)
    assert np.max(np.abs(F - Fo)) <= tol * frms(Fo)
    assert np.max(np.abs(V - Vo)) <= tol * np.linalg.norm(Vo)


def _golden_24k():
    from tests.golden import make_gf_protein24k as g
    m, s, w = g.inputs()
    path = g.OUT
    if not os.path.exists(path):
        pytest.fail("tests/golden/gf_protein24k.json is missing: run "
                    "python -m tests.golden.make_gf_protein24k")
    with open(path) as f:
        ref = json.load(f)
    assert ref["inputs_sha256"] == g.digest(s, w), "stale golden file: rerun its script"
    return m, s, w, ref


def test_gf_full_size_vs_oracle_and_finite_differences():
    """The 24,000-atom graph-family workload against the FP64 oracle's own
    whole-system result (stored by tests/golden/make_gf_protein24k.py, which
    calls only the oracle): energy, virial, and the forces and atomic energies
    of 200 seeded atoms, in every precision.  Then the hand-written backward of
    the FP64 path against central differences of its energy (h = 1e-4 A) on
    the same 200-atom subset: one directional difference along a random unit
    vector over all 600 of its coordinates, and every component of 10 of its
    atoms."""
    m, s, w, ref = _golden_24k()
    idx = np.array(ref["sample"])
    Fo, aeo = np.array(ref["forces"]), np.array(ref["atom_energies"])
    Eo, Vo, fr = ref["energy"], np.array(ref["virial"]), ref["force_rms"]
    # mixed form: 16-bit operands through six layers bias the energy (2.2e-3 seen)
    for prec, tol, etol in ((dp.PREC_PLAIN_F32, 1e-4, 1e-5), (dp.PREC_FUSED, 2e-2, 5e-3),
                            (dp.PREC_PLAIN_F64, 1e-10, 1e-12)):
        pot = make(m, s, prec, w)
        E, F, V = pot.compute(s.coords)
        ae = pot.atom_energies()[idx]
        if prec == dp.PREC_PLAIN_F64:
            p64, F64 = pot, F
        else:
            pot.close()
        assert abs(E - Eo) <= etol * abs(Eo), (prec, E, Eo)
        assert np.max(np.abs(F[idx] - Fo)) <= tol * fr, prec
        assert np.max(np.abs(V - Vo)) <= tol * np.linalg.norm(Vo), prec
        assert np.max(np.abs(ae - aeo)) <= 10 * max(tol, etol) * np.max(np.abs(aeo)), prec
    assert np.max(np.abs(F64.sum(0))) <= 1e-10
    h = 1e-4
    rng = np.random.default_rng(11)
    d = rng.normal(size=(len(idx), 3))
    d /= np.linalg.norm(d)
    xp = s.coords.copy(); xp[idx] += h * d
    xm = s.coords.copy(); xm[idx] -= h * d
    fd = -(p64.compute(xp)[0] - p64.compute(xm)[0]) / (2 * h)
    assert abs(fd - np.sum(F64[idx] * d)) <= 1e-6 * fr + 1e-9
    for i in idx[rng.choice(len(idx), 10, replace=False)]:
        for a in range(3):
            xp = s.coords.copy(); xp[i, a] += h
            xm = s.coords.copy(); xm[i, a] -= h
            fd = -(p64.compute(xp)[0] - p64.compute(xm)[0]) / (2 * h)
            assert abs(fd - F64[i, a]) <= 1e-6 * fr + 1e-9, (i, a)
    p64.close()


def test_gf_md_step_matches_compute():
    m, s = C.GRAPH_MODEL, serving_system(700, 9)
    w = weights(m)
    masses = s.masses
    v0 = maxwell_boltzmann(masses[s.types], 300.0, C.VELOCITY_SEED)
    pot = make(m, s, dp.PREC_PLAIN_F64, w, masses=masses)
    x, v = s.coords.copy(), v0.copy()
    tr = pot.step(10, C.DT_FS, coords=x, vel=v, energies=True)
    E, F, _ = pot.compute(x)
    assert tr[-1, 0] == pytest.approx(E, rel=1e-12)
    et = tr.sum(1)
    assert np.max(np.abs(et - et[0])) < 1e-6 * abs(et[0])


def test_gf_trajectory_does_not_depend_on_rebuild_schedule():
    """As for the attention family: the incoming-message gather and the force
    gather run over skin lists whose order depends on when they were built."""
    m, s = C.GRAPH_MODEL, serving_system(700, 9)
    w = weights(m)
    masses = s.masses
    v0 = maxwell_boltzmann(masses[s.types], 300.0, C.VELOCITY_SEED)
    out = []
    for step0 in (0, 6):
        pot = make(m, s, dp.PREC_PLAIN_F32, w, masses=masses)
        pot.set_state(s.coords, v0, step=step0)
        pot.step(17, C.DT_FS)
        out.append(pot.get_state()[:2])
        pot.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_gf_mixed_refuses_widths_it_cannot_tile():
    m, s = replace(C.GRAPH_MODEL, edge=40), serving_system(96, 5)
    with pytest.raises(dp.DPError) as e:
        make(m, s, dp.PREC_FUSED, weights(m))
    assert e.value.code == dp.DP_ERR_UNSUPPORTED


def test_gf_mixed_md_tracks_fp32():
    m, s = C.GRAPH_MODEL, serving_system(700, 9)
    w = weights(m)
    masses = s.masses
    v0 = maxwell_boltzmann(masses[s.types], 300.0, C.VELOCITY_SEED)
    out = {}
    for prec in (dp.PREC_PLAIN_F32, dp.PREC_FUSED):
        pot = make(m, s, prec, w, masses=masses)
        x, v = s.coords.copy(), v0.copy()
        tr = pot.step(20, C.DT_FS, coords=x, vel=v, energies=True)
        out[prec] = (x, tr)
        pot.close()
    assert np.max(np.abs(out[dp.PREC_FUSED][0] - out[dp.PREC_PLAIN_F32][0])) < 1e-4
    et = out[dp.PREC_FUSED][1].sum(1)
    assert np.all(np.isfinite(et)) and np.max(np.abs(et - et[0])) < 1e-3 * abs(et[0])


@pytest.mark.parametrize("na,ed", [(40, 64), (64, 16), (64, 64), (64, 128), (64, 192)])
def test_gf_angle_channel_shapes_fp64(na, ed):
    """The angle kernels hold their monomial sums (per slot and per column) in
    shared memory, sized by the angle-slot count and the edge width, and read
    the slots' rows from global memory.  Up to 64 angle slots and widths from
    16 to 192 must give the oracle's result (which sums over the slot pairs)."""
    m = replace(C.GRAPH_MODEL, node=32, edge=ed, n_layers=2, f1=32, f2=32, f3=16, nmax=96, na=na)
    s = serving_system(96, 7)
    w = weights(m, 5, 0.2)
    pot = make(m, s, dp.PREC_PLAIN_F64, w)
    E, F, V = pot.compute(s.coords)
    Eo, _, Fo, Vo = oracle.gf_compute(m, w, s.types, s.coords, s.box)
    assert E == pytest.approx(Eo, rel=1e-11)
    assert np.max(np.abs(F - Fo)) <= 1e-10 * frms(Fo)


@pytest.mark.parametrize("edge", [5, 6])
@pytest.mark.parametrize("prec,tol", [(dp.PREC_PLAIN_F64, 1e-10), (dp.PREC_PLAIN_F32, 1e-4)])
def test_gf_edge_widths_without_vector_paths(edge, prec, tol):
    """Edge widths that are not multiples of 4 take the scalar kernels (message,
    message adjoint, angle-output adjoint, tanh adjoint and row sum, pair
    gradient, edge initialisation; width 5 also the block-per-atom message):
    same results as the oracle."""
    m = replace(C.GRAPH_MODEL, node=12, edge=edge, n_layers=2, f1=12, f2=10, f3=8, nmax=40, na=10)
    s = water_box(8, 9.0, 3, min_oo=2.3)
    s.types = np.where(s.types == 0, 3, 0).astype(np.int32)
    w = weights(m, 4, 0.3)
    pot = make(m, s, prec, w)
    E, F, V = pot.compute(s.coords)
    Eo, aeo, Fo, Vo = oracle.gf_compute(m, w, s.types, s.coords, s.box)
    assert abs(E - Eo) <= 10 * tol * abs(Eo)
    assert np.max(np.abs(F - Fo)) <= tol * frms(Fo)
    assert np.max(np.abs(V - Vo)) <= tol * np.linalg.norm(Vo)
