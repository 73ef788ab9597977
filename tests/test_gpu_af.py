"""GPU parity of the attention-family path against the FP64 oracle, through the C ABI.

Tolerances (from the model's arithmetic; force RMS = RMS of the oracle's force
components over the atoms compared):
  plain FP64:  |dF| <= 1e-10 * F_rms, |dE| <= 1e-11 |E|   (rounding order only)
  plain FP32:  |dF| <= 1e-4 * F_rms                          (FP32 throughout)
  fused:       |dF| <= 2e-2 * F_rms, |dE| <= 1e-3 |E|        (16-bit tensor-core operands)
Integer work (neighbour indices and images) is compared exactly.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import paper_2602_02234_b300 as dp
from synth import configs as C, maxwell_boltzmann, normal_blob, protein_in_water, serving_system, water_box

pytestmark = pytest.mark.gpu

TOL_F = {dp.PREC_PLAIN_F64: 1e-10, dp.PREC_PLAIN_F32: 1e-4, dp.PREC_FUSED: 2e-2}
TOL_E = {dp.PREC_PLAIN_F64: 1e-11, dp.PREC_PLAIN_F32: 2e-5, dp.PREC_FUSED: 1e-3}


def weights(model, seed=C.WEIGHT_SEED):
    return normal_blob(oracle.af_weight_count(model), seed)


def make(model, system, prec, w=None, masses=None):
    w = weights(model) if w is None else w
    return dp.DeepPotential(dp.model_desc(model, prec), system.types, system.box, w,
                            masses=masses), w


def frms(F):
    return float(np.sqrt(np.mean(F ** 2)))


# ------------------------------------------------------------------ neighbours
@pytest.mark.parametrize("name", ["water64", "water96_small_box", "slab900", "protein24k"])
def test_neighbour_lists_exact(name):
    if name == "water64":
        s, m = C.water64(), C.WATER64_MODEL
    elif name == "water96_small_box":
        s, m = serving_system(96, 5), C.ATTN_MODEL
    elif name == "slab900":       # two axes below 3 cells: the per-axis image search
        s, m = protein_in_water(900, 90, (26.0, 19.0, 19.0), 21), C.ATTN_MODEL
    else:
        s, m = C.protein24k(), C.ATTN_MODEL
    pot, w = make(m, s, dp.PREC_PLAIN_F32)
    pot.compute(s.coords)
    cnt, nj, img = pot.neighbours()
    ocnt, onj, oimg, _ = oracle.neighbours(s.coords, s.box, m.rc, m.nmax)
    assert np.array_equal(cnt, ocnt)
    assert np.array_equal(nj, onj)
    assert np.array_equal(img, oimg)


# ------------------------------------------------------------------ energies / forces
@pytest.mark.parametrize("prec", [dp.PREC_PLAIN_F64, dp.PREC_PLAIN_F32, dp.PREC_FUSED])
def test_water64_energy_forces_virial(prec):
    """The 64-water model (embedding 1-25-50-100, one attention layer, nmax 46):
    the fused form runs it with the embedding widths padded to 32, 64 and 128
    (zero weights; LayerNorm statistics over the 100 real columns)."""
    m, s = C.WATER64_MODEL, C.water64()
    pot, w = make(m, s, prec)
    E, F, V = pot.compute(s.coords)
    Eo, aeo, Fo, Vo = oracle.af_compute(m, w, s.types, s.coords, s.box)
    fr = frms(Fo)
    assert abs(E - Eo) <= TOL_E[prec] * abs(Eo)
    assert np.max(np.abs(F - Fo)) <= TOL_F[prec] * fr
    assert np.max(np.abs(V - Vo)) <= TOL_F[prec] * np.linalg.norm(Vo)
    ae = pot.atom_energies()
    assert np.max(np.abs(ae - aeo)) <= 10 * TOL_E[prec] * np.max(np.abs(aeo)) + 1e-14


@pytest.mark.parametrize("case", ["water96_small_box", "isolated_atom", "dimer", "water_tiny_box"])
def test_edge_cases_fp64(case):
    m = replace(C.ATTN_MODEL, n_layers=2, nmax=64)
    if case == "water96_small_box":
        s = serving_system(96, 7)
    elif case == "isolated_atom":
        s = water_box(1, 30.0, 1)
        s.coords, s.types = s.coords[:1], s.types[:1]
    elif case == "dimer":
        s = water_box(1, 30.0, 1)
        s.coords = np.array([[1.0, 1.0, 1.0], [29.5, 2.0, 1.5]])   # across the boundary
        s.types = np.array([3, 0], dtype=np.int32)
    else:
        s = water_box(2, 5.5, 3, min_oo=2.0)      # box < rc: own images are neighbours
        s.types = np.where(s.types == 0, 3, 0).astype(np.int32)
    pot, w = make(m, s, dp.PREC_PLAIN_F64)
    E, F, V = pot.compute(s.coords)
    Eo, _, Fo, Vo = oracle.af_compute(m, w, s.types, s.coords, s.box)
    assert E == pytest.approx(Eo, rel=1e-11, abs=1e-12)
    scale = max(frms(Fo), 1e-12)
    assert np.max(np.abs(F - Fo)) <= 1e-9 * scale + 1e-14


def _sampled_parity(prec, sample_seed=3, n_sample=8, system=C.protein24k):
    m, s = C.ATTN_MODEL, system()
    pot, w = make(m, s, prec)
    E, F, V = pot.compute(s.coords)
    rng = np.random.default_rng(sample_seed)
    # include blob (protein) atoms and the most crowded atom (truncated list)
    cnt = oracle.neighbours(s.coords, s.box, m.rc, 1)[0]
    sample = np.unique(np.concatenate([rng.choice(s.n, n_sample - 2, replace=False),
                                       [rng.integers(0, s.blob_atoms), int(np.argmax(cnt))]]))
    Fo = oracle.af_forces_subset(m, w, s.types, s.coords, s.box, sample)
    ae_o = oracle.af_atoms(m, w, s.types, s.coords, s.box, sample)["atom_e"]
    ae = pot.atom_energies()[sample]
    return F[sample], Fo, ae, ae_o, E


@pytest.mark.parametrize("prec", [dp.PREC_PLAIN_F32, dp.PREC_FUSED])
def test_protein24k_sampled_parity(prec):
    F, Fo, ae, ae_o, E = _sampled_parity(prec)
    assert np.isfinite(E)
    assert np.max(np.abs(F - Fo)) <= TOL_F[prec] * frms(Fo)
    assert np.max(np.abs(ae - ae_o)) <= 10 * TOL_E[prec] * np.max(np.abs(ae_o))


@pytest.mark.parametrize("prec", [dp.PREC_PLAIN_F32, dp.PREC_FUSED])
def test_protein100k_sampled_parity(prec):
    """The 100,000-atom configuration (6,001-atom blob + 31,333 waters) in the
    launch configuration its benchmark times: sampled forces and atomic
    energies against the oracle."""
    F, Fo, ae, ae_o, E = _sampled_parity(prec, sample_seed=7, system=C.protein100k)
    assert np.isfinite(E)
    assert np.max(np.abs(F - Fo)) <= TOL_F[prec] * frms(Fo)
    assert np.max(np.abs(ae - ae_o)) <= 10 * TOL_E[prec] * np.max(np.abs(ae_o))


def test_zero_net_force_and_symmetric_virial_full_size():
    m, s = C.ATTN_MODEL, C.protein24k()
    pot, _ = make(m, s, dp.PREC_PLAIN_F32)
    E, F, V = pot.compute(s.coords)
    assert np.max(np.abs(F.sum(0))) <= 1e-4 * frms(F) * np.sqrt(s.n)
    assert np.max(np.abs(V - V.T)) <= 1e-4 * np.linalg.norm(V)


# ------------------------------------------------------------------ MD
def test_md_matches_oracle_fp64():
    m, s = C.WATER64_MODEL, C.water64()
    masses = s.masses
    v0 = maxwell_boltzmann(masses[s.types], 300.0, C.VELOCITY_SEED)
    pot, w = make(m, s, dp.PREC_PLAIN_F64, masses=masses)
    x = s.coords.copy()
    v = v0.copy()
    tr = pot.step(40, C.DT_FS, coords=x, vel=v, energies=True)
    xo, vo, ep, ek = oracle.af_md(m, w, s.types, masses, s.coords, v0, s.box, 40, C.DT_FS)
    assert np.max(np.abs(x - xo)) < 1e-9
    assert np.max(np.abs(v - vo)) < 1e-11
    assert np.max(np.abs(tr[:, 0] - ep)) < 1e-9 * abs(ep[0])
    assert np.max(np.abs(tr[:, 1] - ek)) < 1e-9 * abs(ek[0])


def test_md_resident_state_resume_is_bitwise():
    m, s = C.WATER64_MODEL, C.water64()
    masses = s.masses
    v0 = maxwell_boltzmann(masses[s.types], 300.0, C.VELOCITY_SEED)
    pot, w = make(m, s, dp.PREC_PLAIN_F32, masses=masses)
    pot.set_state(s.coords, v0, 0)
    pot.step(25, C.DT_FS)
    xa, va, step_a = pot.get_state()
    pot.step(25, C.DT_FS)
    xb, vb, step_b = pot.get_state()
    assert (step_a, step_b) == (25, 50)
    pot2, _ = make(m, s, dp.PREC_PLAIN_F32, w=w, masses=masses)
    pot2.set_state(xa, va, step_a)
    pot2.step(25, C.DT_FS)
    xc, vc, step_c = pot2.get_state()
    assert step_c == 50
    assert np.array_equal(xb, xc) and np.array_equal(vb, vc)


@pytest.mark.parametrize("prec", [dp.PREC_PLAIN_F32, dp.PREC_FUSED])
def test_trajectory_does_not_depend_on_rebuild_schedule(prec):
    """Shifting the step counter moves the neighbour-list rebuilds (every 10
    steps) to other points of the same trajectory; the skin lists then hold
    their entries in another order, and the forces must not notice (bitwise)."""
    m, s = C.ATTN_MODEL, serving_system(700, 9)
    masses = s.masses
    v0 = maxwell_boltzmann(masses[s.types], 300.0, C.VELOCITY_SEED)
    out = []
    for step0 in (0, 5, 7):
        pot, _ = make(m, s, prec, masses=masses)
        pot.set_state(s.coords, v0, step=step0)
        pot.step(23, C.DT_FS)
        out.append(pot.get_state()[:2])
        pot.close()
    for x, v in out[1:]:
        assert np.array_equal(x, out[0][0]) and np.array_equal(v, out[0][1])


@pytest.mark.parametrize("prec", [dp.PREC_PLAIN_F64, dp.PREC_FUSED])
def test_host_round_trip_each_step_matches_resident_stepping(prec):
    """dp_step(1) fed back its own host output each step (the resident forces
    are kept when the coordinates come back unchanged) equals resident
    stepping bit for bit; a changed coordinate is picked up."""
    m, s = replace(C.ATTN_MODEL, n_layers=2) if prec == dp.PREC_PLAIN_F64 else C.ATTN_MODEL, \
        serving_system(300, 4)
    masses = s.masses
    v0 = maxwell_boltzmann(masses[s.types], 300.0, C.VELOCITY_SEED)
    a, _ = make(m, s, prec, masses=masses)
    xa, va = s.coords.copy(), v0.copy()
    ta = a.step(6, C.DT_FS, coords=xa, vel=va, energies=True)
    b, _ = make(m, s, prec, masses=masses)
    xb, vb = s.coords.copy(), v0.copy()
    tb = np.concatenate([b.step(1, C.DT_FS, coords=xb, vel=vb, energies=True) for _ in range(6)])
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(ta, tb)
    # a moved atom must not reuse the old forces
    xc = xb.copy()
    xc[7, 0] += 0.05
    xe, ve = xc.copy(), vb.copy()
    b.step(1, C.DT_FS, coords=xe, vel=ve)
    c, _ = make(m, s, prec, masses=masses)
    c.set_state(xc, vb, 0)
    c.step(1, C.DT_FS)
    xf, vf, _ = c.get_state()
    assert np.array_equal(xe, xf) and np.array_equal(ve, vf)


def test_dpenergy_autograd_matches_finite_differences():
    import torch
    m = replace(C.ATTN_MODEL, n_layers=1, nmax=64)
    s = serving_system(96, 11)
    pot, w = make(m, s, dp.PREC_PLAIN_F64)
    x = torch.tensor(s.coords, dtype=torch.float64, device="cuda", requires_grad=True)
    E = dp.DPEnergy.apply(x, pot)
    E.backward()
    g = x.grad.cpu().numpy()
    h = 1e-4
    for i, a in [(0, 0), (17, 1), (50, 2)]:
        xp = s.coords.copy(); xp[i, a] += h
        xm = s.coords.copy(); xm[i, a] -= h
        fd = (pot.compute(xp)[0] - pot.compute(xm)[0]) / (2 * h)
        assert g[i, a] == pytest.approx(fd, abs=1e-8 * max(1.0, abs(fd)))


def test_errors_are_reported_not_raised_on_device():
    m, s = C.WATER64_MODEL, C.water64()
    pot, _ = make(m, s, dp.PREC_PLAIN_F32)
    with pytest.raises(dp.DPError) as e:
        pot.step(1, 0.5)                  # no masses given at init
    assert e.value.code == dp.DP_ERR_ARG
    bad = s.coords.copy()
    bad[3, 1] = np.nan
    with pytest.raises(dp.DPError):
        pot.compute(bad)
    # the context stays usable
    E, F, V = pot.compute(s.coords)
    assert np.isfinite(E)
    # a box edge below (rc + skin) / 14 would need more periodic images per
    # axis than the small-box search holds
    tiny = water_box(1, 30.0, 1)
    with pytest.raises(dp.DPError) as e:
        dp.DeepPotential(dp.model_desc(m, dp.PREC_PLAIN_F32), tiny.types[:1],
                         np.array([0.3, 30.0, 30.0]), weights(m))
    assert e.value.code == dp.DP_ERR_ARG


# ------------------------------------------------------------------ fused path
def test_fused_full_system_vs_oracle():
    """Every atom of a 700-atom protein-in-water box (configuration-2 model)."""
    m, s = C.ATTN_MODEL, serving_system(700, 9)
    pot, w = make(m, s, dp.PREC_FUSED)
    E, F, V = pot.compute(s.coords)
    Eo, aeo, Fo, Vo = oracle.af_compute(m, w, s.types, s.coords, s.box)
    assert abs(E - Eo) <= TOL_E[dp.PREC_FUSED] * abs(Eo)
    assert np.max(np.abs(F - Fo)) <= TOL_F[dp.PREC_FUSED] * frms(Fo)
    assert np.max(np.abs(V - Vo)) <= TOL_F[dp.PREC_FUSED] * np.linalg.norm(Vo)
    assert np.max(np.abs(F.sum(0))) < 1e-10


@pytest.mark.parametrize("shape", [
    dict(e1=16, e2=48, m2=8, n_layers=1, f1=64, f2=32, f3=16, nmax=100),
    dict(e1=64, e2=128, m2=16, n_layers=2, f1=256, f2=128, f3=48, nmax=128),
    dict(e1=48, e2=80, m2=4, n_layers=0, f1=32, f2=32, f3=32, nmax=90),
])
def test_fused_other_supported_shapes_vs_oracle(shape):
    """Embedding widths that are not multiples of 32, no attention layer, the
    widest fitting layer and the largest neighbour limit the fused path takes."""
    m, s = replace(C.ATTN_MODEL, **shape), serving_system(300, 4)
    pot, w = make(m, s, dp.PREC_FUSED)
    E, F, V = pot.compute(s.coords)
    Eo, aeo, Fo, Vo = oracle.af_compute(m, w, s.types, s.coords, s.box)
    assert abs(E - Eo) <= TOL_E[dp.PREC_FUSED] * abs(Eo)
    assert np.max(np.abs(F - Fo)) <= TOL_F[dp.PREC_FUSED] * frms(Fo)
    assert np.max(np.abs(V - Vo)) <= TOL_F[dp.PREC_FUSED] * np.linalg.norm(Vo)


def test_fused_vs_plain_full_size():
    """All 24,000 atoms against the FP32 path (itself pinned to the oracle)."""
    m, s = C.ATTN_MODEL, C.protein24k()
    fused, w = make(m, s, dp.PREC_FUSED)
    plain, _ = make(m, s, dp.PREC_PLAIN_F32, w=w)
    E, F, V = fused.compute(s.coords)
    Ep, Fp, Vp = plain.compute(s.coords)
    assert abs(E - Ep) <= TOL_E[dp.PREC_FUSED] * abs(Ep)
    assert np.max(np.abs(F - Fp)) <= TOL_F[dp.PREC_FUSED] * frms(Fp)


@pytest.mark.parametrize("change", [dict(hidden=96), dict(heads=2), dict(m1=160),
                                    dict(m1=100, message_passing=1), dict(nmax=130)])
def test_fused_unsupported_sizes_are_refused(change):
    m, s = replace(C.WATER64_MODEL, **change), C.water64()
    with pytest.raises(dp.DPError) as e:
        make(m, s, dp.PREC_FUSED)
    assert e.value.code == dp.DP_ERR_UNSUPPORTED


@pytest.mark.parametrize("shape", [dict(m1=72, e1=20, e2=36, n_layers=2),
                                   dict(m1=120, e1=8, e2=100, n_layers=1, m2=8),
                                   dict(nmax=12, m2=2, n_layers=1)])
def test_fused_padded_widths_vs_oracle(shape):
    """Embedding and attention widths below the tile width (padded inside the
    packed tiles) on the 300-atom water box, every atom against the oracle;
    and a neighbour limit of 12 (every list truncated, two row groups of the
    128-row tiles real) with an axis of 2."""
    m, s = replace(C.ATTN_MODEL, **shape), serving_system(300, 4)
    pot, w = make(m, s, dp.PREC_FUSED)
    E, F, V = pot.compute(s.coords)
    Eo, aeo, Fo, Vo = oracle.af_compute(m, w, s.types, s.coords, s.box)
    assert abs(E - Eo) <= TOL_E[dp.PREC_FUSED] * abs(Eo)
    assert np.max(np.abs(F - Fo)) <= TOL_F[dp.PREC_FUSED] * frms(Fo)
    assert np.max(np.abs(V - Vo)) <= TOL_F[dp.PREC_FUSED] * np.linalg.norm(Vo)


def test_fused_md_tracks_plain():
    m, s = C.ATTN_MODEL, serving_system(700, 9)
    masses = s.masses
    v0 = maxwell_boltzmann(masses[s.types], 300.0, C.VELOCITY_SEED)
    out = {}
    for prec in (dp.PREC_PLAIN_F32, dp.PREC_FUSED):
        pot, _ = make(m, s, prec, masses=masses)
        x, v = s.coords.copy(), v0.copy()
        tr = pot.step(20, C.DT_FS, coords=x, vel=v, energies=True)
        out[prec] = (x, tr)
    dx = np.max(np.abs(out[dp.PREC_FUSED][0] - out[dp.PREC_PLAIN_F32][0]))
    assert dx < 1e-4                      # 10 fs of dynamics with ~1 % force noise
    et = out[dp.PREC_FUSED][1].sum(1)
    assert np.all(np.isfinite(et)) and np.max(np.abs(et - et[0])) < 1e-3 * abs(et[0])


# ------------------------------------------------------------------ DP group
@pytest.mark.parametrize("prec", [dp.PREC_PLAIN_F32, dp.PREC_FUSED])
def test_dp_group_equals_the_members_alone(prec):
    """The protein-only deep potential of the paper (Sec. III): the 300-atom
    blob of a 3,000-atom protein-in-water box as the group."""
    m = C.ATTN_MODEL
    s = protein_in_water(3000, 300, (31.07, 31.07, 31.07), 11)
    mask = np.zeros(s.n, bool)
    mask[: s.blob_atoms] = True
    pot, w = make(m, s, prec)
    pot.set_group(mask)
    E, F, V = pot.compute(s.coords)
    Eo, aeo, Fo, Vo = oracle.af_compute_group(m, w, s.types, s.coords, s.box, mask)
    assert abs(E - Eo) <= TOL_E[prec] * abs(Eo)
    assert np.max(np.abs(F[mask] - Fo[mask])) <= TOL_F[prec] * frms(Fo[mask])
    assert np.max(np.abs(V - Vo)) <= TOL_F[prec] * np.linalg.norm(Vo)
    assert np.all(F[~mask] == 0) and np.all(pot.atom_energies()[~mask] == 0)
    # non-members are invisible: moving them changes nothing, bit for bit
    x2 = s.coords.copy()
    x2[~mask] += np.random.default_rng(2).normal(0, 0.3, (int((~mask).sum()), 3))
    E2, F2, _ = pot.compute(x2)
    assert E2 == E and np.array_equal(F2, F)
    # back to every atom
    pot.set_group(None)
    E3, F3, _ = pot.compute(s.coords)
    ref, _ = make(m, s, prec, w=w)
    E4, F4, _ = ref.compute(s.coords)
    assert E3 == E4 and np.array_equal(F3, F4)


# ------------------------------------------------------------------ fitting heads
@pytest.mark.parametrize("prec", [dp.PREC_PLAIN_F32, dp.PREC_FUSED])
def test_fitting_heads_share_one_descriptor(prec):
    """Three fitting heads on the configuration-2 model: every head's energy
    matches the single-head model with that head's fitting nets; forces,
    virial and dp_compute's energy are head 0's."""
    m = replace(C.ATTN_MODEL, fit_heads=3)
    s = serving_system(700, 9)
    w = weights(m)
    pot = dp.DeepPotential(dp.model_desc(m, prec), s.types, s.box, w)
    E, F, V = pot.compute(s.coords)
    he = pot.head_energies()
    eo, (Eo, aeo, Fo, Vo) = oracle.af_compute_heads(m, w, s.types, s.coords, s.box)
    assert he.shape == (3,) and he[0] == E
    for h in range(3):
        # a head's total can be small by cancellation: scale by its atomic energies
        wh, dh = oracle.af_head_blob(m, w, h)
        ae_h = oracle.af_compute(dh, wh, s.types, s.coords, s.box)[1]
        assert abs(he[h] - eo[h]) <= TOL_E[prec] * np.sum(np.abs(ae_h))
    assert len(set(np.round(eo, 6))) == 3                  # the heads really differ
    assert np.max(np.abs(F - Fo)) <= TOL_F[prec] * frms(Fo)
    assert np.max(np.abs(V - Vo)) <= TOL_F[prec] * np.linalg.norm(Vo)


@pytest.mark.parametrize("prec", [dp.PREC_PLAIN_F64, dp.PREC_PLAIN_F32, dp.PREC_FUSED])
def test_energy_beyond_the_exact_sums_range_is_reported(prec):
    """Forces, virials and energies are summed exactly in 128-bit fixed point
    (2^-80 resolution, so a sum must stay below 2^47 in magnitude).  A total
    energy beyond that range, made of in-range atomic energies, is reported
    as DP_ERR_NONFINITE instead of wrapping; one just inside it is summed."""
    m, s = C.WATER64_MODEL, C.water64()
    n = len(s.types)
    base = weights(m)

    def with_bias(b):
        w = base.copy()
        for a in range(m.n_species):
            w[oracle.af_weight_slice(m, "fb4", a)] = b
        return w

    # 192 atoms x 1e12 eV = 1.9e14 eV > 2^47 = 1.4e14 eV (each atom < 2^46)
    pot = dp.DeepPotential(dp.model_desc(m, prec), s.types, s.box, with_bias(1e12))
    with pytest.raises(dp.DPError) as e:
        pot.compute(s.coords)
    assert e.value.code == dp.DP_ERR_NONFINITE
    pot.close()
    # 192 x 1e11 eV = 1.9e13 eV: in range; the bias dominates every atom
    pot = dp.DeepPotential(dp.model_desc(m, prec), s.types, s.box, with_bias(1e11))
    E, F, V = pot.compute(s.coords)
    assert np.isfinite(E) and abs(E - n * 1e11) <= 1e-6 * n * 1e11
    assert np.all(np.isfinite(F)) and np.all(np.isfinite(V))
    pot.close()


@pytest.mark.parametrize("prec", [dp.PREC_PLAIN_F32, dp.PREC_FUSED])
def test_isolated_atoms_keep_their_energy(prec):
    """Atoms with no neighbour within rc (the fused kernels skip their
    per-atom pipeline) still carry the fitting of a zero descriptor, and no
    force; the rest of the box is unaffected."""
    m = C.ATTN_MODEL
    base = serving_system(300, 4)
    L = base.box.copy()
    L[0] += 30.0                                 # empty slab beyond the water
    x = np.concatenate([base.coords % base.box, [[base.box[0] + 15.0, 3.0, 4.0],
                                                 [base.box[0] + 15.0, 9.0, 11.0]]])
    t = np.concatenate([base.types, [1, 4]]).astype(np.int32)
    from synth import System
    s = System(coords=x, types=t, box=L, species=base.species, note="isolated", blob_atoms=0)
    pot, w = make(m, s, prec)
    E, F, V = pot.compute(s.coords)
    Eo, aeo, Fo, Vo = oracle.af_compute(m, w, s.types, s.coords, s.box)
    ae = pot.atom_energies()
    assert abs(E - Eo) <= TOL_E[prec] * np.sum(np.abs(aeo))
    assert np.all(F[-2:] == 0)
    assert np.max(np.abs(ae[-2:] - aeo[-2:])) <= 1e-3 * np.max(np.abs(aeo[-2:])) + 1e-6
    assert np.max(np.abs(F - Fo)) <= TOL_F[prec] * frms(Fo)


# ------------------------------------------------------------------ message passing
MP_MODEL = replace(C.ATTN_MODEL, message_passing=1)
_mp_oracle_cache = {}


def _mp_system():
    return protein_in_water(2400, 150, (26.8, 26.8, 33.5), 5)


def _mp_oracle(model, s, key):
    if key not in _mp_oracle_cache:
        _mp_oracle_cache[key] = oracle.af_compute(model, weights(model), s.types, s.coords, s.box)
    return _mp_oracle_cache[key]


@pytest.mark.parametrize("prec", [dp.PREC_PLAIN_F64, dp.PREC_PLAIN_F32])
def test_message_passing_vs_oracle(prec):
    """2,400 atoms (protein blob in water, 19 tiles of 128 with a ragged tail):
    energies, atomic energies, forces and virial against the FP64 oracle."""
    s = _mp_system()
    pot, w = make(MP_MODEL, s, prec)
    E, F, V = pot.compute(s.coords)
    Eo, aeo, Fo, Vo = _mp_oracle(MP_MODEL, s, "protein2400")
    fr = frms(Fo)
    assert abs(E - Eo) <= TOL_E[prec] * abs(Eo)
    assert np.max(np.abs(F - Fo)) <= TOL_F[prec] * fr
    assert np.max(np.abs(V - Vo)) <= TOL_F[prec] * np.linalg.norm(Vo)
    ae = pot.atom_energies()
    assert np.max(np.abs(ae - aeo)) <= 10 * TOL_E[prec] * np.max(np.abs(aeo)) + 1e-14


def test_message_passing_edge_cases_fp64():
    """A box smaller than rc (own images are neighbours, one atom's slots name
    the same atom several times) and an isolated atom beside a dimer."""
    m = replace(MP_MODEL, n_layers=2, nmax=64)
    s = water_box(2, 5.5, 3, min_oo=2.0)
    s.types = np.where(s.types == 0, 3, 0).astype(np.int32)
    pot, w = make(m, s, dp.PREC_PLAIN_F64)
    E, F, V = pot.compute(s.coords)
    Eo, _, Fo, Vo = oracle.af_compute(m, w, s.types, s.coords, s.box)
    assert E == pytest.approx(Eo, rel=1e-11, abs=1e-12)
    assert np.max(np.abs(F - Fo)) <= 1e-9 * frms(Fo) + 1e-14
    s = water_box(1, 30.0, 1)
    s.coords = np.array([[1.0, 1.0, 1.0], [29.5, 2.0, 1.5], [15.0, 15.0, 15.0]])
    s.types = np.array([3, 0, 1], dtype=np.int32)
    pot, w = make(m, s, dp.PREC_PLAIN_F64)
    E, F, V = pot.compute(s.coords)
    Eo, aeo, Fo, Vo = oracle.af_compute(m, w, s.types, s.coords, s.box)
    assert E == pytest.approx(Eo, rel=1e-11, abs=1e-12)
    assert np.max(np.abs(F - Fo)) <= 1e-9 * frms(Fo) + 1e-14
    assert np.all(F[2] == 0)


@pytest.mark.parametrize("prec", [dp.PREC_PLAIN_F32, dp.PREC_FUSED])
def test_message_passing_trajectory_does_not_depend_on_rebuild_schedule(prec):
    """The reverse gather of the message adjoint sums the slots naming an atom
    in (i, p) order, not in skin-list order: shifted rebuilds change nothing."""
    m, s = replace(MP_MODEL, n_layers=2), serving_system(700, 9)
    masses = s.masses
    v0 = maxwell_boltzmann(masses[s.types], 300.0, C.VELOCITY_SEED)
    out = []
    for step0 in (0, 5, 7):
        pot, _ = make(m, s, prec, masses=masses)
        pot.set_state(s.coords, v0, step=step0)
        pot.step(23, C.DT_FS)
        out.append(pot.get_state()[:2])
        pot.close()
    for x, v in out[1:]:
        assert np.array_equal(x, out[0][0]) and np.array_equal(v, out[0][1])


def _hops_to(k, nj, layers):
    """Atoms i that reach atom k within `layers` links i -> j of the kept lists."""
    n = nj.shape[0]
    src = np.repeat(np.arange(n), nj.shape[1])
    dst = nj.reshape(-1)
    keep = dst >= 0
    src, dst = src[keep], dst[keep]
    order = np.argsort(dst, kind="stable")
    src, dst = src[order], dst[order]
    start = np.searchsorted(dst, np.arange(n + 1))
    reach = np.zeros(n, bool)
    reach[k] = True
    frontier = np.array([k])
    for _ in range(layers):
        nxt = np.unique(np.concatenate([src[start[j]:start[j + 1]] for j in frontier]))
        nxt = nxt[~reach[nxt]]
        reach[nxt] = True
        frontier = nxt
    return reach


@pytest.mark.parametrize("prec", [dp.PREC_PLAIN_F32, dp.PREC_FUSED])
def test_message_passing_locality_full_size(prec):
    """24,000 atoms: moving one atom changes the atomic energy of every atom
    whose kept lists reach it in one link, and leaves every atom that cannot
    reach it within L links bit for bit unchanged (the L x rc halo), with the
    net force zero."""
    s = C.protein24k()
    pot, w = make(MP_MODEL, s, prec)
    E0, F0, _ = pot.compute(s.coords)
    ae0 = pot.atom_energies()
    cnt0, nj0, img0 = pot.neighbours()
    assert np.max(np.abs(F0.sum(0))) <= 1e-3 * frms(F0) * np.sqrt(s.n)
    k = s.blob_atoms + 1000
    x = s.coords.copy()
    x[k] += np.array([1e-3, -2e-3, 1.5e-3])
    pot.compute(x)
    ae1 = pot.atom_energies()
    cnt1, nj1, _ = pot.neighbours()
    # links of either evaluation (k may enter or leave a list at the cutoff)
    both = np.concatenate([nj0, nj1], 1)
    reach = _hops_to(k, both, MP_MODEL.n_layers)
    one = np.array([k in set(nj0[i]) and k in set(nj1[i]) for i in range(s.n)])
    one[k] = True
    assert np.array_equal(ae1[~reach], ae0[~reach])
    assert np.all(ae1[one] != ae0[one])
    assert reach.sum() > one.sum() > 1


# The fused form's energy error is a per-atom bias of about -2e-4 eV from its
# 16-bit operands (9.3e-4 of |E| for the model without messages on this
# system); the message adds one more 16-bit rounding of G' per layer, so the
# energy bound is doubled.  Forces keep the fused bound.
TOL_E_FUSED_MP = 2e-3


def test_message_passing_fused_vs_oracle():
    """The fused form runs one launch per layer with the cross-atom steps in
    between; same 2,400-atom system."""
    s = _mp_system()
    pot, w = make(MP_MODEL, s, dp.PREC_FUSED)
    E, F, V = pot.compute(s.coords)
    Eo, aeo, Fo, Vo = _mp_oracle(MP_MODEL, s, "protein2400")
    fr = frms(Fo)
    assert abs(E - Eo) <= TOL_E_FUSED_MP * abs(Eo)
    assert np.max(np.abs(F - Fo)) <= TOL_F[dp.PREC_FUSED] * fr
    assert np.max(np.abs(V - Vo)) <= TOL_F[dp.PREC_FUSED] * np.linalg.norm(Vo)


def test_message_passing_fused_vs_plain_full_size():
    s = C.protein24k()
    w = weights(MP_MODEL)
    out = {}
    for prec in (dp.PREC_PLAIN_F32, dp.PREC_FUSED):
        pot, _ = make(MP_MODEL, s, prec, w=w)
        out[prec] = pot.compute(s.coords)
        pot.close()
    E32, F32, _ = out[dp.PREC_PLAIN_F32]
    Ef, Ff, _ = out[dp.PREC_FUSED]
    assert abs(Ef - E32) <= TOL_E_FUSED_MP * abs(E32)
    assert np.max(np.abs(Ff - F32)) <= TOL_F[dp.PREC_FUSED] * frms(F32)


def test_message_passing_fused_with_inert_messages_is_the_fused_model():
    """Wm = 0, bm = 0: the per-layer launches, the FP32 residual stream kept
    between them, the message, the atom channel and the adjoint's cross-atom
    steps must reproduce the single-launch fused model bit for bit."""
    s = _mp_system()
    w = weights(MP_MODEL)
    for l in range(MP_MODEL.n_layers):
        w[oracle.afmp_weight_slice(MP_MODEL, "Wm", l)] = 0.0
        w[oracle.afmp_weight_slice(MP_MODEL, "bm", l)] = 0.0
    keep = np.ones(len(w), bool)
    keep[oracle.afmp_weight_slice(MP_MODEL, "Wt")] = False
    for l in range(MP_MODEL.n_layers):
        keep[oracle.afmp_weight_slice(MP_MODEL, "Wm", l)] = False
        keep[oracle.afmp_weight_slice(MP_MODEL, "bm", l)] = False
    a, _ = make(MP_MODEL, s, dp.PREC_FUSED, w=w)
    b, _ = make(C.ATTN_MODEL, s, dp.PREC_FUSED, w=w[keep])
    Ea, Fa, Va = a.compute(s.coords)
    Eb, Fb, Vb = b.compute(s.coords)
    assert Ea == Eb and np.array_equal(Fa, Fb) and np.array_equal(Va, Vb)
    assert np.array_equal(a.atom_energies(), b.atom_energies())


def test_md_retries_after_a_neighbour_capacity_overflow():
    """300 atoms start dilute (the skin capacity is sized from the mean
    density: 160 entries per atom) and fall towards the box centre, so the
    lists rebuilt during dp_step outgrow it.  dp_step restores its on-device
    checkpoint, doubles the capacity and reruns the steps; the trajectory must
    still be the oracle's."""
    m = replace(C.ATTN_MODEL, n_layers=1, nmax=64)
    rng = np.random.default_rng(17)
    L = 20.0
    g = (np.arange(7) + 0.5) * (L / 7)
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)[:300]
    x0 = pts + rng.uniform(-0.3, 0.3, pts.shape)
    types = (np.arange(300) % 2 == 0).astype(np.int32) * 3       # O-like and H
    box = np.full(3, L)
    masses = np.array([1.008, 12.011, 14.007, 15.999, 32.06])
    v0 = -0.04 * (x0 - L / 2)                                    # A/fs, inwards
    w = weights(m)
    pot = dp.DeepPotential(dp.model_desc(m, dp.PREC_PLAIN_F64), types, box, w, masses=masses)
    pot.set_state(x0, v0, 0)
    pot.step(20, C.DT_FS)
    x, v, _ = pot.get_state()
    xo, vo, _, _ = oracle.af_md(m, w, types, masses, x0, v0, box, 20, C.DT_FS)
    # the final configuration needs more skin entries than the first capacity
    cnt = oracle.neighbours(xo, box, m.rc + 1.0, 1)[0]
    assert cnt.max() > 160
    assert np.max(np.abs(x - xo)) < 1e-9 and np.max(np.abs(v - vo)) < 1e-9
