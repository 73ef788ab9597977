"""Pins of the FP64 attention-family oracle against facts that do not come from it.

* switch: closed-form values and vanishing derivatives at both ends;
* neighbours: cell list == brute force (C), and == a numpy brute force, exactly;
* gradient: central finite differences (h = 1e-4 A), strain derivative of E;
* a second, independent reading of the whole model in PyTorch + autograd;
* closed forms: fitting bias only, a dimer with no attention layer, a dimer with
  one attention layer whose query/key weights vanish;
* invariants: translation, same-species permutation, rotation of an isolated
  cluster, cubic symmetry under periodic boundaries, zero net force, symmetric
  virial, E constant for a pair beyond rc and continuous at rc;
* NVE: energy fluctuation ~ dt^2, time reversibility.
"""
import itertools
import math
from dataclasses import replace

import numpy as np
import pytest
import torch

import oracle
from synth import configs as C, normal_blob, serving_system, water_box
from tests import af_torch_ref

TINY = C.AttnModel(n_species=2, e1=6, e2=10, m1=16, m2=4, n_layers=2, hidden=16, heads=2,
                   f1=20, f2=18, f3=12, nmax=40, rc=6.0, rs=0.5)


def blob(model, seed=7, sigma=0.1):
    return normal_blob(oracle.af_weight_count(model), seed, sigma)


def small_water(n_mol=8, L=9.0, seed=3):
    return water_box(n_mol, L, seed, min_oo=2.3)


# ---------------------------------------------------------------- switch
def test_switch_closed_form():
    rs, rc = 0.5, 6.0
    assert oracle.switch(0.3, rs, rc) == (1.0, 0.0)
    assert oracle.switch(rs, rs, rc) == (1.0, 0.0)
    assert oracle.switch(rc, rs, rc) == (0.0, 0.0)
    assert oracle.switch(7.0, rs, rc) == (0.0, 0.0)
    sw, dsw = oracle.switch(0.5 * (rs + rc), rs, rc)
    assert sw == pytest.approx(0.5, abs=1e-15)
    # at u = 1/2 the quintic smoothstep has slope 15/8 per unit u
    assert dsw == pytest.approx(-15.0 / 8.0 / (rc - rs), rel=1e-14)
    # first and second derivatives vanish at both ends (one-sided differences)
    h = 1e-4
    for r0, side in ((rs, +1), (rc, -1)):
        d1 = oracle.switch(r0 + side * h, rs, rc)[1]
        assert abs(d1) < 1e-6
        d2 = (oracle.switch(r0 + side * 2 * h, rs, rc)[1] - oracle.switch(r0 + side * h, rs, rc)[1]) / h
        assert abs(d2) < 1e-3
    # derivative against central differences in the interior
    for r in np.linspace(0.7, 5.8, 9):
        fd = (oracle.switch(r + 1e-6, rs, rc)[0] - oracle.switch(r - 1e-6, rs, rc)[0]) / 2e-6
        assert oracle.switch(r, rs, rc)[1] == pytest.approx(fd, abs=1e-8)


# ---------------------------------------------------------------- neighbours
def _numpy_brute(coords, box, rc):
    lst = af_torch_ref.select_neighbours(coords, box, rc, 10 ** 6)
    return [[(j, tuple(int(v) for v in im)) for j, im in row] for row in lst]


@pytest.mark.parametrize("L,n_mol", [(5.5, 2), (7.0, 4), (9.86, 32), (12.42, 64)])
def test_neighbours_small_box_vs_numpy(L, n_mol):
    """Boxes under 2 rc: several images of one atom are neighbours; under rc the
    atom's own images are too."""
    s = water_box(n_mol, L, 11, min_oo=2.0)
    cnt, nj, ni, _ = oracle.neighbours(s.coords, s.box, 6.0, 800, use_cells=False)
    ref = _numpy_brute(s.coords, s.box, 6.0)
    for i in range(s.n):
        got = [(int(nj[i, k]), tuple(int(v) for v in ni[i, k])) for k in range(cnt[i])]
        assert got == ref[i]
    if L < 12:
        assert any(len(set(int(j) for j in nj[i, :cnt[i]])) < cnt[i] for i in range(s.n))
    if L < 6:
        assert any(nj[i, k] == i for i in range(s.n) for k in range(cnt[i]))


def test_neighbours_cells_equal_brute():
    s = water_box(220, 19.0, 5)          # 3 x 3 x 3 cells of edge >= 6 A
    a = oracle.neighbours(s.coords, s.box, 6.0, 200, use_cells=True)
    b = oracle.neighbours(s.coords, s.box, 6.0, 200, use_cells=False)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_neighbours_truncation_keeps_nearest():
    s = C.water64()
    cnt, nj, ni, nr = oracle.neighbours(s.coords, s.box, 6.0, 46)
    full = _numpy_brute(s.coords, s.box, 6.0)
    assert cnt.min() > 46                  # 46 always truncates at 0.1 atoms/A^3
    for i in range(s.n):
        assert [(int(nj[i, k]), tuple(int(v) for v in ni[i, k])) for k in range(46)] == full[i][:46]
        d = np.linalg.norm(nr[i], axis=1)
        assert np.all(np.diff(d) >= 0)


# ---------------------------------------------------------------- gradient
def _fd_forces(model, w, types, x, box, atoms, h=1e-4):
    out = np.zeros((len(atoms), 3))
    for q, i in enumerate(atoms):
        for a in range(3):
            xp = x.copy(); xp[i, a] += h
            xm = x.copy(); xm[i, a] -= h
            out[q, a] = -(oracle.af_compute(model, w, types, xp, box)[0]
                          - oracle.af_compute(model, w, types, xm, box)[0]) / (2 * h)
    return out


@pytest.mark.parametrize("case", ["dimer", "trimer", "water8", "cluster20"])
def test_forces_central_differences(case):
    rng = np.random.default_rng(1)
    if case == "dimer":
        x = np.array([[10.0, 10.0, 10.0], [12.1, 10.7, 9.4]]); t = np.array([0, 1]); box = np.full(3, 40.0)
    elif case == "trimer":
        x = np.array([[10.0, 10.0, 10.0], [11.0, 10.2, 10.1], [10.3, 12.0, 11.0]]); t = np.array([0, 1, 1])
        box = np.full(3, 40.0)
    elif case == "water8":
        s = small_water(); x, t, box = s.coords, s.types, s.box
    else:
        x = 10 + rng.uniform(0, 6, size=(20, 3)); t = rng.integers(0, 2, 20); box = np.full(3, 40.0)
    w = blob(TINY)
    _, _, F, _ = oracle.af_compute(TINY, w, t, x, box)
    atoms = list(range(min(len(t), 6)))
    fd = _fd_forces(TINY, w, t, x, box, atoms)
    scale = np.sqrt(np.mean(F ** 2))
    assert np.max(np.abs(fd - F[atoms])) < 1e-7 * max(scale, 1e-3) + 1e-10


def test_forces_fd_water64_config_model():
    """The configuration's own model sizes (M1 100, one attention layer), Nmax
    raised to 138 so that no neighbour is truncated."""
    m = replace(C.WATER64_MODEL, nmax=138)
    w = blob(m, seed=C.WEIGHT_SEED)
    s = C.water64()
    _, _, F, _ = oracle.af_compute(m, w, s.types, s.coords, s.box)
    fd = _fd_forces(m, w, s.types, s.coords, s.box, [5, 77])
    assert np.max(np.abs(fd - F[[5, 77]])) < 1e-8


def test_virial_is_minus_strain_derivative():
    s = small_water()
    w = blob(TINY)
    E, _, F, V = oracle.af_compute(TINY, w, s.types, s.coords, s.box)
    assert np.allclose(V, V.T, atol=1e-12)
    eps = 1e-6
    for a in range(3):
        def e_at(e):
            M = np.eye(3); M[a, a] += e
            return oracle.af_compute(TINY, w, s.types, s.coords @ M.T, s.box * np.diag(M))[0]
        assert V[a, a] == pytest.approx(-(e_at(eps) - e_at(-eps)) / (2 * eps), abs=1e-8)
    # off-diagonal strain on an isolated cluster (no box change needed)
    x = s.coords - s.coords.mean(0) + 30.0
    E, _, F, V = oracle.af_compute(TINY, w, s.types, x, np.full(3, 60.0))
    for a, b in ((0, 1), (1, 2), (2, 0)):
        def e_at(e):
            M = np.eye(3); M[a, b] += e
            return oracle.af_compute(TINY, w, s.types, (x - 30.0) @ M.T + 30.0, np.full(3, 60.0))[0]
        assert V[a, b] == pytest.approx(-(e_at(eps) - e_at(-eps)) / (2 * eps), abs=1e-8)


# ---------------------------------------------------------------- second reading
@pytest.mark.parametrize("case", ["water8", "water64_tiny"])
def test_matches_torch_autograd_restatement(case):
    if case == "water8":
        s = small_water(); m = TINY
    else:
        s = C.water64(); m = replace(TINY, nmax=46)
    w = blob(m)
    E, ae, F, V = oracle.af_compute(m, w, s.types, s.coords, s.box)
    x = torch.tensor(s.coords, dtype=torch.float64, requires_grad=True)
    Et = af_torch_ref.energy(m.as_dict(), w, s.types, x, s.box)
    Et.backward()
    Ft = -x.grad.numpy()
    assert E == pytest.approx(float(Et.detach()), rel=1e-12)
    assert np.max(np.abs(F - Ft)) <= 1e-10 * np.max(np.abs(Ft))


def test_config1_model_matches_torch():
    """Config-1 sizes (M1 100, H 128, 4 heads, fitting 1600->240^3, Nmax 46)."""
    m = C.WATER64_MODEL
    w = blob(m, seed=C.WEIGHT_SEED)
    s = C.water64()
    sub = slice(0, 8)
    x = torch.tensor(s.coords, dtype=torch.float64, requires_grad=True)
    nb = af_torch_ref.select_neighbours(s.coords, s.box, m.rc, m.nmax)
    # energy of the first 8 atoms only: restrict the sum by zeroing the others' types' output
    Et = af_torch_ref.energy(m.as_dict(), w, s.types, x, s.box, nbrs=nb)
    E, ae, F, V = oracle.af_compute(m, w, s.types, s.coords, s.box)
    assert E == pytest.approx(float(Et.detach()), rel=1e-12)
    Et.backward()
    assert np.max(np.abs(F - (-x.grad.numpy()))) < 1e-10 * np.max(np.abs(F))
    del sub


# ---------------------------------------------------------------- closed forms
def test_bias_only_model():
    m = TINY
    w = np.zeros(oracle.af_weight_count(m))
    w[oracle.af_weight_slice(m, "fb4", 0)] = 0.37
    w[oracle.af_weight_slice(m, "fb4", 1)] = -1.25
    s = small_water()
    E, ae, F, V = oracle.af_compute(m, w, s.types, s.coords, s.box)
    n_o = int(np.sum(s.types == 0)); n_h = int(np.sum(s.types == 1))
    assert E == pytest.approx(0.37 * n_o - 1.25 * n_h, rel=1e-14)
    assert np.all(ae[s.types == 0] == 0.37) and np.all(ae[s.types == 1] == -1.25)
    assert np.all(F == 0) and np.all(V == 0)


def _np_mlp3(x, W1, b1, W2, b2, W3, b3):
    return np.tanh(np.tanh(np.tanh(x @ W1 + b1) @ W2 + b2) @ W3 + b3)


def _dimer_setup(m, r, w):
    x = np.array([[20.0, 20.0, 20.0], [20.0 + r * 0.6, 20.0 + r * 0.8, 20.0]])
    t = np.array([0, 1])
    box = np.full(3, 50.0)
    sw, _ = oracle.switch(r, m.rs, m.rc)
    s = sw / r
    emb = {k: w[oracle.af_weight_slice(m, k, tj)] for k in ("eW1", "eb1", "eW2", "eb2", "eW3", "eb3")
           for tj in (0,)}
    return x, t, box, s, sw


def _fit(m, w, t, D):
    g = lambda k: w[oracle.af_weight_slice(m, k, t)]
    y = np.tanh(D @ g("fW1").reshape(-1, m.f1) + g("fb1"))
    y = np.tanh(y @ g("fW2").reshape(m.f1, m.f2) + g("fb2"))
    y = np.tanh(y @ g("fW3").reshape(m.f2, m.f3) + g("fb3"))
    return float(y @ g("fW4") + g("fb4")[0])


def _emb(m, w, t, s):
    g = lambda k: w[oracle.af_weight_slice(m, k, t)]
    return _np_mlp3(np.array([s]), g("eW1").reshape(1, -1), g("eb1"), g("eW2").reshape(m.e1, m.e2),
                    g("eb2"), g("eW3").reshape(m.e2, m.m1), g("eb3"))


def test_dimer_without_attention_closed_form():
    """One neighbour each: T = R~ G^T / Nmax, so D = |R~|^2 G G[:M2]^T / Nmax^2 and
    |R~|^2 = 2 s^2."""
    m = replace(TINY, n_layers=0)
    w = blob(m, seed=3)
    r = 3.3
    x, t, box, s, sw = _dimer_setup(m, r, w)
    E = oracle.af_compute(m, w, t, x, box)[0]
    want = 0.0
    for centre, other in ((0, 1), (1, 0)):
        G = _emb(m, w, t[other], s)
        D = (2 * s * s / m.nmax ** 2) * np.outer(G, G[:m.m2]).reshape(-1)
        want += _fit(m, w, t[centre], D)
    assert E == pytest.approx(want, rel=1e-13, abs=1e-14)


def test_dimer_attention_with_zero_query_key():
    """One neighbour: the softmax has one entry, the gate is rh.rh = 1, so the
    layer is G <- LayerNorm(G + G Wv Wo + bo) whatever Wq and Wk are."""
    m = replace(TINY, n_layers=1)
    w = blob(m, seed=4)
    r = 2.2
    x, t, box, s, sw = _dimer_setup(m, r, w)
    E = oracle.af_compute(m, w, t, x, box)[0]
    Wv = w[oracle.af_weight_slice(m, "Wv", 0)].reshape(m.m1, m.hidden)
    Wo = w[oracle.af_weight_slice(m, "Wo", 0)].reshape(m.hidden, m.m1)
    bo = w[oracle.af_weight_slice(m, "bo", 0)]
    want = 0.0
    for centre, other in ((0, 1), (1, 0)):
        G = _emb(m, w, t[other], s)
        z = G + G @ Wv @ Wo + bo
        G = (z - z.mean()) / np.sqrt(z.var() + 1e-5)
        D = (2 * s * s / m.nmax ** 2) * np.outer(G, G[:m.m2]).reshape(-1)
        want += _fit(m, w, t[centre], D)
    assert E == pytest.approx(want, rel=1e-12)


def test_pair_beyond_cutoff_and_continuity():
    m = TINY
    w = blob(m, seed=5)
    box = np.full(3, 50.0)
    t = np.array([0, 1])
    e_alone = oracle.af_compute(m, w, t[:1], np.array([[20.0, 20, 20]]), box)[0] + \
        oracle.af_compute(m, w, t[1:], np.array([[20.0, 20, 20]]), box)[0]
    for r in (6.0, 6.5, 9.0):
        x = np.array([[20.0, 20, 20], [20.0 + r, 20, 20]])
        assert oracle.af_compute(m, w, t, x, box)[0] == pytest.approx(e_alone, abs=1e-14)
    # approaching rc from inside, E - E_alone vanishes at least as (rc - r)^3
    # (the switch is C^2 at rc); halving the gap must shrink it 8-fold or more
    d = [abs(oracle.af_compute(m, w, t, np.array([[20.0, 20, 20], [26.0 - h, 20, 20]]), box)[0] - e_alone)
         for h in (0.4, 0.2)]
    assert d[0] > 0 and d[1] / d[0] < 1.0 / 8.0


# ---------------------------------------------------------------- invariants
def test_translation_permutation_rotation():
    m = TINY
    w = blob(m)
    s = small_water()
    E, ae, F, V = oracle.af_compute(m, w, s.types, s.coords, s.box)
    # translation (atoms cross the periodic boundary)
    E2, _, F2, _ = oracle.af_compute(m, w, s.types, s.coords + np.array([3.7, -12.1, 40.3]), s.box)
    assert E2 == pytest.approx(E, rel=1e-12) and np.allclose(F2, F, atol=1e-12)
    # same-species permutation
    perm = np.arange(s.n)
    rng = np.random.default_rng(2)
    for t in (0, 1):
        idx = np.nonzero(s.types == t)[0]
        perm[idx] = rng.permutation(idx)
    E3, _, F3, _ = oracle.af_compute(m, w, s.types[perm], s.coords[perm], s.box)
    assert E3 == pytest.approx(E, rel=1e-12) and np.allclose(F3, F[perm], atol=1e-12)
    # cubic symmetry under PBC: (x, y, z) -> (y, -x, z) maps a cubic box onto itself
    R = np.array([[0, 1, 0], [-1, 0, 0], [0, 0, 1.0]])
    E4, _, F4, V4 = oracle.af_compute(m, w, s.types, s.coords @ R.T, s.box)
    assert E4 == pytest.approx(E, rel=1e-12) and np.allclose(F4, F @ R.T, atol=1e-12)
    assert np.allclose(V4, R @ V @ R.T, atol=1e-11)
    # arbitrary rotation of an isolated cluster
    x = s.coords - s.coords.mean(0)
    q = np.linalg.qr(rng.normal(size=(3, 3)))[0]
    big = np.full(3, 60.0)
    Ea, _, Fa, _ = oracle.af_compute(m, w, s.types, x + 30.0, big)
    Eb, _, Fb, _ = oracle.af_compute(m, w, s.types, x @ q.T + 30.0, big)
    assert Eb == pytest.approx(Ea, rel=1e-12) and np.allclose(Fb, Fa @ q.T, atol=1e-12)
    # zero net force
    assert np.max(np.abs(F.sum(0))) < 1e-13


# ---------------------------------------------------------------- NVE
def test_nve_second_order_and_reversible():
    m = replace(TINY, nmax=60)
    w = blob(m, seed=9, sigma=0.3)
    s = small_water(6, 8.0, 4)
    masses = np.array([15.999, 1.008])
    from synth import maxwell_boltzmann
    v0 = maxwell_boltzmann(masses[s.types], 300.0, 1)
    flucts = []
    for dt in (0.5, 0.25):
        n = int(round(10.0 / dt))
        _, _, ep, ek = oracle.af_md(m, w, s.types, masses, s.coords, v0, s.box, n, dt)
        etot = ep + ek
        flucts.append(np.max(np.abs(etot - etot[0])))
    ratio = flucts[0] / flucts[1]
    assert 3.0 < ratio < 5.0, (flucts, ratio)
    # time reversal: run forward, flip velocities, run back
    x1, v1, _, _ = oracle.af_md(m, w, s.types, masses, s.coords, v0, s.box, 20, 0.5)
    x2, v2, _, _ = oracle.af_md(m, w, s.types, masses, x1, -v1, s.box, 20, 0.5)
    assert np.max(np.abs(x2 - s.coords)) < 1e-9
    assert np.max(np.abs(v2 + v0)) < 1e-11


# ---------------------------------------------------------------- DP group
def test_group_equals_full_model_when_the_rest_is_beyond_the_cutoff():
    """Members in one corner of a large box, non-members more than rc away:
    the full model's energies and forces on the members (its own neighbour
    search over every atom) must equal the group evaluation, and the group
    evaluation of every atom must equal the full model."""
    m = TINY
    w = blob(m, seed=13)
    a = small_water(6, 8.0, 4)
    b = small_water(6, 8.0, 9)
    box = np.full(3, 40.0)
    xa = a.coords % 8.0 + 1.0                   # members inside [1, 9]^3
    xb = b.coords % 8.0 + 22.0                  # others inside [22, 30]^3: > 6 A away
    x = np.concatenate([xa, xb])
    t = np.concatenate([a.types, b.types]).astype(np.int32)
    mask = np.arange(len(t)) < len(xa)
    E, ae, F, V = oracle.af_compute(m, w, t, x, box)
    Eg, aeg, Fg, Vg = oracle.af_compute_group(m, w, t, x, box, mask)
    assert np.allclose(aeg[mask], ae[mask], rtol=0, atol=1e-13)
    assert np.allclose(Fg[mask], F[mask], rtol=0, atol=1e-13)
    assert np.all(aeg[~mask] == 0) and np.all(Fg[~mask] == 0)
    assert Eg == pytest.approx(ae[mask].sum(), rel=1e-13)
    E2, ae2, F2, V2 = oracle.af_compute_group(m, w, t, x, box, np.ones(len(t), bool))
    assert E2 == E and np.array_equal(F2, F) and np.array_equal(V2, V)


def test_group_forces_are_central_differences_of_the_group_energy():
    """Non-members sit among the members (mixed in one box): the group energy
    must not see them, and its forces must be its own gradient."""
    m = TINY
    w = blob(m, seed=17)
    s = small_water(10, 9.5, 6)
    mask = np.zeros(s.n, bool)
    mask[: 3 * 6] = True                       # the first six molecules
    E, ae, F, V = oracle.af_compute_group(m, w, s.types, s.coords, s.box, mask)
    h = 1e-4
    for i in (0, 4, 13):
        for k in range(3):
            xp = s.coords.copy(); xp[i, k] += h
            xm = s.coords.copy(); xm[i, k] -= h
            fd = -(oracle.af_compute_group(m, w, s.types, xp, s.box, mask)[0]
                   - oracle.af_compute_group(m, w, s.types, xm, s.box, mask)[0]) / (2 * h)
            assert abs(fd - F[i, k]) < 1e-7 * np.sqrt(np.mean(F[mask] ** 2)) + 1e-10
    # moving a non-member changes nothing
    x2 = s.coords.copy()
    x2[~mask] += 0.37
    E2 = oracle.af_compute_group(m, w, s.types, x2, s.box, mask)[0]
    assert E2 == E


# ---------------------------------------------------------------- sampled forces
def _subset_case(name):
    if name == "water64":              # the config-1 model: nmax 46 truncates every list
        return C.WATER64_MODEL, C.water64()
    if name == "water96_small_box":    # 9.86 A box < 2 rc: several images of one atom
        return replace(C.ATTN_MODEL, n_layers=1), serving_system(96, 5)
    # 700 atoms, nmax lowered to 80 (about 90 lie within rc): lists truncate
    return replace(C.ATTN_MODEL, n_layers=1, nmax=80), serving_system(700, 9)


@pytest.mark.parametrize("name", ["water64", "water96_small_box", "protein700_truncated"])
def test_forces_subset_equals_the_whole_system_forces(name):
    """The sampled-force assembly used at 24,000 and 100,000 atoms (pair
    gradients of the sample and of every centre that lists a sampled atom,
    gathered in numpy) against the whole-system forces of the C oracle, which
    central differences pin.  The sample holds the most crowded atom, whose
    list is truncated, and random atoms; the cases cover truncated lists and a
    box whose atoms see several images of one neighbour."""
    m, s = _subset_case(name)
    w = blob(m, seed=C.WEIGHT_SEED)
    cnt = oracle.neighbours(s.coords, s.box, m.rc, 1)[0]
    if name != "water96_small_box":
        assert np.sum(cnt > m.nmax) > 0          # truncation is active
    else:
        nj = oracle.neighbours(s.coords, s.box, m.rc, 4 * m.nmax)[1]
        assert any(len(set(nj[i, :cnt[i]].tolist())) < cnt[i] for i in range(s.n))
    rng = np.random.default_rng(5)
    sample = np.unique(np.concatenate([rng.choice(s.n, 9, replace=False),
                                       [int(np.argmax(cnt)), 0]])).astype(np.int32)
    F_sub = oracle.af_forces_subset(m, w, s.types, s.coords, s.box, sample)
    E, ae, F, V = oracle.af_compute(m, w, s.types, s.coords, s.box)
    fr = np.sqrt(np.mean(F ** 2))
    assert np.max(np.abs(F_sub - F[sample])) <= 1e-12 * fr
    # the sampled atomic energies come from the same per-centre routine
    ae_sub = oracle.af_atoms(m, w, s.types, s.coords, s.box, sample)["atom_e"]
    assert np.max(np.abs(ae_sub - ae[sample])) <= 1e-12 * np.max(np.abs(ae))
