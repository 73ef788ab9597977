"""Pins of the FP64 graph-family oracle against facts that do not come from it:
central finite differences, the strain derivative, an independent PyTorch
autograd restatement, closed forms (bias-only fitting, no layers, a dimer with
one layer), invariants and the cutoff behaviour."""
from dataclasses import replace

import numpy as np
import pytest
import torch

import oracle
from synth import configs as C, normal_blob, water_box
from tests import gf_torch_ref

TINY = replace(C.GRAPH_MODEL, n_species=5, node=16, edge=8, n_layers=2, f1=12, f2=10, f3=8,
               nmax=40, na=10)


def blob(model, seed=3, sigma=0.3):
    return normal_blob(oracle.gf_weight_count(model), seed, sigma)


def small_system(n_mol=8, L=9.0, seed=3):
    s = water_box(n_mol, L, seed, min_oo=2.3)
    s.types = np.where(s.types == 0, 3, 0).astype(np.int32)   # O -> 3, H -> 0
    s.types[::5] = 1                                            # a few carbons
    return s


def fd(model, w, s, atoms, h=1e-4):
    out = np.zeros((len(atoms), 3))
    for q, i in enumerate(atoms):
        for a in range(3):
            xp = s.coords.copy(); xp[i, a] += h
            xm = s.coords.copy(); xm[i, a] -= h
            out[q, a] = -(oracle.gf_compute(model, w, s.types, xp, s.box)[0]
                          - oracle.gf_compute(model, w, s.types, xm, s.box)[0]) / (2 * h)
    return out


@pytest.mark.parametrize("case", ["water8", "water_small_box", "config3_sizes"])
def test_gf_forces_central_differences(case):
    if case == "water8":
        m, s = TINY, small_system()
    elif case == "water_small_box":
        m, s = TINY, small_system(4, 6.6, 5)        # many periodic images of each atom
    else:
        m, s = replace(C.GRAPH_MODEL, n_layers=2, nmax=60), small_system(6, 8.0, 7)
    w = blob(m)
    E, _, F, V = oracle.gf_compute(m, w, s.types, s.coords, s.box)
    atoms = [0, 3, 7]
    ref = fd(m, w, s, atoms)
    scale = float(np.sqrt(np.mean(F ** 2)))
    assert np.max(np.abs(ref - F[atoms])) < 1e-7 * scale + 1e-10
    assert np.max(np.abs(F.sum(0))) < 1e-12
    assert np.allclose(V, V.T, atol=1e-12)


def test_gf_virial_is_minus_strain_derivative():
    m, s = TINY, small_system()
    w = blob(m)
    E, _, F, V = oracle.gf_compute(m, w, s.types, s.coords, s.box)
    eps = 1e-6
    for a in range(3):
        def e_at(e):
            M = np.eye(3); M[a, a] += e
            return oracle.gf_compute(m, w, s.types, s.coords @ M.T, s.box * np.diag(M))[0]
        assert V[a, a] == pytest.approx(-(e_at(eps) - e_at(-eps)) / (2 * eps), abs=1e-8)


def test_gf_matches_torch_autograd_restatement():
    m, s = TINY, small_system()
    w = blob(m)
    E, ae, F, V = oracle.gf_compute(m, w, s.types, s.coords, s.box)
    x = torch.tensor(s.coords, dtype=torch.float64, requires_grad=True)
    Et = gf_torch_ref.energy(m.as_dict(), w, s.types, x, s.box)
    Et.backward()
    assert E == pytest.approx(float(Et.detach()), rel=1e-12)
    assert np.max(np.abs(F + x.grad.numpy())) <= 1e-10 * np.max(np.abs(F))


def test_gf_bias_only_and_no_layers():
    m, s = TINY, small_system()
    w = np.zeros(oracle.gf_weight_count(m))
    for t in range(m.n_species):
        w[oracle.gf_weight_slice(m, "c4", t)] = 0.1 * (t + 1)
    E, ae, F, V = oracle.gf_compute(m, w, s.types, s.coords, s.box)
    assert np.allclose(ae, 0.1 * (s.types + 1), rtol=0, atol=0)
    assert np.all(F == 0)
    # no layers: nodes are the species rows, nothing depends on positions
    m0 = replace(TINY, n_layers=0)
    w0 = blob(m0)
    E0, ae0, F0, V0 = oracle.gf_compute(m0, w0, s.types, s.coords, s.box)
    assert np.all(F0 == 0)
    Wt = w0[oracle.gf_weight_slice(m0, "Wt")].reshape(m0.n_species, m0.node)
    for i in (0, 1, 5):
        t = s.types[i]
        g = lambda k: w0[oracle.gf_weight_slice(m0, k, t)]
        y = np.tanh(Wt[t] @ g("F1").reshape(m0.node, -1) + g("c1"))
        y = np.tanh(y @ g("F2").reshape(m0.f1, -1) + g("c2"))
        y = np.tanh(y @ g("F3").reshape(m0.f2, -1) + g("c3"))
        assert ae0[i] == pytest.approx(float(y @ g("F4") + g("c4")[0]), rel=1e-13)


def test_gf_dimer_one_layer_closed_form():
    """Two atoms, one layer: the edge and angle updates do not reach the energy,
    so e_i = fit(n_i + tanh([n_i, m_i] Wn + bn)) with
    m_i = sw/nmax * tanh(s w_e + b_e) * (n_j Wm)."""
    m = replace(TINY, n_layers=1)
    w = blob(m, seed=11)
    r = 2.7
    x = np.array([[10.0, 10.0, 10.0], [10.0 + 0.36 * r, 10.0 + 0.48 * r, 10.0 + 0.8 * r]])
    t = np.array([1, 3], dtype=np.int32)
    box = np.full(3, 40.0)
    E = oracle.gf_compute(m, w, t, x, box)[0]
    sw, _ = oracle.switch(r, m.rs, m.rc)
    s = sw / r
    W = lambda k, a=0: w[oracle.gf_weight_slice(m, k, a)]
    Wt = W("Wt").reshape(m.n_species, m.node)
    e0 = np.tanh(s * W("we") + W("be0"))
    want = 0.0
    for i, j in ((0, 1), (1, 0)):
        ni, nj = Wt[t[i]], Wt[t[j]]
        mi = sw / m.nmax * e0 * (nj @ W("Wm").reshape(m.node, m.edge))
        n1 = ni + np.tanh(np.concatenate([ni, mi]) @ W("Wn").reshape(m.node + m.edge, m.node) + W("bn"))
        y = np.tanh(n1 @ W("F1", t[i]).reshape(m.node, -1) + W("c1", t[i]))
        y = np.tanh(y @ W("F2", t[i]).reshape(m.f1, -1) + W("c2", t[i]))
        y = np.tanh(y @ W("F3", t[i]).reshape(m.f2, -1) + W("c3", t[i]))
        want += float(y @ W("F4", t[i]) + W("c4", t[i])[0])
    assert E == pytest.approx(want, rel=1e-13)


def test_gf_invariants():
    m, s = TINY, small_system()
    w = blob(m)
    E, _, F, V = oracle.gf_compute(m, w, s.types, s.coords, s.box)
    E2, _, F2, _ = oracle.gf_compute(m, w, s.types, s.coords + np.array([4.1, -9.3, 22.2]), s.box)
    assert E2 == pytest.approx(E, rel=1e-12) and np.allclose(F2, F, atol=1e-12)
    rng = np.random.default_rng(4)
    perm = np.arange(s.n)
    for t in np.unique(s.types):
        idx = np.nonzero(s.types == t)[0]
        perm[idx] = rng.permutation(idx)
    E3, _, F3, _ = oracle.gf_compute(m, w, s.types[perm], s.coords[perm], s.box)
    assert E3 == pytest.approx(E, rel=1e-12) and np.allclose(F3, F[perm], atol=1e-12)
    x = s.coords - s.coords.mean(0)
    q = np.linalg.qr(rng.normal(size=(3, 3)))[0]
    big = np.full(3, 60.0)
    Ea, _, Fa, _ = oracle.gf_compute(m, w, s.types, x + 30.0, big)
    Eb, _, Fb, _ = oracle.gf_compute(m, w, s.types, x @ q.T + 30.0, big)
    assert Eb == pytest.approx(Ea, rel=1e-12) and np.allclose(Fb, Fa @ q.T, atol=1e-12)


def test_gf_pair_beyond_cutoff():
    m = TINY
    w = blob(m, seed=5)
    box = np.full(3, 50.0)
    t = np.array([0, 3], dtype=np.int32)
    alone = sum(oracle.gf_compute(m, w, t[k:k + 1], np.array([[20.0, 20, 20]]), box)[0] for k in (0, 1))
    for r in (6.0, 7.5):
        x = np.array([[20.0, 20, 20], [20.0 + r, 20, 20]])
        assert oracle.gf_compute(m, w, t, x, box)[0] == pytest.approx(alone, abs=1e-14)
    # E - E_alone is linear in sw here (messages are sw-weighted), and sw
    # vanishes as (rc - r)^3 (plus higher orders): halving the gap shrinks it by
    # about 8 (0.133 at these gaps); a switch that is not C^2 would give >= 1/4
    d = [abs(oracle.gf_compute(m, w, t, np.array([[20.0, 20, 20], [26.0 - h, 20, 20]]), box)[0] - alone)
         for h in (0.4, 0.2)]
    assert d[0] > 0 and d[1] / d[0] < 0.15


def test_stored_24k_result_is_current_and_consistent():
    """The stored whole-system oracle result at 24,000 atoms (the expected
    value of the full-size graph-family GPU test) belongs to the current
    generators and weights (input digest), and obeys the model's invariants:
    zero net force and a symmetric virial."""
    import json
    from tests.golden import make_gf_protein24k as g
    m, s, w = g.inputs()
    with open(g.OUT) as f:
        ref = json.load(f)
    assert ref["inputs_sha256"] == g.digest(s, w)
    assert len(ref["sample"]) >= 200 and len(ref["forces"]) == len(ref["sample"])
    V = np.array(ref["virial"])
    assert np.max(np.abs(V - V.T)) <= 1e-9 * np.linalg.norm(V)
    assert np.max(np.abs(ref["net_force"])) <= 1e-9 * ref["force_rms"] * np.sqrt(s.n)
    assert np.array_equal(np.array(ref["sample"]), g.sample(s, m))
