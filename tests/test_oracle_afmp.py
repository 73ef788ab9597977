"""Pins of the FP64 oracle of the attention family with cross-atom message
passing (afmp_oracle.c) to facts other than itself:

* message weights Wm = 0, bm = 0 make the atom channel inert (U = 0): the
  model is then the base attention family, whose oracle is pinned on its own;
* a second reading in PyTorch with autograd forces (tests/af_torch_ref.py);
* forces are minus central differences of the energy;
* the receptive field is L neighbour hops: on a chain whose atoms see only
  their two nearest neighbours, atom 0's energy moves with atom L and is
  bitwise blind to atom L + 1;
* zero net force and a symmetric virial (translation and rotation invariance).
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

import oracle
from synth import configs as C, normal_blob, water_box
from tests import af_torch_ref

TINY = C.AttnModel(n_species=2, e1=6, e2=10, m1=16, m2=4, n_layers=2, hidden=16, heads=2,
                   f1=20, f2=18, f3=12, nmax=40, rc=6.0, rs=0.5)
TINY_MP = replace(TINY, message_passing=1)


def mp_blob(model, seed=7, sigma=0.1):
    return normal_blob(oracle.af_weight_count(model), seed, sigma)


def small_water(n_mol=8, L=9.0, seed=3):
    return water_box(n_mol, L, seed, min_oo=2.3)


def base_part(model_mp, w_mp):
    """The base model's blob inside a message-passing blob (Wt, Wm, bm removed)."""
    drop = [oracle.afmp_weight_slice(model_mp, "Wt")]
    for l in range(model_mp.n_layers):
        drop += [oracle.afmp_weight_slice(model_mp, "Wm", l), oracle.afmp_weight_slice(model_mp, "bm", l)]
    keep = np.ones(len(w_mp), bool)
    for s in drop:
        keep[s] = False
    return np.asarray(w_mp)[keep]


def test_blob_layout():
    m = TINY_MP
    base = oracle.af_weight_count(TINY)
    extra = m.n_species * m.m1 + m.n_layers * (m.m1 * m.m1 + m.m1)
    assert oracle.af_weight_count(m) == base + extra
    # Wt follows the embedding nets; Wm, bm close every layer block
    emb = m.n_species * (m.e1 * 2 + m.e1 * m.e2 + m.e2 + m.e2 * m.m1 + m.m1)
    assert oracle.afmp_weight_slice(m, "Wt").start == emb
    layer = 4 * m.m1 * m.hidden + m.m1 + m.m1 * m.m1 + m.m1
    wm0 = oracle.afmp_weight_slice(m, "Wm", 0)
    assert wm0.start == emb + m.n_species * m.m1 + 4 * m.m1 * m.hidden + m.m1
    assert oracle.afmp_weight_slice(m, "Wm", 1).start == wm0.start + layer
    assert oracle.afmp_weight_slice(m, "bm", 1).stop == oracle.afmp_weight_slice(m, "Wm", 1).stop + m.m1


def test_inert_message_weights_reduce_to_the_base_model():
    s = small_water()
    w = mp_blob(TINY_MP)
    for l in range(TINY_MP.n_layers):
        w[oracle.afmp_weight_slice(TINY_MP, "Wm", l)] = 0.0
        w[oracle.afmp_weight_slice(TINY_MP, "bm", l)] = 0.0
    E, ae, F, V = oracle.af_compute(TINY_MP, w, s.types, s.coords, s.box)
    Eb, aeb, Fb, Vb = oracle.af_compute(TINY, base_part(TINY_MP, w), s.types, s.coords, s.box)
    assert E == pytest.approx(Eb, rel=1e-13)
    assert np.max(np.abs(ae - aeb)) <= 1e-13 * np.max(np.abs(aeb))
    assert np.max(np.abs(F - Fb)) <= 1e-12 * np.max(np.abs(Fb))
    assert np.max(np.abs(V - Vb)) <= 1e-12 * np.max(np.abs(Vb))


def test_message_weights_change_the_energy():
    s = small_water()
    w = mp_blob(TINY_MP)
    E = oracle.af_compute(TINY_MP, w, s.types, s.coords, s.box)[0]
    w0 = w.copy()
    w0[oracle.afmp_weight_slice(TINY_MP, "bm", 1)] += 0.05
    assert abs(oracle.af_compute(TINY_MP, w0, s.types, s.coords, s.box)[0] - E) > 1e-6


@pytest.mark.parametrize("case", ["water8", "water64_3layers"])
def test_matches_torch_autograd_restatement(case):
    if case == "water8":
        s, m = small_water(), TINY_MP
    else:
        s, m = C.water64(), replace(TINY_MP, n_layers=3, nmax=46)
    w = mp_blob(m, seed=11)
    E, ae, F, V = oracle.af_compute(m, w, s.types, s.coords, s.box)
    x = torch.tensor(s.coords, dtype=torch.float64, requires_grad=True)
    Et = af_torch_ref.energy_mp(m.as_dict(), w, s.types, x, s.box)
    Et.backward()
    Ft = -x.grad.numpy()
    assert E == pytest.approx(float(Et.detach()), rel=1e-12)
    assert np.max(np.abs(F - Ft)) <= 1e-10 * np.max(np.abs(Ft))


def test_forces_are_minus_energy_differences():
    s = small_water()
    w = mp_blob(TINY_MP, seed=5, sigma=0.2)
    E, ae, F, V = oracle.af_compute(TINY_MP, w, s.types, s.coords, s.box)
    eps = 1e-5
    rng = np.random.default_rng(0)
    for i in rng.choice(s.n, 4, replace=False):
        for a in range(3):
            xp = s.coords.copy(); xp[i, a] += eps
            xm = s.coords.copy(); xm[i, a] -= eps
            Ep = oracle.af_compute(TINY_MP, w, s.types, xp, s.box)[0]
            Em = oracle.af_compute(TINY_MP, w, s.types, xm, s.box)[0]
            assert F[i, a] == pytest.approx(-(Ep - Em) / (2 * eps), abs=2e-7 * max(1.0, np.max(np.abs(F))))


def test_net_force_zero_and_virial_symmetric():
    s = small_water(n_mol=12, L=10.0, seed=9)
    w = mp_blob(TINY_MP, seed=2, sigma=0.2)
    E, ae, F, V = oracle.af_compute(TINY_MP, w, s.types, s.coords, s.box)
    scale = np.max(np.abs(F))
    assert np.max(np.abs(F.sum(0))) <= 1e-11 * scale * s.n
    assert np.max(np.abs(V - V.T)) <= 1e-11 * np.max(np.abs(V))


@pytest.mark.parametrize("layers", [1, 2, 3])
def test_receptive_field_is_layers_hops(layers):
    """A chain along x with spacing 0.7 rc: every atom sees exactly its two
    chain neighbours.  e_0 must depend on atom `layers` and not on atom
    `layers` + 1 (the halo is layers x rc); without message passing only on
    atom 1."""
    m = replace(TINY_MP, n_layers=layers)
    n = 10
    sp = 0.7 * m.rc
    box = np.array([n * sp + 4 * m.rc, 30.0, 30.0])
    x0 = np.zeros((n, 3))
    x0[:, 0] = 2 * m.rc + sp * np.arange(n)
    x0[:, 1] = 15.0 + 0.3 * np.sin(np.arange(n))
    x0[:, 2] = 15.0 + 0.3 * np.cos(np.arange(n))
    types = np.arange(n, dtype=np.int32) % 2
    w = mp_blob(m, seed=4, sigma=0.3)
    for l in range(layers):      # strong messages: each hop attenuates the signal ~30x
        sl = oracle.afmp_weight_slice(m, "Wm", l)
        w[sl] = np.random.default_rng(l).normal(0.0, 1.0, sl.stop - sl.start)
    ae0 = oracle.af_compute(m, w, types, x0, box)[1]

    def e0_after_moving(k):
        x = x0.copy()
        x[k, 1] += 1.0           # sideways: the chain's neighbour sets stay as they were
        return oracle.af_compute(m, w, types, x, box)[1][0]

    # far above FP64 rounding (1e-13 relative is ~500 ulps), and exactly zero beyond
    assert abs(e0_after_moving(layers) - ae0[0]) > 1e-13 * abs(ae0[0])
    assert e0_after_moving(layers + 1) == ae0[0]
    # without message passing the halo is one hop
    wb = w.copy()
    for l in range(layers):
        wb[oracle.afmp_weight_slice(m, "Wm", l)] = 0.0
        wb[oracle.afmp_weight_slice(m, "bm", l)] = 0.0
    e_base = oracle.af_compute(m, wb, types, x0, box)[1][0]
    x = x0.copy()
    x[2, 1] += 1.0
    assert oracle.af_compute(m, wb, types, x, box)[1][0] == e_base
