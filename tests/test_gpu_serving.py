"""Continuous batching (dp_server): a system's trajectory is the same alone and
in a mix (bitwise: per-atom work and per-system reductions do not depend on the
batch), equals the single-system dp_step path, admission respects the memory
capacity, requests that arrive while others run are admitted at once, and the
served energies, forces and trajectories agree with the FP64 oracle."""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import paper_2602_02234_b300 as dp
from synth import configs as C, maxwell_boltzmann, normal_blob, serving_system

pytestmark = pytest.mark.gpu

M = C.ATTN_MODEL
M_MP = replace(C.ATTN_MODEL, message_passing=1)


def weights(model=M):
    return normal_blob(oracle.af_weight_count(model), C.WEIGHT_SEED)


def masses():
    return serving_system(96, 1).masses


def server(model=M, **kw):
    return dp.Server(dp.model_desc(model, dp.PREC_FUSED), weights(model), masses(), dt_fs=C.DT_FS,
                     **kw)


def vel(s, seed):
    return maxwell_boltzmann(masses()[s.types], 300.0, seed)


def run_to_end(srv, ids):
    out = {}
    for _ in range(10000):
        srv.tick()
        for k, rid in ids.items():
            if k not in out:
                r = srv.poll(rid)
                if r is not None:
                    out[k] = r
        if len(out) == len(ids):
            return out
    raise AssertionError("requests did not finish")


@pytest.mark.parametrize("model", [M, M_MP], ids=["attention", "message_passing"])
def test_alone_equals_mixed_and_single_context(model):
    """With message passing too: an atom's messages come from its own system
    and the adjoint's reverse sums visit slots in (i, p) order, whatever the
    batch holds."""
    target = serving_system(320, 3)
    others = [serving_system(n, 10 + n) for n in (96, 700, 1500)]
    v_t = vel(target, 1)
    # alone
    srv = server(model, max_slots=8)
    alone = run_to_end(srv, {"t": srv.submit(target.types, target.box, target.coords, v_t, 30)})["t"]
    srv.close()
    # in a mix: others already running, one joins later, some leave early
    srv = server(model, max_slots=8)
    ids = {"o0": srv.submit(others[0].types, others[0].box, others[0].coords, vel(others[0], 2), 12),
           "o1": srv.submit(others[1].types, others[1].box, others[1].coords, vel(others[1], 3), 40)}
    for _ in range(5):
        srv.tick()
    ids["t"] = srv.submit(target.types, target.box, target.coords, v_t, 30)
    for _ in range(3):
        srv.tick()
    ids["o2"] = srv.submit(others[2].types, others[2].box, others[2].coords, vel(others[2], 4), 10)
    mixed = run_to_end(srv, ids)
    st = srv.stats()
    srv.close()
    assert st["max_resident"] >= 3
    assert np.array_equal(alone[0], mixed["t"][0])
    assert np.array_equal(alone[1], mixed["t"][1])
    assert np.array_equal(alone[2], mixed["t"][2])
    # the same run through a single-system context
    pot = dp.DeepPotential(dp.model_desc(model, dp.PREC_FUSED), target.types, target.box,
                           weights(model), masses=masses())
    x, v = target.coords.copy(), v_t.copy()
    tr = pot.step(30, C.DT_FS, coords=x, vel=v, energies=True)
    assert np.max(np.abs(x - alone[0])) < 1e-9
    assert np.max(np.abs(tr - alone[2])) < 1e-6 * np.max(np.abs(tr))


def test_admission_respects_memory_capacity():
    systems = [serving_system(600, 20 + k) for k in range(3)]
    srv = server(max_slots=8, max_atoms=1000)
    assert srv.capacity()[0] == 1000
    ids = {k: srv.submit(s.types, s.box, s.coords, vel(s, k), 6) for k, s in enumerate(systems)}
    out = run_to_end(srv, ids)
    st = srv.stats()
    srv.close()
    assert st["max_resident_atoms"] <= 1000 and st["max_resident"] == 1
    assert st["waits_for_memory"] > 0
    done = sorted((out[k][3]["tick_admitted"], out[k][3]["tick_done"]) for k in out)
    for (a0, d0), (a1, d1) in zip(done, done[1:]):
        assert a1 >= d0                    # one after another
    with pytest.raises(dp.DPError) as e:
        s = serving_system(1500, 9)
        srv2 = server(max_slots=2, max_atoms=1000)
        srv2.submit(s.types, s.box, s.coords, vel(s, 1), 2)
    assert e.value.code == dp.DP_ERR_OOM


def test_late_arrival_overlaps_running_work():
    a, b = serving_system(900, 31), serving_system(250, 32)
    srv = server(max_slots=4)
    ia = srv.submit(a.types, a.box, a.coords, vel(a, 1), 30)
    for _ in range(10):
        srv.tick()
    ib = srv.submit(b.types, b.box, b.coords, vel(b, 2), 5)
    out = run_to_end(srv, {"a": ia, "b": ib})
    srv.close()
    assert out["b"][3]["tick_admitted"] < out["a"][3]["tick_done"]
    assert out["b"][3]["tick_done"] < out["a"][3]["tick_done"]


def test_served_systems_match_the_oracle():
    """Served results against the FP64 oracle, not only against other GPU runs.

    Four uneven systems (96 to 1,200 atoms; the 96-atom box is smaller than
    2 rc) share the batch, admitted at different ticks.  The integration is
    FP64, so a one-step request returns the forces it used: the first drift
    gives F(x0) = (x1 - x0 - dt v0) 2 m / (dt^2 kappa) and the closing kick
    F(x1) = 2 m (v1 - v0) / (dt kappa) - F(x0).  Both are held to the fused
    bound (2e-2 of the oracle's force RMS) and the energy of the step to 1e-3.
    Four-step requests are compared with the oracle's own velocity-Verlet
    run: per-step energies within 1e-3, and positions within the drift that a
    force error at the bound can cause, n^2 dt^2 kappa / m_min times it."""
    m, w, ms = M, weights(), masses()
    kappa = oracle.KAPPA
    dt = C.DT_FS
    systems = [serving_system(96, 41), serving_system(320, 42), serving_system(700, 43),
               serving_system(1200, 44)]
    steps = [1, 4, 1, 4]
    v0 = [vel(s, 50 + k) for k, s in enumerate(systems)]
    srv = server(max_slots=8)
    ids = {}
    for k in (0, 3):
        ids[k] = srv.submit(systems[k].types, systems[k].box, systems[k].coords, v0[k], steps[k])
    srv.tick()
    for k in (1, 2):
        ids[k] = srv.submit(systems[k].types, systems[k].box, systems[k].coords, v0[k], steps[k])
    out = run_to_end(srv, ids)
    srv.close()
    for k, s in enumerate(systems):
        x, v, e, _ = out[k]
        mass = ms[s.types][:, None]
        _, _, F0o, _ = oracle.af_compute(m, w, s.types, s.coords, s.box)
        fr = frms(F0o)
        if steps[k] == 1:
            F0 = (x - s.coords - dt * v0[k]) * 2.0 * mass / (dt * dt * kappa)
            assert np.max(np.abs(F0 - F0o)) <= 2e-2 * fr, k
            E1o, _, F1o, _ = oracle.af_compute(m, w, s.types, x, s.box)
            F1 = 2.0 * mass * (v - v0[k]) / (dt * kappa) - F0
            assert np.max(np.abs(F1 - F1o)) <= 2e-2 * frms(F1o), k
            assert abs(e[0, 0] - E1o) <= 1e-3 * abs(E1o), k
        else:
            n = steps[k]
            xo, vo, epo, eko = oracle.af_md(m, w, s.types, ms, s.coords, v0[k], s.box, n, dt)
            assert np.all(np.abs(e[:, 0] - epo) <= 1e-3 * np.abs(epo)), k
            bound = n * n * dt * dt * kappa / np.min(ms[s.types]) * 2e-2 * fr
            assert np.max(np.abs(x - xo)) <= bound, (k, np.max(np.abs(x - xo)), bound)


def test_served_message_passing_forces_match_the_oracle():
    """The model with cross-atom messages in a mixed batch: one-step requests
    return the forces they used (FP64 integration), held to the fused bound
    against the whole-system message-passing oracle; the step's energy to the
    2e-3 that the extra 16-bit rounding of the messages allows."""
    m, w, ms = M_MP, weights(M_MP), masses()
    kappa, dt = oracle.KAPPA, C.DT_FS
    systems = [serving_system(96, 61), serving_system(700, 62), serving_system(320, 63)]
    v0 = [vel(s, 70 + k) for k, s in enumerate(systems)]
    srv = server(M_MP, max_slots=4)
    ids = {0: srv.submit(systems[0].types, systems[0].box, systems[0].coords, v0[0], 1)}
    srv.tick()
    for k in (1, 2):
        ids[k] = srv.submit(systems[k].types, systems[k].box, systems[k].coords, v0[k], 1)
    out = run_to_end(srv, ids)
    srv.close()
    for k, s in enumerate(systems):
        x, v, e, _ = out[k]
        mass = ms[s.types][:, None]
        _, _, F0o, _ = oracle.af_compute(m, w, s.types, s.coords, s.box)
        F0 = (x - s.coords - dt * v0[k]) * 2.0 * mass / (dt * dt * kappa)
        assert np.max(np.abs(F0 - F0o)) <= 2e-2 * frms(F0o), k
        E1o, _, F1o, _ = oracle.af_compute(m, w, s.types, x, s.box)
        F1 = 2.0 * mass * (v - v0[k]) / (dt * kappa) - F0
        assert np.max(np.abs(F1 - F1o)) <= 2e-2 * frms(F1o), k
        assert abs(e[0, 0] - E1o) <= 2e-3 * abs(E1o), k


def frms(F):
    return float(np.sqrt(np.mean(F ** 2)))
