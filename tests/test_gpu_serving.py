"""Continuous batching (dp_server): a system's trajectory is the same alone and
in a mix (bitwise: per-atom work and per-system reductions do not depend on the
batch), equals the single-system dp_step path, admission respects the memory
capacity, and requests that arrive while others run are admitted at once."""
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
