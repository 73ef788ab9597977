"""dp_neighbour_list_noalloc: the allocation-free neighbour lists, for callers
that cannot allocate device memory.  Checked through the C ABI against the
lists of the regular entry points (dp_compute + dp_get_neighbours), on two
calls in a row on the same stream -- the second on a different system, so a
stale scratch array from the first call would show.  Integer results: exact.
"""
import numpy as np
import pytest

import oracle
import paper_2602_02234_b300 as dp
from synth import configs as C, normal_blob, serving_system

pytestmark = pytest.mark.gpu


def regular_lists(system, model):
    w = normal_blob(oracle.af_weight_count(model), C.WEIGHT_SEED)
    pot = dp.DeepPotential(dp.model_desc(model, dp.PREC_PLAIN_F32), system.types, system.box, w)
    pot.compute(system.coords)
    out = pot.neighbours()
    pot.close()
    return out


def test_noalloc_matches_regular_entry_points_twice():
    import torch
    stream = torch.cuda.Stream()
    cases = [(C.water64(), C.WATER64_MODEL), (serving_system(96, 5), C.ATTN_MODEL),
             (serving_system(700, 9), C.ATTN_MODEL)]
    first = None
    for k, (s, m) in enumerate(cases):
        want_cnt, want_j, want_img = regular_lists(s, m)
        x = torch.tensor(s.coords, dtype=torch.float64, device="cuda")
        for call in range(2):
            cnt, j, img = dp.neighbour_list_noalloc(x, s.box, m.rc, m.nmax, stream=stream)
            torch.cuda.synchronize()
            assert np.array_equal(cnt.cpu().numpy(), want_cnt)
            assert np.array_equal(j.cpu().numpy(), want_j)
            assert np.array_equal(img.cpu().numpy(), want_img)
        if first is None:
            first = (x, s, m, want_j)
    # back to the first system after the others have used the scratch array
    x, s, m, want_j = first
    cnt, j, img = dp.neighbour_list_noalloc(x, s.box, m.rc, m.nmax, stream=stream)
    torch.cuda.synchronize()
    assert np.array_equal(j.cpu().numpy(), want_j)


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch
    x = torch.zeros((1025, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(dp.DPError) as e:
        dp.neighbour_list_noalloc(x, [50.0, 50.0, 50.0], 6.0, 120)
    assert e.value.code == dp.DP_ERR_ARG and "1024" in str(e.value)
