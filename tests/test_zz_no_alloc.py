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


def _raw_call(x, box, rc, nmax):
    """The C entry point itself, so that the outputs of a failed call can be read."""
    import ctypes
    import torch
    n = x.shape[0]
    j = torch.full((n, nmax), 7, dtype=torch.int32, device=x.device)
    img = torch.full((n, nmax, 3), 7, dtype=torch.int32, device=x.device)
    cnt = torch.full((n,), 7, dtype=torch.int32, device=x.device)
    b = np.ascontiguousarray(box, dtype=np.float64)
    rc_ = dp.lib().dp_neighbour_list_noalloc(ctypes.c_void_p(x.data_ptr()), n,
                                             b.ctypes.data, float(rc), int(nmax),
                                             ctypes.c_void_p(j.data_ptr()),
                                             ctypes.c_void_p(img.data_ptr()),
                                             ctypes.c_void_p(cnt.data_ptr()), None)
    torch.cuda.synchronize()
    return rc_, cnt.cpu().numpy(), j.cpu().numpy(), img.cpu().numpy()


def test_noalloc_overflow_is_reported_and_the_next_call_starts_clean():
    """215 atoms in an 8 A box (about 380 within 6 A on average, so some atoms
    have more than the 384 the scratch array holds): the call returns
    DP_ERR_NLIST_OVERFLOW, the atoms that overflowed report 385 with empty
    rows, and every other atom's list is the oracle's.  A box of 1 A, where an
    atom's own images alone exceed the limit, is refused before any launch.
    A normal system afterwards gets the regular lists: the status word of the
    shared scratch array was cleared."""
    import torch
    rng = np.random.default_rng(17)
    box = np.full(3, 8.0)
    xs = rng.uniform(0.0, 8.0, size=(215, 3))
    ocnt, onj, oimg, _ = oracle.neighbours(xs, box, 6.0, 384)
    over = ocnt > 384
    assert over.any() and (~over).any()
    x = torch.tensor(xs, dtype=torch.float64, device="cuda")
    rc_, cnt, j, img = _raw_call(x, box, 6.0, 384)
    assert rc_ == dp.DP_ERR_NLIST_OVERFLOW
    assert np.all(cnt[over] == 385)
    assert np.all(j[over] == -1) and np.all(img[over] == 0)
    assert np.array_equal(cnt[~over], ocnt[~over])
    assert np.array_equal(j[~over], onj[~over]) and np.array_equal(img[~over], oimg[~over])
    # own images alone beyond the limit: refused on the host
    with pytest.raises(dp.DPError) as e:
        dp.neighbour_list_noalloc(x[:4].contiguous(), [1.0, 1.0, 1.0], 6.0, 46)
    assert e.value.code == dp.DP_ERR_NLIST_OVERFLOW and "images" in str(e.value)
    # the shared scratch array's status word starts clean on the next call
    s, m = serving_system(96, 5), C.ATTN_MODEL
    want_cnt, want_j, want_img = regular_lists(s, m)
    xn = torch.tensor(s.coords, dtype=torch.float64, device="cuda")
    cnt, j, img = dp.neighbour_list_noalloc(xn, s.box, m.rc, m.nmax)
    torch.cuda.synchronize()
    assert np.array_equal(cnt.cpu().numpy(), want_cnt)
    assert np.array_equal(j.cpu().numpy(), want_j)
    assert np.array_equal(img.cpu().numpy(), want_img)
