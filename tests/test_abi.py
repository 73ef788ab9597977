"""The C ABI without a GPU: the library loads, exports every function that
include/dp.h declares, the ctypes struct matches the C layout, and the
host-only calls (weight count, argument checks) behave."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import paper_2602_02234_b300 as dp
from synth import configs as CF

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dp.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dp_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    out = subprocess.run(["nm", "-D", "--defined-only", dp.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (dp_\w+)", out))
    names = declared_functions()
    assert len(names) >= 12
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = dp.lib()
    for n in names:
        assert hasattr(lib, n)


def test_struct_layout_matches_c():
    code = r'''
#include <stdio.h>
#include <stddef.h>
#include "dp.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(dp_model_desc), offsetof(dp_model_desc, rcut),
         offsetof(dp_model_desc, angle_rcut), offsetof(dp_model_desc, f1),
         offsetof(dp_model_desc, skin), offsetof(dp_model_desc, rebuild_every),
         offsetof(dp_model_desc, fit_heads), offsetof(dp_model_desc, message_passing));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(src, "w").write(code)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    M = dp.ModelDesc
    assert vals == [C.sizeof(M), M.rcut.offset, M.angle_rcut.offset, M.f1.offset, M.skin.offset,
                    M.rebuild_every.offset, M.fit_heads.offset, M.message_passing.offset]


@pytest.mark.parametrize("model", [CF.WATER64_MODEL, CF.ATTN_MODEL])
def test_weight_count_matches_oracle(model):
    for prec in (dp.PREC_PLAIN_F64, dp.PREC_PLAIN_F32, dp.PREC_FUSED):
        assert dp.weight_count(dp.model_desc(model, prec)) == oracle.af_weight_count(model)


def test_argument_errors_without_gpu():
    d = dp.model_desc(CF.WATER64_MODEL, dp.PREC_PLAIN_F32)
    d.m2 = d.m1 + 1
    with pytest.raises(dp.DPError) as e:
        dp.weight_count(d)
    assert e.value.code == dp.DP_ERR_ARG
    d = dp.model_desc(CF.WATER64_MODEL, dp.PREC_PLAIN_F32)
    w = np.zeros(dp.weight_count(d) - 1)
    with pytest.raises(dp.DPError) as e:
        dp.DeepPotential(d, [0, 1, 1], [10.0, 10, 10], w)
    assert e.value.code == dp.DP_ERR_ARG and "weight blob" in str(e.value)
    w = np.zeros(dp.weight_count(d))
    with pytest.raises(dp.DPError) as e:
        dp.DeepPotential(d, [0, 5, 1], [10.0, 10, 10], w)
    assert e.value.code == dp.DP_ERR_ARG and "species" in str(e.value)
    with pytest.raises(dp.DPError) as e:
        dp.DeepPotential(d, [0, 1, 1], [10.0, -1, 10], w)
    assert e.value.code == dp.DP_ERR_ARG


def test_weight_count_with_fitting_heads_matches_the_oracle():
    from dataclasses import replace
    from synth import configs as C
    for k in (1, 2, 4):
        m = replace(C.ATTN_MODEL, fit_heads=k)
        assert dp.weight_count(dp.model_desc(m, dp.PREC_PLAIN_F32)) == oracle.af_weight_count(m)
    m = replace(C.ATTN_MODEL, fit_heads=3)
    w = np.arange(oracle.af_weight_count(m), dtype=np.float64)
    w0, d0 = oracle.af_head_blob(m, w, 0)
    w2, _ = oracle.af_head_blob(m, w, 2)
    n1 = oracle.af_weight_count(d0)
    assert len(w0) == len(w2) == n1 and d0["fit_heads"] == 1
    fl = oracle.af_weight_count(m) - n1
    assert np.array_equal(w0, w[:n1]) and np.array_equal(w2[n1 - fl // 2:], w[-(fl // 2):])


def test_message_passing_desc_and_weight_count():
    from dataclasses import replace
    from synth import configs as C
    m = replace(C.ATTN_MODEL, message_passing=1)
    for prec in (dp.PREC_PLAIN_F64, dp.PREC_PLAIN_F32):
        assert dp.weight_count(dp.model_desc(m, prec)) == oracle.af_weight_count(m)
    d = dp.model_desc(m, dp.PREC_PLAIN_F32)
    d.fit_heads = 2
    with pytest.raises(dp.DPError) as e:
        dp.weight_count(d)
    assert e.value.code == dp.DP_ERR_ARG
    d = dp.model_desc(C.GRAPH_MODEL, dp.PREC_PLAIN_F32)
    d.message_passing = 1
    with pytest.raises(dp.DPError) as e:
        dp.weight_count(d)
    assert e.value.code == dp.DP_ERR_ARG


def test_library_is_built_from_the_current_sources():
    """libdp.so must be newer than every source and header under csrc/ (a
    stale library would test and time old code)."""
    import glob
    pkg = os.path.join(ROOT, "paper_2602_02234_b300")
    lib_path = os.path.join(pkg, "libdp.so")
    srcs = glob.glob(os.path.join(pkg, "csrc", "*")) + [os.path.join(ROOT, "include", "dp.h")]
    newest = max(os.path.getmtime(f) for f in srcs)
    assert os.path.getmtime(lib_path) >= newest, "libdp.so is older than its sources: rebuild"
