"""The C-ABI library loads on a machine without a GPU and exports every function that
include/mp.h declares; host-only entry points work without a device."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mp_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2201_04058_b300 import mp
    names = declared_functions()
    assert len(names) >= 20
    L = mp.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(names) == set(mp.EXPORTS)


def test_strerror_and_defaults():
    from paper_2201_04058_b300 import mp
    assert mp.strerror(mp.MP_ERR_OVERFLOW).startswith("path count")
    c = mp.mp_config_default()
    assert c.policy == mp.MP_POLICY_ATRAPOS and c.planner == mp.MP_PLAN_DP and c.force_bin_class == -1


def test_create_without_gpu_fails_cleanly():
    import torch
    from paper_2201_04058_b300 import mp
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(mp.MPError) as e:
        mp.mp_create(mp.mp_config_default())
    assert e.value.code in (mp.MP_ERR_CUDA, mp.MP_ERR_ARG)


def test_bad_arguments_rejected_on_host():
    from paper_2201_04058_b300 import mp
    with pytest.raises(mp.MPError):
        mp.mp_plan_chain([4, 0, 3], [1, 1])


def test_config_layout_and_new_fields():
    """The ctypes mp_config is exactly as large as the C struct: mp_config_default writes
    every field and nothing past the end; defaults of the budget, cache, Overlap-Tree and
    allocator fields."""
    import ctypes as C
    from paper_2201_04058_b300 import mp
    n = C.sizeof(mp.mp_config)
    buf = (C.c_uint8 * (n + 64))(*([0xAB] * (n + 64)))
    mp.lib().mp_config_default(C.cast(buf, C.POINTER(mp.mp_config)))
    assert all(b == 0xAB for b in bytes(buf)[n:]), "mp_config_default wrote past the ctypes struct"
    assert bytes(buf)[n - 8:n] == b"\0" * 8  # alloc_user, the last field, was written
    c = mp.mp_config_default()
    assert c.otree_construction == mp.MP_OTREE_ONLINE and c.cache_bytes == 0
    assert not c.alloc and not c.free and not c.alloc_user
    assert c.hbm_budget_bytes == 8 << 30


def test_allocator_hooks_must_come_in_pairs():
    from paper_2201_04058_b300 import mp
    c = mp.mp_config_default()
    fn = mp.ALLOC_FN(lambda n, s, u: None)
    c.alloc = C_cast(fn)
    with pytest.raises(mp.MPError) as e:
        mp.mp_create(c)
    assert e.value.code == mp.MP_ERR_ARG
    c = mp.mp_config_default()
    c.otree_construction = 7
    with pytest.raises(mp.MPError) as e:
        mp.mp_create(c)
    assert e.value.code == mp.MP_ERR_ARG


def C_cast(fn):
    import ctypes as C
    return C.cast(fn, C.c_void_p)
