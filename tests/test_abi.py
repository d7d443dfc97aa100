"""The C-ABI library loads and exports every function include/lbm_fs.h declares;
parameter validation happens on the host before any allocation (no GPU
needed for either)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1201_0351_gb300 import lbm_fs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(lbm_fs_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_every_declared_function_is_exported():
    lib = lbm_fs.load()
    names = declared_functions()
    assert {"lbm_fs_create", "lbm_fs_add_box", "lbm_fs_step", "lbm_fs_forces", "lbm_fs_read_fields"} <= names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding carries the same names
    assert all(hasattr(lbm_fs, n) for n in names if n not in ("lbm_fs_last_error_string", "lbm_fs_version",
                                                               "lbm_fs_noalloc_last_error_string"))


def _params(**kw):
    p = lbm_fs.lbm_fs_params()
    p.nx = p.ny = p.nz = 8
    p.tau = 0.6
    p.rho_gas = 1.0
    p.eps = 1e-2
    n = 8 ** 3
    keep = [np.ones(n, np.uint8), np.ones(n), np.ones(n)]
    p.init_flags, p.init_fill, p.init_rho = (a.ctypes.data for a in keep)
    for k, v in kw.items():
        if k in ("gravity", "body_accel"):
            getattr(p, k)[:] = v
        else:
            setattr(p, k, v)
    return p, keep


@pytest.mark.parametrize("bad", [dict(tau=0.5), dict(tau=0.4), dict(nx=0), dict(storage=7), dict(rho_gas=0.0),
                                 dict(eps=-1.0), dict(gravity=(0.0, 0.0, -0.05)), dict(init_flags=None),
                                 dict(sigma=-1e-3), dict(sigma=float("inf"))])
def test_invalid_parameters_rejected_before_allocation(bad):
    p, keep = _params(**bad)
    with pytest.raises(lbm_fs.LbmFsError) as e:
        lbm_fs.lbm_fs_create(p)
    assert e.value.code == lbm_fs.LBM_FS_EINVAL


def test_allocator_callbacks_must_come_in_pairs():
    p, keep = _params()
    p.dev_alloc = lbm_fs.DEV_ALLOC(lambda n, c: None)
    with pytest.raises(lbm_fs.LbmFsError) as e:
        lbm_fs.lbm_fs_create(p)
    assert e.value.code == lbm_fs.LBM_FS_EINVAL


def test_null_handle_calls_fail_cleanly():
    lib = lbm_fs.load()
    assert lib.lbm_fs_step(None, 1) == lbm_fs.LBM_FS_EINVAL
    assert lib.lbm_fs_sync(None) == lbm_fs.LBM_FS_EINVAL
    assert lib.lbm_fs_destroy(None) == lbm_fs.LBM_FS_EINVAL
    assert b"null" in lib.lbm_fs_last_error_string()


def test_noalloc_entry_rejects_bad_sizes_on_host():
    lib = lbm_fs.load()
    buf = ctypes.c_double(0.0)
    p = ctypes.cast(ctypes.pointer(buf), ctypes.c_void_p)
    assert lib.lbm_fs_liquid_mass_noalloc(p, p, -1, p, None) == lbm_fs.LBM_FS_EINVAL
    assert lib.lbm_fs_liquid_mass_noalloc(p, p, 268435457, p, None) == lbm_fs.LBM_FS_EINVAL
    assert lib.lbm_fs_liquid_mass_noalloc(None, p, 10, p, None) == lbm_fs.LBM_FS_EINVAL


def test_batch_rejects_bad_arguments_on_host():
    lib = lbm_fs.load()
    out = ctypes.c_void_p()
    p, keep = _params()
    assert lib.lbm_fs_batch_create(ctypes.byref(p), 0, ctypes.byref(out)) == lbm_fs.LBM_FS_EINVAL
    q, keep2 = _params(storage=lbm_fs.LBM_FS_F16S)
    arr = (lbm_fs.lbm_fs_params * 2)(p, q)
    assert lib.lbm_fs_batch_create(arr, 2, ctypes.byref(out)) == lbm_fs.LBM_FS_EINVAL
    assert b"storage" in lib.lbm_fs_last_error_string()
    big, keep3 = _params(nx=70000)
    assert lib.lbm_fs_batch_create(ctypes.byref(big), 1, ctypes.byref(out)) == lbm_fs.LBM_FS_EINVAL
    assert not out.value
    for name in ("lbm_fs_batch_step", "lbm_fs_batch_sync", "lbm_fs_batch_destroy"):
        fn = getattr(lib, name)
        assert (fn(None, 1) if name == "lbm_fs_batch_step" else fn(None)) == lbm_fs.LBM_FS_EINVAL
    cfg = lbm_fs.lbm_fs_batch_config_t(zb=9, bulk_blocks=0, list_cells=1024)
    assert lib.lbm_fs_batch_set_config(None, ctypes.byref(cfg)) == lbm_fs.LBM_FS_EINVAL
