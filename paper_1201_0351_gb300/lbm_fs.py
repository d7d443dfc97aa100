"""Python binding of the C ABI in include/lbm_fs.h (argument marshalling only).

Every step of the method runs in the CUDA library libgb300_lbmfs.so; this
module only converts arguments.  PyTorch supplies device memory (its caching
allocator, through the dev_alloc / dev_free callbacks) and the CUDA stream.
There is no CPU fallback: a missing library or a missing GPU raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

LBM_FS_OK, LBM_FS_EINVAL, LBM_FS_ENOMEM, LBM_FS_ECUDA = 0, -1, -2, -3
LBM_FS_ESTATE, LBM_FS_EUNSTABLE, LBM_FS_ETIMEOUT, LBM_FS_EOVERFLOW = -4, -5, -6, -7
STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ESTATE", -5: "EUNSTABLE", -6: "ETIMEOUT",
                -7: "EOVERFLOW"}
LBM_FS_F64, LBM_FS_F32, LBM_FS_F16S = 0, 1, 2
STORAGE = {"f64": LBM_FS_F64, "f32": LBM_FS_F32, "f16s": LBM_FS_F16S}
FIELD_FLAGS, FIELD_FILL, FIELD_MASS, FIELD_RHO, FIELD_VEL, FIELD_F = 1, 2, 4, 8, 16, 32

DEV_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
DEV_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class lbm_fs_params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("periodic", C.c_uint32),
                ("tau", C.c_double), ("gravity", C.c_double * 3), ("body_accel", C.c_double * 3),
                ("rho_gas", C.c_double), ("eps", C.c_double), ("storage", C.c_int32),
                ("init_flags", C.c_void_p), ("init_fill", C.c_void_p), ("init_rho", C.c_void_p),
                ("init_vel", C.c_void_p), ("init_on_device", C.c_int32),
                ("dev_alloc", DEV_ALLOC), ("dev_free", DEV_FREE), ("alloc_ctx", C.c_void_p),
                ("stream", C.c_void_p), ("use_graphs", C.c_int32), ("sigma", C.c_double),
                ("wall_vel", C.c_double * 18), ("readings", C.c_uint32), ("normal_deadband", C.c_double),
                ("virtual_mass", C.c_double), ("force_mean", C.c_int32), ("neighbour_rule", C.c_int32)]


# bits of lbm_fs_params.readings, and the scenario keyword each one serves
READING_DEADBAND, READING_VIRTUAL_MASS, READING_FORCE_MEAN, READING_NEIGHBOUR_RULE = 1, 2, 4, 8
READINGS = {"deadband": ("normal_deadband", READING_DEADBAND, float),
            "virtual_mass": ("virtual_mass", READING_VIRTUAL_MASS, float),
            "force_mean": ("force_mean", READING_FORCE_MEAN, lambda v: int(bool(v))),
            "neighbour_rule": ("neighbour_rule", READING_NEIGHBOUR_RULE, lambda v: int(bool(v)))}


class lbm_fs_box(C.Structure):
    _fields_ = [("center", C.c_double * 3), ("half", C.c_double * 3), ("quat", C.c_double * 4),
                ("density_ratio", C.c_double), ("vel", C.c_double * 3), ("omega", C.c_double * 3),
                ("mode", C.c_int32), ("rot_axis", C.c_double * 3), ("lin_damping", C.c_double),
                ("shape", C.c_int32)]


class lbm_fs_body_state_t(C.Structure):
    _fields_ = [("F", C.c_double * 3), ("T", C.c_double * 3), ("S", C.c_double), ("center", C.c_double * 3),
                ("quat", C.c_double * 4), ("vel", C.c_double * 3), ("omega", C.c_double * 3)]


class lbm_fs_stats_t(C.Structure):
    _fields_ = [("step", C.c_int64), ("liquid_mass", C.c_double), ("mass0", C.c_double), ("covered", C.c_double),
                ("uncovered", C.c_double), ("lost_excess", C.c_double), ("n_interface", C.c_int64),
                ("n_filled", C.c_int64), ("n_emptied", C.c_int64), ("n_new_from_gas", C.c_int64),
                ("n_new_from_liquid", C.c_int64), ("n_pending", C.c_int64), ("status", C.c_uint32),
                ("kernel_launches", C.c_int64), ("wall_source", C.c_double), ("n_general", C.c_int64)]


class lbm_fs_batch_config_t(C.Structure):
    _fields_ = [("zb", C.c_int32), ("bulk_blocks", C.c_int32), ("list_cells", C.c_int32), ("lanes", C.c_int32),
                ("bulk_ms", C.c_double)]


EXPORTS = ("lbm_fs_create", "lbm_fs_destroy", "lbm_fs_add_box", "lbm_fs_step", "lbm_fs_forces", "lbm_fs_body_state",
           "lbm_fs_body_states",
           "lbm_fs_read_fields", "lbm_fs_stats", "lbm_fs_sync", "lbm_fs_kernel_times", "lbm_fs_last_error_string",
           "lbm_fs_version", "lbm_fs_liquid_mass_noalloc", "lbm_fs_noalloc_last_error_string",
           "lbm_fs_batch_create", "lbm_fs_batch_destroy", "lbm_fs_batch_tank", "lbm_fs_batch_step",
           "lbm_fs_batch_sync", "lbm_fs_batch_autotune", "lbm_fs_batch_set_config", "lbm_fs_batch_get_config",
           "lbm_fs_batch_kernel_times", "lbm_fs_batch_launches", "lbm_fs_fp64_rate")

_lib = None


class LbmFsError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__("%s failed: %s (%s)" % (where, STATUS_NAMES.get(code, code), msg))
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libgb300_lbmfs.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_needed else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libgb300_lbmfs.so is missing (build it with __graft_entry__.build())")
    lib = C.CDLL(path)
    P, I32, D = C.c_void_p, C.c_int32, C.POINTER(C.c_double)
    lib.lbm_fs_create.argtypes = [C.POINTER(lbm_fs_params), C.POINTER(P)]
    lib.lbm_fs_destroy.argtypes = [P]
    lib.lbm_fs_add_box.argtypes = [P, C.POINTER(lbm_fs_box), C.POINTER(I32)]
    lib.lbm_fs_step.argtypes = [P, I32]
    lib.lbm_fs_forces.argtypes = [P, I32, D, D, D, D]
    lib.lbm_fs_body_state.argtypes = [P, I32, C.POINTER(lbm_fs_body_state_t)]
    lib.lbm_fs_body_states.argtypes = [P, I32, I32, C.POINTER(lbm_fs_body_state_t)]
    lib.lbm_fs_read_fields.argtypes = [P, C.c_uint32, C.POINTER(C.c_void_p), I32]
    lib.lbm_fs_stats.argtypes = [P, C.POINTER(lbm_fs_stats_t)]
    lib.lbm_fs_sync.argtypes = [P]
    lib.lbm_fs_kernel_times.argtypes = [P, I32, D, C.POINTER(C.c_char_p), I32, C.POINTER(I32)]
    lib.lbm_fs_last_error_string.restype = C.c_char_p
    lib.lbm_fs_last_error_string.argtypes = []
    lib.lbm_fs_version.restype = I32
    lib.lbm_fs_liquid_mass_noalloc.argtypes = [P, P, C.c_int64, P, P]
    lib.lbm_fs_noalloc_last_error_string.restype = C.c_char_p
    lib.lbm_fs_noalloc_last_error_string.argtypes = []
    CFG = C.POINTER(lbm_fs_batch_config_t)
    lib.lbm_fs_batch_create.argtypes = [C.POINTER(lbm_fs_params), I32, C.POINTER(P)]
    lib.lbm_fs_batch_destroy.argtypes = [P]
    lib.lbm_fs_batch_tank.argtypes = [P, I32, C.POINTER(P)]
    lib.lbm_fs_batch_step.argtypes = [P, I32]
    lib.lbm_fs_batch_sync.argtypes = [P]
    lib.lbm_fs_batch_autotune.argtypes = [P, CFG]
    lib.lbm_fs_batch_set_config.argtypes = [P, CFG]
    lib.lbm_fs_batch_get_config.argtypes = [P, CFG]
    lib.lbm_fs_batch_kernel_times.argtypes = [P, I32, D, C.POINTER(C.c_char_p), I32, C.POINTER(I32)]
    lib.lbm_fs_batch_launches.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.lbm_fs_fp64_rate.argtypes = [I32, I32, D, P]
    for name in EXPORTS:
        if name not in ("lbm_fs_last_error_string", "lbm_fs_version", "lbm_fs_noalloc_last_error_string"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(code: int, where: str):
    if code != LBM_FS_OK:
        raise LbmFsError(code, where, load().lbm_fs_last_error_string().decode())


# ------------------------------------------------- C-ABI-named entry points

def lbm_fs_create(params: lbm_fs_params) -> C.c_void_p:
    h = C.c_void_p()
    _check(load().lbm_fs_create(C.byref(params), C.byref(h)), "lbm_fs_create")
    return h


def lbm_fs_destroy(h):
    _check(load().lbm_fs_destroy(h), "lbm_fs_destroy")


def lbm_fs_add_box(h, box: lbm_fs_box) -> int:
    out = C.c_int32(-1)
    _check(load().lbm_fs_add_box(h, C.byref(box), C.byref(out)), "lbm_fs_add_box")
    return out.value


def lbm_fs_step(h, nsteps: int):
    _check(load().lbm_fs_step(h, int(nsteps)), "lbm_fs_step")


def lbm_fs_forces(h, body: int):
    F, T, c, q = (C.c_double * 3)(), (C.c_double * 3)(), (C.c_double * 3)(), (C.c_double * 4)()
    _check(load().lbm_fs_forces(h, int(body), F, T, c, q), "lbm_fs_forces")
    return np.array(F), np.array(T), np.array(c), np.array(q)


def lbm_fs_body_state(h, body: int) -> dict:
    s = lbm_fs_body_state_t()
    _check(load().lbm_fs_body_state(h, int(body), C.byref(s)), "lbm_fs_body_state")
    return dict(F=np.array(s.F), T=np.array(s.T), S=s.S, center=np.array(s.center), quat=np.array(s.quat),
                vel=np.array(s.vel), omega=np.array(s.omega))


def lbm_fs_body_states(h, first: int, count: int, out=None):
    """States of bodies first .. first+count-1 with one synchronisation; out
    may be a preallocated (lbm_fs_body_state_t * count) array."""
    if out is None:
        out = (lbm_fs_body_state_t * count)()
    _check(load().lbm_fs_body_states(h, int(first), int(count), out), "lbm_fs_body_states")
    return out


def lbm_fs_read_fields(h, mask: int, dst: Sequence[Optional[int]], dst_on_device: bool):
    arr = (C.c_void_p * 6)(*[C.c_void_p(p) if p else None for p in dst])
    _check(load().lbm_fs_read_fields(h, int(mask), arr, 1 if dst_on_device else 0), "lbm_fs_read_fields")


def lbm_fs_stats(h) -> dict:
    s = lbm_fs_stats_t()
    _check(load().lbm_fs_stats(h, C.byref(s)), "lbm_fs_stats")
    return {k: getattr(s, k) for k, _ in lbm_fs_stats_t._fields_}


def lbm_fs_sync(h):
    _check(load().lbm_fs_sync(h), "lbm_fs_sync")


def lbm_fs_kernel_times(h, nsteps: int):
    cap = 32
    ms = (C.c_double * cap)()
    names = (C.c_char_p * cap)()
    nk = C.c_int32(0)
    _check(load().lbm_fs_kernel_times(h, int(nsteps), ms, names, cap, C.byref(nk)), "lbm_fs_kernel_times")
    return {names[k].decode(): ms[k] for k in range(nk.value)}


def lbm_fs_liquid_mass_noalloc(flags_dev: int, mass_dev: int, n: int, out_dev: int, stream: int = 0):
    """Liquid mass from device arrays without any device allocation (see the
    C declaration for the limits and the shared fixed scratch)."""
    code = load().lbm_fs_liquid_mass_noalloc(C.c_void_p(flags_dev), C.c_void_p(mass_dev), int(n),
                                             C.c_void_p(out_dev), C.c_void_p(stream) if stream else None)
    if code != LBM_FS_OK:
        raise LbmFsError(code, "lbm_fs_liquid_mass_noalloc", load().lbm_fs_noalloc_last_error_string().decode())


def lbm_fs_batch_create(params: Sequence[lbm_fs_params]):
    arr = (lbm_fs_params * len(params))(*params)
    b = C.c_void_p()
    _check(load().lbm_fs_batch_create(arr, len(params), C.byref(b)), "lbm_fs_batch_create")
    return b


def lbm_fs_batch_destroy(b):
    _check(load().lbm_fs_batch_destroy(b), "lbm_fs_batch_destroy")


def lbm_fs_batch_tank(b, k: int):
    h = C.c_void_p()
    _check(load().lbm_fs_batch_tank(b, int(k), C.byref(h)), "lbm_fs_batch_tank")
    return h


def lbm_fs_batch_step(b, nsteps: int):
    _check(load().lbm_fs_batch_step(b, int(nsteps)), "lbm_fs_batch_step")


def lbm_fs_batch_sync(b):
    _check(load().lbm_fs_batch_sync(b), "lbm_fs_batch_sync")


def _cfg_dict(c: lbm_fs_batch_config_t) -> dict:
    return dict(zb=c.zb, bulk_blocks=c.bulk_blocks, list_cells=c.list_cells, lanes=c.lanes, bulk_ms=c.bulk_ms)


def lbm_fs_batch_autotune(b) -> dict:
    c = lbm_fs_batch_config_t()
    _check(load().lbm_fs_batch_autotune(b, C.byref(c)), "lbm_fs_batch_autotune")
    return _cfg_dict(c)


def lbm_fs_batch_get_config(b) -> dict:
    c = lbm_fs_batch_config_t()
    _check(load().lbm_fs_batch_get_config(b, C.byref(c)), "lbm_fs_batch_get_config")
    return _cfg_dict(c)


def lbm_fs_batch_set_config(b, zb: int, bulk_blocks: int, list_cells: int, lanes: int = 0):
    c = lbm_fs_batch_config_t(zb=int(zb), bulk_blocks=int(bulk_blocks), list_cells=int(list_cells), lanes=int(lanes))
    _check(load().lbm_fs_batch_set_config(b, C.byref(c)), "lbm_fs_batch_set_config")


def lbm_fs_batch_kernel_times(b, nsteps: int):
    cap = 32
    ms = (C.c_double * cap)()
    names = (C.c_char_p * cap)()
    nk = C.c_int32(0)
    _check(load().lbm_fs_batch_kernel_times(b, int(nsteps), ms, names, cap, C.byref(nk)), "lbm_fs_batch_kernel_times")
    return {names[k].decode(): ms[k] for k in range(nk.value)}


def lbm_fs_batch_launches(b):
    n, st = C.c_int64(0), C.c_int64(0)
    _check(load().lbm_fs_batch_launches(b, C.byref(n), C.byref(st)), "lbm_fs_batch_launches")
    return n.value, st.value


def lbm_fs_fp64_rate(op: int, iters: int = 1 << 16, stream: int = 0) -> float:
    """Double-precision operations per second of this GPU (op 0 FMA, 1 add,
    2 multiply)."""
    r = C.c_double(0.0)
    code = load().lbm_fs_fp64_rate(int(op), int(iters), C.byref(r), C.c_void_p(stream) if stream else None)
    if code != LBM_FS_OK:
        raise LbmFsError(code, "lbm_fs_fp64_rate", "probe launch failed")
    return r.value


# ------------------------------------------------------------ convenience

class TorchAllocator:
    """dev_alloc / dev_free callbacks on PyTorch's caching allocator."""

    def __init__(self, device: int, stream: int):
        import torch

        self.torch = torch
        self.device = device
        self.stream = stream
        self.live = {}

        def _alloc(nbytes, ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
            except Exception:
                return None

        def _free(ptr, ctx):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.c_alloc = DEV_ALLOC(_alloc)
        self.c_free = DEV_FREE(_free)


def make_box(b) -> lbm_fs_box:
    box = lbm_fs_box()
    box.center[:] = [float(v) for v in b.center]
    box.half[:] = [float(v) for v in b.half]
    box.quat[:] = [float(v) for v in b.quat]
    box.density_ratio = float(b.density_ratio)
    box.vel[:] = [float(v) for v in b.vel]
    box.omega[:] = [float(v) for v in b.omega]
    box.mode = int(b.mode)
    box.rot_axis[:] = [float(v) for v in b.rot_axis]
    box.lin_damping = float(b.lin_damping)
    box.shape = int(getattr(b, "shape", 0))
    return box


def scenario_params(sc, storage: str, stream: int, use_graphs: bool, alloc=None, keep=None, device=None):
    """lbm_fs_params for a scenario of paper_1201_0351_gb300.inputs with its
    initial arrays as host buffers (device tensors when device is given);
    the buffers are appended to keep and must live until the create call
    returns."""
    p = lbm_fs_params()
    p.nx, p.ny, p.nz, p.periodic = sc.nx, sc.ny, sc.nz, sc.periodic
    p.tau = sc.tau
    p.gravity[:] = list(sc.gravity)
    p.body_accel[:] = list(sc.body_accel)
    p.rho_gas, p.eps = sc.rho_gas, sc.eps
    p.storage = STORAGE[storage]
    keep = [] if keep is None else keep
    flags = np.ascontiguousarray(sc.flags, np.uint8)
    fill = np.ascontiguousarray(sc.fill, np.float64)
    rho = np.ascontiguousarray(sc.rho, np.float64)
    vel = None if sc.vel is None else np.ascontiguousarray(sc.vel, np.float64).reshape(-1)
    if device is None:
        arrs = [flags, fill, rho, vel]
        keep += arrs
        p.init_flags, p.init_fill, p.init_rho = (a.ctypes.data for a in arrs[:3])
        p.init_vel = vel.ctypes.data if vel is not None else None
        p.init_on_device = 0
    else:
        import torch

        ts = [torch.from_numpy(a).to(device) if a is not None else None for a in (flags, fill, rho, vel)]
        keep += ts
        p.init_flags, p.init_fill, p.init_rho = (t.data_ptr() for t in ts[:3])
        p.init_vel = ts[3].data_ptr() if ts[3] is not None else None
        p.init_on_device = 1
    if alloc is not None:
        p.dev_alloc, p.dev_free = alloc.c_alloc, alloc.c_free
    p.stream = stream
    p.use_graphs = 1 if use_graphs else 0
    p.sigma = float(getattr(sc, "sigma", 0.0) or 0.0)
    wall_vel = getattr(sc, "wall_vel", None)
    if wall_vel is not None:
        p.wall_vel[:] = [float(v) for v in np.asarray(wall_vel, dtype=np.float64).reshape(18)]
    for key, value in (getattr(sc, "readings", None) or {}).items():
        field, bit, conv = READINGS[key]
        setattr(p, field, conv(value))
        p.readings |= bit
    return p


class _Handle:
    """Read-side calls shared by a simulation and a tank of a batch (self.h,
    self.n, self.device, self.torch, self.nbodies)."""

    def add_box(self, b) -> int:
        i = lbm_fs_add_box(self.h, make_box(b))
        self.nbodies += 1
        return i

    def sync(self):
        lbm_fs_sync(self.h)

    def body(self, b: int = 0) -> dict:
        return lbm_fs_body_state(self.h, b)

    def stats(self) -> dict:
        return lbm_fs_stats(self.h)

    def flags(self) -> np.ndarray:
        """The cell classes alone (one byte per cell)."""
        out = np.zeros(self.n, np.uint8)
        lbm_fs_read_fields(self.h, FIELD_FLAGS, [out.ctypes.data, None, None, None, None, None], False)
        return out

    def fields(self, want_f: bool = False, on_device: bool = False) -> dict:
        n = self.n
        mask = FIELD_FLAGS | FIELD_FILL | FIELD_MASS | FIELD_RHO | FIELD_VEL | (FIELD_F if want_f else 0)
        if on_device:
            t = self.torch
            bufs = [t.empty(n, dtype=t.uint8, device=self.device), t.empty(n, dtype=t.float64, device=self.device),
                    t.empty(n, dtype=t.float64, device=self.device), t.empty(n, dtype=t.float64, device=self.device),
                    t.empty(3 * n, dtype=t.float64, device=self.device),
                    t.empty(19 * n, dtype=t.float64, device=self.device) if want_f else None]
            lbm_fs_read_fields(self.h, mask, [b.data_ptr() if b is not None else None for b in bufs], True)
            out = [b.cpu().numpy() if b is not None else None for b in bufs]
        else:
            out = [np.zeros(n, np.uint8), np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(3 * n),
                   np.zeros(19 * n) if want_f else None]
            lbm_fs_read_fields(self.h, mask, [a.ctypes.data if a is not None else None for a in out], False)
        res = dict(flags=out[0], fill=out[1], mass=out[2], rho=out[3], u=out[4].reshape(n, 3))
        if want_f:
            res["f"] = out[5].reshape(19, n)
        return res


class Simulation(_Handle):
    """One handle of the library for a scenario of paper_1201_0351_gb300.inputs.

    storage: 'f64', 'f32' or 'f16s'.  Initial arrays are passed as host buffers
    (the library uploads them) unless host_init=False, in which case they are
    first copied to device tensors.
    """

    def __init__(self, sc, storage: str = "f64", use_graphs: bool = True, torch_alloc: bool = True,
                 host_init: bool = True, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the free-surface LBM library needs a CUDA GPU")
        load()
        self.torch = torch
        self.sc = sc
        self.n = sc.nx * sc.ny * sc.nz
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.alloc = TorchAllocator(self.device, self.stream.cuda_stream) if torch_alloc else None
        keep = []
        p = scenario_params(sc, storage, self.stream.cuda_stream, use_graphs, self.alloc, keep,
                            None if host_init else self.device)
        self.params = p
        self.h = lbm_fs_create(p)
        del keep
        self.nbodies = 0
        for b in sc.boxes:
            self.add_box(b)

    def step(self, n: int = 1):
        lbm_fs_step(self.h, n)

    def kernel_times(self, nsteps: int) -> dict:
        return lbm_fs_kernel_times(self.h, nsteps)

    def close(self):
        if getattr(self, "h", None):
            lbm_fs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TankView(_Handle):
    """Tank k of a Batch: the read-side calls of a simulation (and add_box
    between batch steps); the batch steps it."""

    def __init__(self, batch, k: int, sc):
        self.torch = batch.torch
        self.h = lbm_fs_batch_tank(batch.h, k)
        self.sc = sc
        self.n = sc.nx * sc.ny * sc.nz
        self.device = batch.device
        self.nbodies = 0


class Batch:
    """Many scenarios stepped together by the batched form of the library
    (one launch per kernel for all tanks, packed block tables, CUDA graphs)."""

    def __init__(self, scenarios, storage: str = "f16s", use_graphs: bool = True, torch_alloc: bool = True,
                 stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the free-surface LBM library needs a CUDA GPU")
        load()
        self.torch = torch
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.alloc = TorchAllocator(self.device, self.stream.cuda_stream) if torch_alloc else None
        keep = []
        params = [scenario_params(sc, storage, self.stream.cuda_stream, use_graphs, self.alloc, keep)
                  for sc in scenarios]
        self.h = lbm_fs_batch_create(params)
        del keep
        self.tanks = [TankView(self, k, sc) for k, sc in enumerate(scenarios)]
        for t, sc in zip(self.tanks, scenarios):
            for b in sc.boxes:
                t.add_box(b)
        self.cells = sum(t.n for t in self.tanks)

    def step(self, n: int = 1):
        lbm_fs_batch_step(self.h, n)

    def sync(self):
        lbm_fs_batch_sync(self.h)

    def autotune(self) -> dict:
        return lbm_fs_batch_autotune(self.h)

    def config(self) -> dict:
        return lbm_fs_batch_get_config(self.h)

    def set_config(self, zb: int, bulk_blocks: int, list_cells: int, lanes: int = 0):
        lbm_fs_batch_set_config(self.h, zb, bulk_blocks, list_cells, lanes)

    def kernel_times(self, nsteps: int) -> dict:
        return lbm_fs_batch_kernel_times(self.h, nsteps)

    def launches(self):
        return lbm_fs_batch_launches(self.h)

    def close(self):
        if getattr(self, "h", None):
            lbm_fs_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
