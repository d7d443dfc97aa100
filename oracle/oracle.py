"""ctypes wrapper of the C oracle (TEST INFRASTRUCTURE ONLY).

The C file is compiled with -O2 -ffp-contract=off so that no multiply-add is
fused (every operation is one IEEE-754 rounding, on x86-64 and on AArch64).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

LIQUID, INTERFACE, GAS, OBSTACLE = 1, 2, 4, 8


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, one thread)."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "lbm_oracle.h"))):
        tmp = LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build_oracle())
        P, D, I = C.c_void_p, C.POINTER(C.c_double), C.c_int
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [I, I, I, C.c_uint, C.c_double, D, D, C.c_double, C.c_double,
                                   C.POINTER(C.c_uint8), D, D, D]
        lib.orc_destroy.argtypes = [P]
        lib.orc_add_box.restype = I
        lib.orc_add_box.argtypes = [P, D, D, D, C.c_double, D, D, I, D, C.c_double, I]
        lib.orc_step.restype = I
        lib.orc_step.argtypes = [P, I]
        lib.orc_compute_forces.argtypes = [P]
        lib.orc_get_fields.argtypes = [P, C.POINTER(C.c_uint8), D, D, D, D, D]
        lib.orc_get_body.argtypes = [P, I, D, D, D, D, D, D, D]
        lib.orc_get_ledger.argtypes = [P, D]
        lib.orc_error.restype = I
        lib.orc_error.argtypes = [P]
        lib.orc_time.restype = C.c_long
        lib.orc_time.argtypes = [P]
        lib.orc_get_counts.argtypes = [P, C.POINTER(C.c_long)]
        lib.orc_lattice.argtypes = [C.POINTER(C.c_int), D, C.POINTER(C.c_int)]
        lib.orc_feq.argtypes = [C.c_double, D, D]
        lib.orc_force_term.argtypes = [C.c_double, D, D, D]
        lib.orc_set_mutation.argtypes = [I]
        lib.orc_set_surface_tension.argtypes = [P, C.c_double]
        lib.orc_set_wall_velocity.argtypes = [P, D]
        lib.orc_set_readings.argtypes = [P, C.c_double, C.c_double, I, I]
        lib.orc_set_body_force.argtypes = [P, I, D, D]
        lib.orc_bodies_step.argtypes = [P]
        _lib = lib
        return lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _d3(v, n=3):
    return (C.c_double * n)(*[float(x) for x in v])


def lattice():
    lib = _load()
    c = np.zeros((19, 3), np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, np.int32)
    lib.orc_lattice(c.ctypes.data_as(C.POINTER(C.c_int)), _dp(w), opp.ctypes.data_as(C.POINTER(C.c_int)))
    return c, w, opp


def feq(rho, u):
    out = np.zeros(19)
    _load().orc_feq(float(rho), _d3(u), _dp(out))
    return out


def force_term(rho, u, a):
    out = np.zeros(19)
    _load().orc_force_term(float(rho), _d3(u), _d3(a), _dp(out))
    return out


def set_mutation(m: int):
    _load().orc_set_mutation(int(m))


class OracleSim:
    """One simulation in the oracle, built from a scenario of the input module."""

    def __init__(self, sc):
        lib = _load()
        self.lib = lib
        self.sc = sc
        self.n = sc.nx * sc.ny * sc.nz
        flags = np.ascontiguousarray(sc.flags, dtype=np.uint8)
        fill = np.ascontiguousarray(sc.fill, dtype=np.float64)
        rho = np.ascontiguousarray(sc.rho, dtype=np.float64)
        vel = getattr(sc, "vel", None)
        self._vel = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64).reshape(-1)
        self.h = lib.orc_create(sc.nx, sc.ny, sc.nz, sc.periodic, sc.tau, _d3(sc.gravity), _d3(sc.body_accel),
                                sc.rho_gas, sc.eps, flags.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(fill), _dp(rho),
                                None if self._vel is None else _dp(self._vel))
        if not self.h:
            raise ValueError("oracle rejected the scenario")
        sigma = float(getattr(sc, "sigma", 0.0) or 0.0)
        if sigma:
            lib.orc_set_surface_tension(self.h, sigma)
        wall_vel = getattr(sc, "wall_vel", None)
        if wall_vel is not None:
            self._wv = np.ascontiguousarray(np.asarray(wall_vel, dtype=np.float64).reshape(18))
            lib.orc_set_wall_velocity(self.h, _dp(self._wv))
        rd = getattr(sc, "readings", None)
        if rd is not None:
            self.set_readings(**rd)
        for b in sc.boxes:
            self.add_box(b)

    def add_box(self, b):
        return self.lib.orc_add_box(self.h, _d3(b.center), _d3(b.half), _d3(b.quat, 4), b.density_ratio,
                                    _d3(b.vel), _d3(b.omega), b.mode, _d3(b.rot_axis), b.lin_damping,
                                    int(getattr(b, "shape", 0)))

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    def set_readings(self, deadband: float = 1e-2, virtual_mass: float = 1.0, force_mean: bool = True,
                     neighbour_rule: bool = True):
        """The options where the paper is silent (C declaration of orc_set_readings)."""
        self.lib.orc_set_readings(self.h, float(deadband), float(virtual_mass), int(bool(force_mean)),
                                  int(bool(neighbour_rule)))

    def step(self, n: int = 1) -> int:
        return self.lib.orc_step(self.h, int(n))

    def set_body_force(self, b: int, F, T):
        """Force and torque of body b as if the momentum exchange had produced them."""
        self.lib.orc_set_body_force(self.h, int(b), _d3(F), _d3(T))

    def bodies_step(self):
        """The rigid-body update alone (no fluid step, no remapping)."""
        self.lib.orc_bodies_step(self.h)

    def compute_forces(self):
        self.lib.orc_compute_forces(self.h)

    @property
    def error(self) -> int:
        return self.lib.orc_error(self.h)

    @property
    def time(self) -> int:
        return self.lib.orc_time(self.h)

    def fields(self, want_f: bool = False):
        n = self.n
        flags = np.zeros(n, np.uint8)
        fill, mass, rho = np.zeros(n), np.zeros(n), np.zeros(n)
        u = np.zeros(3 * n)
        f = np.zeros(19 * n) if want_f else None
        self.lib.orc_get_fields(self.h, flags.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(fill), _dp(mass), _dp(rho),
                                _dp(u), _dp(f) if want_f else None)
        out = dict(flags=flags, fill=fill, mass=mass, rho=rho, u=u.reshape(n, 3))
        if want_f:
            out["f"] = f.reshape(19, n)
        return out

    def body(self, b: int = 0):
        F, T, c, v, w = (np.zeros(3) for _ in range(5))
        q = np.zeros(4)
        S = C.c_double(0.0)
        self.lib.orc_get_body(self.h, b, _dp(F), _dp(T), C.byref(S), _dp(c), _dp(q), _dp(v), _dp(w))
        return dict(F=F, T=T, S=S.value, center=c, quat=q, vel=v, omega=w)

    def ledger(self):
        out = np.zeros(6)
        self.lib.orc_get_ledger(self.h, _dp(out))
        return dict(covered=out[0], uncovered=out[1], lost=out[2], M0=out[3], M=out[4], wall=out[5])

    def counts(self):
        out = (C.c_long * 6)()
        self.lib.orc_get_counts(self.h, out)
        return dict(zip(("filled", "emptied", "new_from_gas", "new_from_liquid", "receivers", "covered"), list(out)))
