"""ctypes front end of the FP64 PBD-R oracle (``pbdr_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this module.  It never
imports the product package and the product package never imports it.

The C library is built in place with the system C compiler by ``build()``
(``-O2 -ffp-contract=off``: the FP32 neighbour predicate must round every
operation exactly as written).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pbdr_oracle.c")
LIB = os.path.join(HERE, "liborc_pbdr.so")

STD_VELOCITY = 1 << 0
NO_LINMOM = 1 << 1
NO_ANGMOM = 1 << 2
CONTACT_AVG = 1 << 3
SM_FROM_XI = 1 << 4

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liborc_pbdr.so`` (if stale)."""
    hdr = os.path.join(HERE, "pbdr_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cc = os.environ.get("CC", "cc")
    subprocess.check_call([cc, "-O2", "-std=c11", "-ffp-contract=off", "-fPIC",
                           "-shared", "-o", tmp, SRC, "-lm"])
    os.replace(tmp, LIB)
    return LIB


class _Scene(C.Structure):
    _fields_ = [
        ("num_particles", C.c_int32),
        ("num_bodies", C.c_int32),
        ("body_off", C.POINTER(C.c_int32)),
        ("inv_mass", C.POINTER(C.c_double)),
        ("rest", C.POINTER(C.c_double)),
        ("body_mass", C.POINTER(C.c_double)),
        ("radius", C.c_double),
        ("friction", C.c_double),
        ("gravity", C.c_double * 3),
        ("plane", C.c_double * 4),
        ("dt", C.c_double),
        ("iterations", C.c_int32),
        ("flags", C.c_uint32),
        ("force", C.POINTER(C.c_double)),
        ("torque", C.POINTER(C.c_double)),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            P = C.POINTER
            L.orc_nbr_constants.argtypes = [C.c_float, P(C.c_float), P(C.c_float),
                                            P(C.c_float), P(C.c_float)]
            L.orc_table_size.argtypes = [C.c_int32]
            L.orc_table_size.restype = C.c_uint32
            L.orc_cell_keys.argtypes = [C.c_int32, C.c_void_p, C.c_float, C.c_uint32, C.c_void_p]
            L.orc_sort_keys.argtypes = [C.c_int32, C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p]
            for fn in (L.orc_neighbors_brute,):
                fn.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_float,
                               C.c_void_p, C.c_void_p, C.c_int64]
                fn.restype = C.c_int64
            L.orc_neighbors_grid.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_float,
                                             C.c_float, C.c_void_p, C.c_void_p, C.c_int64]
            L.orc_neighbors_grid.restype = C.c_int64
            L.orc_rest_shape.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_polar_rotation.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_body_inertia.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p]
            L.orc_enforce_momentum.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                               C.c_void_p, C.c_void_p, C.c_double, C.c_uint32,
                                               C.c_void_p, C.c_void_p]
            L.orc_substep.argtypes = [P(_Scene), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
            L.orc_substep.restype = C.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------
# neighbour search (FP32)
# --------------------------------------------------------------------------

def nbr_constants(radius: float):
    vals = [C.c_float() for _ in range(4)]
    lib().orc_nbr_constants(C.c_float(radius), *[C.byref(v) for v in vals])
    return tuple(v.value for v in vals)   # Rn, Rn2, h, inv_h


def table_size(n: int) -> int:
    return int(lib().orc_table_size(n))


def cell_keys(x: np.ndarray, radius: float) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    n = x.shape[0]
    _, _, _, inv_h = nbr_constants(radius)
    keys = np.zeros(max(n, 1), dtype=np.uint32)
    lib().orc_cell_keys(n, _ptr(x), C.c_float(inv_h), table_size(n), _ptr(keys))
    return keys[:n]


def sorted_keys(x: np.ndarray, radius: float):
    """(sorted bucket keys, particle ids), stable by id within a key."""
    keys = cell_keys(x, radius)
    n = keys.shape[0]
    sk = np.zeros(max(n, 1), dtype=np.uint32)
    si = np.zeros(max(n, 1), dtype=np.uint32)
    lib().orc_sort_keys(n, _ptr(keys), table_size(n), _ptr(sk), _ptr(si))
    return sk[:n], si[:n]


def body_index(body_off: np.ndarray) -> np.ndarray:
    body_off = np.asarray(body_off, dtype=np.int64)
    return np.repeat(np.arange(len(body_off) - 1, dtype=np.int32),
                     np.diff(body_off)).astype(np.int32)


def neighbors(x: np.ndarray, body: np.ndarray, radius: float, method: str = "grid"):
    """CSR (off[n+1], idx) of N(p) = {q != p, body(q) != body(p), d2 < Rn^2}."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    body = np.ascontiguousarray(body, dtype=np.int32)
    n = x.shape[0]
    _, Rn2, _, inv_h = nbr_constants(radius)
    off = np.zeros(n + 1, dtype=np.int32)
    cap = 8 * n + 64
    while True:
        idx = np.zeros(cap, dtype=np.int32)
        if method == "brute":
            need = lib().orc_neighbors_brute(n, _ptr(x), _ptr(body), C.c_float(Rn2),
                                             _ptr(off), _ptr(idx), cap)
        else:
            need = lib().orc_neighbors_grid(n, _ptr(x), _ptr(body), C.c_float(Rn2),
                                            C.c_float(inv_h), _ptr(off), _ptr(idx), cap)
        if need <= cap:
            return off, idx[:need].copy()
        cap = int(need)


# --------------------------------------------------------------------------
# shape matching / momentum pieces
# --------------------------------------------------------------------------

def polar_rotation(A: np.ndarray, Rprev: np.ndarray | None = None) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    Rp = np.eye(3) if Rprev is None else np.ascontiguousarray(Rprev, dtype=np.float64)
    R = np.zeros((3, 3))
    lib().orc_polar_rotation(_ptr(A), _ptr(Rp), _ptr(R))
    return R


def body_inertia(x: np.ndarray, mass: np.ndarray, c: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    I = np.zeros((3, 3))
    lib().orc_body_inertia(x.shape[0], _ptr(x), _ptr(mass), _ptr(c), _ptr(I))
    return I


def enforce_momentum(mass, xb, vb, xa, va, dt, flags=0):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (mass, xb, vb, xa, va)]
    n = arrs[0].shape[0]
    xo = np.zeros((n, 3))
    vo = np.zeros((n, 3))
    lib().orc_enforce_momentum(n, *[_ptr(a) for a in arrs], C.c_double(dt),
                               C.c_uint32(flags), _ptr(xo), _ptr(vo))
    return xo, vo


# --------------------------------------------------------------------------
# whole substeps
# --------------------------------------------------------------------------

class OracleScene:
    """FP64 state of one scene stepped by ``orc_substep``.

    ``scene`` is any object with the attributes of a scene description: pos,
    vel, inv_mass, body_off, radius, friction, gravity, plane, dt, iterations,
    flags and optional force/torque ([B,3]).  FP32 inputs are promoted to FP64;
    the rest shape is the configuration at creation.
    """

    def __init__(self, scene):
        self.body_off = np.ascontiguousarray(scene.body_off, dtype=np.int32)
        self.inv_mass = np.ascontiguousarray(scene.inv_mass, dtype=np.float64)
        self.x = np.ascontiguousarray(scene.pos, dtype=np.float64).copy()
        self.v = np.ascontiguousarray(scene.vel, dtype=np.float64).copy()
        n, nb = self.x.shape[0], self.body_off.shape[0] - 1
        self.rest = np.zeros((n, 3))
        self.body_mass = np.zeros(nb)
        lib().orc_rest_shape(n, nb, _ptr(self.body_off), _ptr(self.inv_mass),
                             _ptr(self.x), _ptr(self.rest), _ptr(self.body_mass))
        self.rot = np.tile(np.eye(3), (nb, 1, 1)).copy()
        self.force = None if scene.force is None else np.ascontiguousarray(scene.force, dtype=np.float64)
        self.torque = None if scene.torque is None else np.ascontiguousarray(scene.torque, dtype=np.float64)
        s = _Scene()
        s.num_particles = n
        s.num_bodies = nb
        s.body_off = self.body_off.ctypes.data_as(C.POINTER(C.c_int32))
        s.inv_mass = self.inv_mass.ctypes.data_as(C.POINTER(C.c_double))
        s.rest = self.rest.ctypes.data_as(C.POINTER(C.c_double))
        s.body_mass = self.body_mass.ctypes.data_as(C.POINTER(C.c_double))
        s.radius = float(scene.radius)
        s.friction = float(scene.friction)
        s.gravity = (C.c_double * 3)(*[float(g) for g in scene.gravity])
        s.plane = (C.c_double * 4)(*[float(g) for g in scene.plane])
        s.dt = float(scene.dt)
        s.iterations = int(scene.iterations)
        s.flags = int(scene.flags)
        s.force = (self.force.ctypes.data_as(C.POINTER(C.c_double))
                   if self.force is not None else None)
        s.torque = (self.torque.ctypes.data_as(C.POINTER(C.c_double))
                    if self.torque is not None else None)
        self._s = s

    @property
    def num_particles(self):
        return self.x.shape[0]

    def set_state(self, pos, vel):
        self.x[...] = np.asarray(pos, dtype=np.float64)
        self.v[...] = np.asarray(vel, dtype=np.float64)

    def substep(self, n: int = 1, brute: bool = False):
        L = lib()
        for _ in range(n):
            rc = L.orc_substep(C.byref(self._s), _ptr(self.x), _ptr(self.v),
                               _ptr(self.rot), 1 if brute else 0)
            if rc != 0:
                raise MemoryError("oracle substep failed to allocate")
        return self

    def body_index(self):
        return body_index(self.body_off)

    def masses(self):
        return 1.0 / self.inv_mass

    def body_momenta(self, x=None, v=None):
        """per body: (centre of mass [B,3], P [B,3], L about the CoM [B,3])"""
        x = self.x if x is None else np.asarray(x, dtype=np.float64)
        v = self.v if v is None else np.asarray(v, dtype=np.float64)
        m = self.masses()
        bid = self.body_index()
        nb = self.body_off.shape[0] - 1
        M = np.bincount(bid, weights=m, minlength=nb)
        c = np.stack([np.bincount(bid, weights=m * x[:, k], minlength=nb) for k in range(3)], 1) / M[:, None]
        P = np.stack([np.bincount(bid, weights=m * v[:, k], minlength=nb) for k in range(3)], 1)
        r = x - c[bid]
        rxv = np.cross(r, m[:, None] * v)
        Lm = np.stack([np.bincount(bid, weights=rxv[:, k], minlength=nb) for k in range(3)], 1)
        return c, P, Lm
