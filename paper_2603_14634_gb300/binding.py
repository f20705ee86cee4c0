"""Thin ctypes binding of ``libpbdr.so`` (C ABI in ``include/pbdr.h``).

Functions keep the C names and only marshal arguments; every step of the
solver runs in the library's sm_103a kernels.  ``Context`` is a small
convenience wrapper over the same calls.  There is no CPU fallback: loading
fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from .build import LIB

PBDR_OK = 0
ERRORS = {
    -1: "PBDR_ERR_INVALID", -2: "PBDR_ERR_OOM", -3: "PBDR_ERR_BUDGET",
    -4: "PBDR_ERR_NBR_OVERFLOW", -5: "PBDR_ERR_NONFINITE", -6: "PBDR_ERR_TIMEOUT",
    -7: "PBDR_ERR_CUDA", -8: "PBDR_ERR_UNSUPPORTED",
}
EBIT_NBR_OVERFLOW = 1
EBIT_NONFINITE = 2

EXPORTS = [
    "pbdr_ctx_create", "pbdr_ctx_destroy", "pbdr_create_scene", "pbdr_destroy_scene",
    "pbdr_set_body_wrench", "pbdr_step", "pbdr_read_state", "pbdr_write_state",
    "pbdr_read_states", "pbdr_read_states_async", "pbdr_write_states", "pbdr_scene_info", "pbdr_last_error",
    "pbdr_build_neighbors", "pbdr_read_neighbors", "pbdr_last_launch_count",
    "pbdr_neighbor_total", "pbdr_set_profiling", "pbdr_read_profile",
    "pbdr_neighbors_noalloc", "pbdr_set_option", "pbdr_plan_config",
    "pbdr_step_tangent", "pbdr_write_tangent", "pbdr_read_tangent",
    "pbdr_adjoint", "pbdr_write_adjoint", "pbdr_read_adjoint",
    "pbdr_write_tangent_friction", "pbdr_read_adjoint_friction",
]
NUM_STAGES = 6
STAGES = ("wrench", "predict_keys", "radix_sort", "cells_neighbors", "iterate", "scene_resident")
OPT_PATH = 1
OPT_FUSED_THREADS = 2
OPT_GRAPHS = 3
OPT_AUTOTUNE = 4
OPT_TUNE_AFTER = 5


class PbdrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class SceneDesc(C.Structure):
    _fields_ = [
        ("num_particles", C.c_int32),
        ("num_bodies", C.c_int32),
        ("pos", C.POINTER(C.c_float)),
        ("vel", C.POINTER(C.c_float)),
        ("inv_mass", C.POINTER(C.c_float)),
        ("body_off", C.POINTER(C.c_int32)),
        ("radius", C.c_float),
        ("friction", C.c_float),
        ("gravity", C.c_float * 3),
        ("plane", C.c_float * 4),
        ("dt", C.c_float),
        ("iterations", C.c_int32),
        ("flags", C.c_uint32),
    ]


_lib = None


def load(path: Optional[str] = None):
    """Load libpbdr.so (raises if it is missing: build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libpbdr.so not built ({path}); run __graft_entry__.build()")
    L = C.CDLL(path)
    vp, i32, P = C.c_void_p, C.c_int32, C.POINTER
    L.pbdr_ctx_create.argtypes = [C.c_int, C.c_size_t, P(vp)]
    L.pbdr_ctx_destroy.argtypes = [vp]
    L.pbdr_create_scene.argtypes = [vp, P(SceneDesc), P(i32)]
    L.pbdr_destroy_scene.argtypes = [vp, i32]
    L.pbdr_set_body_wrench.argtypes = [vp, i32, i32, P(C.c_float), P(C.c_float)]
    L.pbdr_step.argtypes = [vp, P(i32), i32, i32, vp]
    L.pbdr_read_state.argtypes = [vp, i32, vp, vp, vp, vp]
    L.pbdr_write_state.argtypes = [vp, i32, vp, vp, vp]
    L.pbdr_read_states.argtypes = [vp, P(i32), i32, vp, vp, vp, vp]
    L.pbdr_read_states_async.argtypes = [vp, P(i32), i32, vp, vp, vp, vp]
    L.pbdr_write_states.argtypes = [vp, P(i32), i32, vp, vp, vp]
    L.pbdr_step_tangent.argtypes = [vp, P(i32), i32, i32, vp]
    L.pbdr_write_tangent.argtypes = [vp, i32, vp, vp, vp]
    L.pbdr_read_tangent.argtypes = [vp, i32, vp, vp, vp]
    L.pbdr_adjoint.argtypes = [vp, P(i32), i32, i32, i32, vp]
    L.pbdr_write_adjoint.argtypes = [vp, i32, vp, vp, vp]
    L.pbdr_read_adjoint.argtypes = [vp, i32, vp, vp, vp]
    L.pbdr_write_tangent_friction.argtypes = [vp, i32, C.c_float, vp]
    L.pbdr_read_adjoint_friction.argtypes = [vp, i32, P(C.c_double), vp]
    L.pbdr_scene_info.argtypes = [vp, i32, P(i32), P(i32)]
    L.pbdr_last_error.argtypes = []
    L.pbdr_last_error.restype = C.c_char_p
    L.pbdr_build_neighbors.argtypes = [vp, P(i32), i32, vp]
    L.pbdr_read_neighbors.argtypes = [vp, i32, vp, vp, vp, vp, C.c_int64, P(C.c_int64), vp]
    L.pbdr_last_launch_count.argtypes = [vp, P(C.c_int64)]
    L.pbdr_neighbor_total.argtypes = [vp, P(i32), i32, P(C.c_int64), vp]
    L.pbdr_set_profiling.argtypes = [vp, C.c_int]
    L.pbdr_read_profile.argtypes = [vp, vp, vp, i32]
    L.pbdr_neighbors_noalloc.argtypes = [vp, vp, i32, C.c_float, vp, vp, vp, vp, i32, vp]
    L.pbdr_set_option.argtypes = [vp, i32, C.c_int64]
    L.pbdr_plan_config.argtypes = [vp, P(i32), i32, vp, i32]
    for name in EXPORTS:
        if name != "pbdr_last_error":
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(rc: int):
    if rc != PBDR_OK:
        msg = load().pbdr_last_error().decode(errors="replace")
        raise PbdrError(rc, msg)


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _ids(ids: Sequence[int]):
    arr = np.ascontiguousarray(np.asarray(ids, dtype=np.int32))
    return arr, arr.ctypes.data_as(C.POINTER(C.c_int32))


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    return int(getattr(stream, "cuda_stream", 0)) or None


# ---- same-name wrappers ------------------------------------------------------

def pbdr_ctx_create(device: int = 0, hbm_budget_bytes: int = 0) -> int:
    h = C.c_void_p()
    _check(load().pbdr_ctx_create(device, hbm_budget_bytes, C.byref(h)))
    return h.value


def pbdr_ctx_destroy(ctx: int) -> None:
    _check(load().pbdr_ctx_destroy(ctx))


def pbdr_create_scene(ctx: int, scene) -> int:
    """``scene``: object with pos [N,3], vel [N,3], inv_mass [N], body_off [B+1],
    radius, friction, gravity, plane, dt, iterations, flags (see scenes.Scene)."""
    pos = np.ascontiguousarray(scene.pos, dtype=np.float32)
    vel = np.ascontiguousarray(scene.vel, dtype=np.float32)
    w = np.ascontiguousarray(scene.inv_mass, dtype=np.float32)
    bo = np.ascontiguousarray(scene.body_off, dtype=np.int32)
    d = SceneDesc()
    d.num_particles = pos.shape[0]
    d.num_bodies = bo.shape[0] - 1
    d.pos = pos.ctypes.data_as(C.POINTER(C.c_float))
    d.vel = vel.ctypes.data_as(C.POINTER(C.c_float))
    d.inv_mass = w.ctypes.data_as(C.POINTER(C.c_float))
    d.body_off = bo.ctypes.data_as(C.POINTER(C.c_int32))
    d.radius = float(scene.radius)
    d.friction = float(scene.friction)
    d.gravity = (C.c_float * 3)(*[float(x) for x in scene.gravity])
    d.plane = (C.c_float * 4)(*[float(x) for x in scene.plane])
    d.dt = float(scene.dt)
    d.iterations = int(scene.iterations)
    d.flags = int(scene.flags)
    out = C.c_int32()
    _check(load().pbdr_create_scene(ctx, C.byref(d), C.byref(out)))
    sid = out.value
    force = getattr(scene, "force", None)
    torque = getattr(scene, "torque", None)
    if force is not None or torque is not None:
        B = d.num_bodies
        F = np.zeros((B, 3), np.float32) if force is None else np.asarray(force, np.float32).reshape(B, 3)
        T = np.zeros((B, 3), np.float32) if torque is None else np.asarray(torque, np.float32).reshape(B, 3)
        for b in range(B):
            pbdr_set_body_wrench(ctx, sid, b, F[b], T[b])
    return sid


def pbdr_destroy_scene(ctx: int, scene: int) -> None:
    _check(load().pbdr_destroy_scene(ctx, scene))


def pbdr_set_body_wrench(ctx: int, scene: int, body: int, F, tau) -> None:
    F = np.ascontiguousarray(F, dtype=np.float32)
    tau = np.ascontiguousarray(tau, dtype=np.float32)
    _check(load().pbdr_set_body_wrench(ctx, scene, body, F.ctypes.data_as(C.POINTER(C.c_float)),
                                       tau.ctypes.data_as(C.POINTER(C.c_float))))


def pbdr_step(ctx: int, ids: Sequence[int], substeps: int = 1, stream=None) -> None:
    arr, p = _ids(ids)
    _check(load().pbdr_step(ctx, p, len(arr), substeps, _stream(stream)))


def pbdr_step_tangent(ctx: int, ids: Sequence[int], substeps: int = 1, stream=None) -> None:
    arr, p = _ids(ids)
    _check(load().pbdr_step_tangent(ctx, p, len(arr), substeps, _stream(stream)))


def pbdr_write_tangent(ctx: int, scene: int, dpos=None, dvel=None, stream=None) -> None:
    dpos = None if dpos is None else np.ascontiguousarray(dpos, dtype=np.float32)
    dvel = None if dvel is None else np.ascontiguousarray(dvel, dtype=np.float32)
    _check(load().pbdr_write_tangent(ctx, scene, _ptr(dpos), _ptr(dvel), _stream(stream)))


def pbdr_read_tangent(ctx: int, scene: int, stream=None):
    """-> (dpos [N,3], dvel [N,3])"""
    n, _ = pbdr_scene_info(ctx, scene)
    dpos = np.empty((n, 3), np.float32)
    dvel = np.empty((n, 3), np.float32)
    _check(load().pbdr_read_tangent(ctx, scene, _ptr(dpos), _ptr(dvel), _stream(stream)))
    return dpos, dvel


def pbdr_adjoint(ctx: int, ids: Sequence[int], substeps: int, checkpoint_every: int = 20,
                 stream=None) -> None:
    arr, p = _ids(ids)
    _check(load().pbdr_adjoint(ctx, p, len(arr), substeps, checkpoint_every, _stream(stream)))


def pbdr_write_adjoint(ctx: int, scene: int, xbar=None, vbar=None, stream=None) -> None:
    xbar = None if xbar is None else np.ascontiguousarray(xbar, dtype=np.float32)
    vbar = None if vbar is None else np.ascontiguousarray(vbar, dtype=np.float32)
    _check(load().pbdr_write_adjoint(ctx, scene, _ptr(xbar), _ptr(vbar), _stream(stream)))


def pbdr_read_adjoint(ctx: int, scene: int, stream=None):
    """-> (xbar [N,3], vbar [N,3])"""
    n, _ = pbdr_scene_info(ctx, scene)
    xb = np.empty((n, 3), np.float32)
    vb = np.empty((n, 3), np.float32)
    _check(load().pbdr_read_adjoint(ctx, scene, _ptr(xb), _ptr(vb), _stream(stream)))
    return xb, vb


def pbdr_write_tangent_friction(ctx: int, scene: int, dmu: float, stream=None) -> None:
    _check(load().pbdr_write_tangent_friction(ctx, scene, float(dmu), _stream(stream)))


def pbdr_read_adjoint_friction(ctx: int, scene: int, stream=None) -> float:
    out = C.c_double()
    _check(load().pbdr_read_adjoint_friction(ctx, scene, C.byref(out), _stream(stream)))
    return out.value


def pbdr_scene_info(ctx: int, scene: int):
    n, b = C.c_int32(), C.c_int32()
    _check(load().pbdr_scene_info(ctx, scene, C.byref(n), C.byref(b)))
    return n.value, b.value


def pbdr_read_state(ctx: int, scene: int, stream=None, pos=None, vel=None):
    """-> (pos [N,3], vel [N,3], err_bits); pos/vel may be given (float32, C order)."""
    n, _ = pbdr_scene_info(ctx, scene)
    pos = np.empty((n, 3), np.float32) if pos is None else pos
    vel = np.empty((n, 3), np.float32) if vel is None else vel
    err = np.zeros(1, np.uint32)
    _check(load().pbdr_read_state(ctx, scene, _ptr(pos), _ptr(vel), _ptr(err), _stream(stream)))
    return pos, vel, int(err[0])


def pbdr_write_state(ctx: int, scene: int, pos=None, vel=None, stream=None) -> None:
    pos = None if pos is None else np.ascontiguousarray(pos, dtype=np.float32)
    vel = None if vel is None else np.ascontiguousarray(vel, dtype=np.float32)
    _check(load().pbdr_write_state(ctx, scene, _ptr(pos), _ptr(vel), _stream(stream)))


def pbdr_read_states(ctx: int, ids: Sequence[int], pos=None, vel=None, stream=None,
                     want_err: bool = True):
    arr, p = _ids(ids)
    total = sum(pbdr_scene_info(ctx, int(s))[0] for s in arr) if (pos is None or vel is None) else None
    pos = np.empty((total, 3), np.float32) if pos is None else pos
    vel = np.empty((total, 3), np.float32) if vel is None else vel
    err = np.zeros(len(arr), np.uint32) if want_err else None
    _check(load().pbdr_read_states(ctx, p, len(arr), _ptr(pos), _ptr(vel), _ptr(err), _stream(stream)))
    return pos, vel, err


def pbdr_read_states_async(ctx: int, ids: Sequence[int], pos, vel, err, stream=None) -> None:
    """Enqueues a batched read into caller-owned host buffers (page-locked
    for an asynchronous copy); they are valid once the stream reaches it."""
    arr, p = _ids(ids)
    _check(load().pbdr_read_states_async(ctx, p, len(arr), _ptr(pos), _ptr(vel), _ptr(err), _stream(stream)))


def pbdr_write_states(ctx: int, ids: Sequence[int], pos=None, vel=None, stream=None) -> None:
    arr, p = _ids(ids)
    _check(load().pbdr_write_states(ctx, p, len(arr), _ptr(pos), _ptr(vel), _stream(stream)))


def pbdr_build_neighbors(ctx: int, ids: Sequence[int], stream=None) -> None:
    arr, p = _ids(ids)
    _check(load().pbdr_build_neighbors(ctx, p, len(arr), _stream(stream)))


def pbdr_set_option(ctx: int, option: int, value: int) -> None:
    _check(load().pbdr_set_option(ctx, option, value))


NUM_CLASSES = 4   # size classes of the scene-resident kernel


def pbdr_plan_config(ctx: int, ids: Sequence[int]):
    """-> list of per-class dicts (capacity, scenes, threads, scratch bits, ctas)"""
    arr, p = _ids(ids)
    out = np.zeros(5 * NUM_CLASSES, np.int32)
    _check(load().pbdr_plan_config(ctx, p, len(arr), _ptr(out), out.size))
    keys = ("capacity", "scenes", "threads", "scratch_bits", "ctas")
    return [dict(zip(keys, map(int, out[5 * k:5 * k + 5]))) for k in range(NUM_CLASSES)]


def pbdr_read_neighbors(ctx: int, scene: int, stream=None, lists_only: bool = False):
    """-> (sorted_key [N] u32, sorted_id [N] u32, off [N+1] i32, idx i32);
    with lists_only the first two are None (the scene-resident kernel keeps
    only the lists)."""
    n, _ = pbdr_scene_info(ctx, scene)
    sk = None if lists_only else np.zeros(max(n, 1), np.uint32)
    si = None if lists_only else np.zeros(max(n, 1), np.uint32)
    off = np.zeros(n + 1, np.int32)
    cnt = C.c_int64()
    L = load()
    _check(L.pbdr_read_neighbors(ctx, scene, _ptr(sk), _ptr(si), _ptr(off), None, 0,
                                 C.byref(cnt), _stream(stream)))
    idx = np.zeros(max(cnt.value, 1), np.int32)
    _check(L.pbdr_read_neighbors(ctx, scene, None, None, None, _ptr(idx), cnt.value,
                                 C.byref(cnt), _stream(stream)))
    if lists_only:
        return None, None, off, idx[:cnt.value]
    return sk[:n], si[:n], off, idx[:cnt.value]


def pbdr_last_launch_count(ctx: int) -> int:
    v = C.c_int64()
    _check(load().pbdr_last_launch_count(ctx, C.byref(v)))
    return v.value


def pbdr_neighbor_total(ctx: int, ids: Sequence[int], stream=None) -> int:
    arr, p = _ids(ids)
    v = C.c_int64()
    _check(load().pbdr_neighbor_total(ctx, p, len(arr), C.byref(v), _stream(stream)))
    return v.value


def pbdr_set_profiling(ctx: int, enable: bool) -> None:
    _check(load().pbdr_set_profiling(ctx, 1 if enable else 0))


def pbdr_read_profile(ctx: int):
    """-> {stage: (ms, launches)} summed since the last read"""
    ms = np.zeros(NUM_STAGES, np.float64)
    ln = np.zeros(NUM_STAGES, np.int64)
    _check(load().pbdr_read_profile(ctx, _ptr(ms), _ptr(ln), NUM_STAGES))
    return {name: (float(ms[k]), int(ln[k])) for k, name in enumerate(STAGES)}


def pbdr_neighbors_noalloc(pos_ptr: int, body_ptr: int, n: int, radius: float,
                           sorted_key_ptr: int, sorted_id_ptr: int, nbr_cnt_ptr: int,
                           nbr_ptr: int, cap: int = 32, stream=None) -> None:
    """Allocation-free neighbour stage of one scene on caller-owned device
    buffers (raw device pointers; see include/pbdr.h)."""
    _check(load().pbdr_neighbors_noalloc(pos_ptr, body_ptr, n, float(radius), sorted_key_ptr,
                                         sorted_id_ptr, nbr_cnt_ptr, nbr_ptr, cap, _stream(stream)))


class Context:
    """Owns one pbdr context on a CUDA device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.h = pbdr_ctx_create(device, hbm_budget_bytes)

    def close(self):
        if self.h:
            pbdr_ctx_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def create_scene(self, scene) -> int:
        return pbdr_create_scene(self.h, scene)

    def destroy_scene(self, sid: int):
        pbdr_destroy_scene(self.h, sid)

    def step(self, ids, substeps: int = 1, stream=None):
        if isinstance(ids, (int, np.integer)):
            ids = [int(ids)]
        pbdr_step(self.h, ids, substeps, stream)

    def read_state(self, sid: int, stream=None):
        return pbdr_read_state(self.h, sid, stream)

    def write_state(self, sid: int, pos=None, vel=None, stream=None):
        pbdr_write_state(self.h, sid, pos, vel, stream)

    def read_states(self, ids, pos=None, vel=None, stream=None):
        return pbdr_read_states(self.h, ids, pos, vel, stream)

    def read_states_async(self, ids, pos, vel, err, stream=None):
        pbdr_read_states_async(self.h, ids, pos, vel, err, stream)

    def write_states(self, ids, pos=None, vel=None, stream=None):
        pbdr_write_states(self.h, ids, pos, vel, stream)

    def step_tangent(self, ids, substeps: int = 1, stream=None):
        if isinstance(ids, (int, np.integer)):
            ids = [int(ids)]
        pbdr_step_tangent(self.h, ids, substeps, stream)

    def write_tangent(self, sid: int, dpos=None, dvel=None, stream=None):
        pbdr_write_tangent(self.h, sid, dpos, dvel, stream)

    def read_tangent(self, sid: int, stream=None):
        return pbdr_read_tangent(self.h, sid, stream)

    def adjoint(self, ids, substeps: int, checkpoint_every: int = 20, stream=None):
        if isinstance(ids, (int, np.integer)):
            ids = [int(ids)]
        pbdr_adjoint(self.h, ids, substeps, checkpoint_every, stream)

    def write_adjoint(self, sid: int, xbar=None, vbar=None, stream=None):
        pbdr_write_adjoint(self.h, sid, xbar, vbar, stream)

    def read_adjoint(self, sid: int, stream=None):
        return pbdr_read_adjoint(self.h, sid, stream)

    def write_tangent_friction(self, sid: int, dmu: float, stream=None):
        pbdr_write_tangent_friction(self.h, sid, dmu, stream)

    def read_adjoint_friction(self, sid: int, stream=None) -> float:
        return pbdr_read_adjoint_friction(self.h, sid, stream)

    def build_neighbors(self, ids, stream=None):
        if isinstance(ids, (int, np.integer)):
            ids = [int(ids)]
        pbdr_build_neighbors(self.h, ids, stream)

    def read_neighbors(self, sid: int, stream=None, lists_only: bool = False):
        return pbdr_read_neighbors(self.h, sid, stream, lists_only)

    def set_option(self, option: int, value: int):
        pbdr_set_option(self.h, option, value)

    def plan_config(self, ids):
        return pbdr_plan_config(self.h, ids)

    def set_path(self, streaming: bool):
        pbdr_set_option(self.h, OPT_PATH, 1 if streaming else 0)

    def set_body_wrench(self, sid: int, body: int, F, tau):
        pbdr_set_body_wrench(self.h, sid, body, F, tau)

    def scene_info(self, sid: int):
        return pbdr_scene_info(self.h, sid)

    def last_launch_count(self) -> int:
        return pbdr_last_launch_count(self.h)

    def neighbor_total(self, ids, stream=None) -> int:
        return pbdr_neighbor_total(self.h, ids, stream)

    def set_profiling(self, enable: bool):
        pbdr_set_profiling(self.h, enable)

    def read_profile(self):
        return pbdr_read_profile(self.h)
