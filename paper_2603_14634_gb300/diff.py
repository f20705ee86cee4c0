"""Differentiable PBD-R on the GPU: forward-mode tangents and reverse-mode
adjoints of the substep.

``pbdr_step_tangent`` advances a scene and a tangent (dX, dV) of its state
together: the derivative of the substep map (Algorithm 1) along one
direction of the initial state.  Many directions of one scene run as copies
of that scene in ONE batched call, so a whole Jacobian over a few rigid
parameters per body costs one batched run.  ``pbdr_adjoint`` takes the
gradient of a scalar loss of the final state back to the initial state
(checkpoints every ``checkpoint_every`` substeps, recomputation in between),
at a cost independent of the number of parameters.

Parameters differentiated here: the initial rigid velocity of every body,
v_b (3) and omega_b (3); its velocity field is v_b + omega_b x (x - c_b)
(c_b = initial centre of mass).  Output: the final centre of mass of every
body after ``steps`` substeps.  ``FinalCoM`` is a ``torch.autograd.Function``
whose backward returns J^T g, from the tangents (``mode="forward"``: the
Jacobian is formed in the forward pass) or from one adjoint run per backward
call (``mode="reverse"``).
"""
from __future__ import annotations

from typing import List, Optional, Tuple

import numpy as np

from . import scenes as _scenes


def body_slices(scene) -> List[slice]:
    off = np.asarray(scene.body_off)
    return [slice(int(off[b]), int(off[b + 1])) for b in range(len(off) - 1)]


def body_coms(scene, pos: np.ndarray) -> np.ndarray:
    """Centre of mass of every body, [B, 3] (FP64)."""
    m = 1.0 / np.asarray(scene.inv_mass, np.float64)
    p = np.asarray(pos, np.float64)
    return np.stack([(m[s, None] * p[s]).sum(0) / m[s].sum() for s in body_slices(scene)])


def rigid_velocity(scene, v_lin: np.ndarray, w_ang: np.ndarray) -> np.ndarray:
    """Particle velocities of per-body rigid motions (v_b, omega_b), [N, 3]."""
    c = body_coms(scene, scene.pos)
    out = np.zeros((scene.num_particles, 3), np.float64)
    p = np.asarray(scene.pos, np.float64)
    for b, s in enumerate(body_slices(scene)):
        out[s] = np.asarray(v_lin[b], np.float64) + np.cross(np.asarray(w_ang[b], np.float64), p[s] - c[b])
    return out


def rigid_seeds(scene) -> List[np.ndarray]:
    """Tangent seeds dV of the 6 B rigid parameters, in the order
    (v_0x, v_0y, v_0z, w_0x, w_0y, w_0z, v_1x, ...)."""
    B = scene.num_bodies
    seeds = []
    for b in range(B):
        for k in range(6):
            v = np.zeros((B, 3))
            w = np.zeros((B, 3))
            (v if k < 3 else w)[b, k % 3] = 1.0
            seeds.append(rigid_velocity(scene, v, w))
    return seeds


MU = "mu"   # seed: the friction coefficient


def com_jacobian(ctx, scene, steps: int, seeds: List, stream=None,
                 batch: Optional[int] = None) -> Tuple[np.ndarray, np.ndarray]:
    """Final body centres of mass [B, 3] and their Jacobian [3B, S] along
    the seeds: velocity tangents dV ([N, 3] each) or ``MU`` (the friction
    coefficient).  Every seed runs as one copy of the scene; copies go
    through ``pbdr_step_tangent`` together (``batch`` at a time)."""
    batch = batch or len(seeds)
    m = 1.0 / np.asarray(scene.inv_mass, np.float64)
    sl = body_slices(scene)
    J = np.zeros((3 * scene.num_bodies, len(seeds)))
    final = None
    for at in range(0, len(seeds), batch):
        group = seeds[at:at + batch]
        ids = []
        try:
            for _ in group:
                ids.append(ctx.create_scene(scene))
            for sid, dv in zip(ids, group):
                if isinstance(dv, str):
                    ctx.write_tangent(sid, None, None, stream)
                    ctx.write_tangent_friction(sid, 1.0, stream)
                else:
                    ctx.write_tangent(sid, None, np.asarray(dv, np.float32), stream)
            ctx.step_tangent(ids, steps, stream)
            for j, sid in enumerate(ids):
                dpos, _ = ctx.read_tangent(sid, stream)
                dp = dpos.astype(np.float64)
                J[:, at + j] = np.concatenate([(m[s, None] * dp[s]).sum(0) / m[s].sum() for s in sl])
                if final is None:
                    pos, _, err = ctx.read_state(sid, stream)
                    if err:
                        raise RuntimeError(f"device error bits {err}")
                    final = body_coms(scene, pos)
        finally:
            for sid in ids:
                ctx.destroy_scene(sid)
    return final, J


def _with_velocity(scene, vel: np.ndarray):
    import copy
    sc = copy.copy(scene)
    sc.vel = np.asarray(vel, np.float32)
    return sc


def final_com_and_jacobian(ctx, scene, v_lin: np.ndarray, w_ang: np.ndarray, steps: int,
                           stream=None, with_mu: bool = False) -> Tuple[np.ndarray, np.ndarray]:
    """Final centres of mass [B, 3] of the scene started with per-body rigid
    velocities (v_lin, w_ang) [B, 3] each, and d(final CoM)/d(v, omega)
    [3B, 6B] (parameter order of ``rigid_seeds``), with a last column
    d/d(mu) when ``with_mu``."""
    sc = _with_velocity(scene, rigid_velocity(scene, v_lin, w_ang))
    seeds = rigid_seeds(sc) + ([MU] if with_mu else [])
    return com_jacobian(ctx, sc, steps, seeds, stream)


def com_loss_adjoint(scene, weights: np.ndarray) -> np.ndarray:
    """dL/dX of L = sum_b weights_b . c_b (c_b = body centre of mass): each
    particle of body b gets weights_b m_p / M_b.  [N, 3]."""
    m = 1.0 / np.asarray(scene.inv_mass, np.float64)
    out = np.zeros((scene.num_particles, 3))
    for b, s in enumerate(body_slices(scene)):
        out[s] = np.asarray(weights[b], np.float64)[None, :] * (m[s] / m[s].sum())[:, None]
    return out


def rigid_gradient(scene, vbar0: np.ndarray) -> np.ndarray:
    """dL/d(v_b, omega_b) [B, 6] from dL/dV of the initial particle
    velocities (V = v_b + omega_b x (x - c_b))."""
    p = np.asarray(scene.pos, np.float64)
    c = body_coms(scene, scene.pos)
    vb = np.asarray(vbar0, np.float64)
    out = np.zeros((scene.num_bodies, 6))
    for b, s in enumerate(body_slices(scene)):
        out[b, :3] = vb[s].sum(0)
        out[b, 3:] = np.cross(p[s] - c[b], vb[s]).sum(0)
    return out


def final_com(ctx, scene, v_lin: np.ndarray, w_ang: np.ndarray, steps: int, stream=None) -> np.ndarray:
    """Final centres of mass [B, 3] of the scene started with per-body rigid
    velocities (v_lin, w_ang), by plain substeps."""
    sc = _with_velocity(scene, rigid_velocity(scene, v_lin, w_ang))
    sid = ctx.create_scene(sc)
    try:
        ctx.step(sid, steps, stream)
        pos, _, err = ctx.read_state(sid, stream)
        if err:
            raise RuntimeError(f"device error bits {err}")
    finally:
        ctx.destroy_scene(sid)
    return body_coms(sc, pos)


def com_gradient_reverse(ctx, scene, v_lin: np.ndarray, w_ang: np.ndarray, steps: int,
                         weights: np.ndarray, checkpoint_every: int = 20,
                         stream=None, with_mu: bool = False):
    """Final centres of mass [B, 3] and dL/d(v_b, omega_b) [B, 6] of
    L = sum_b weights_b . c_b(final), by one adjoint run (and dL/dmu as a
    third value when ``with_mu``).  L is linear in the final state, so its
    adjoint is known before the run; for other losses, step forward first,
    form dL/dX_final, restore the initial state with write_state and then
    call adjoint."""
    sc = _with_velocity(scene, rigid_velocity(scene, v_lin, w_ang))
    sid = ctx.create_scene(sc)
    try:
        ctx.write_adjoint(sid, com_loss_adjoint(sc, weights).astype(np.float32), None, stream)
        ctx.adjoint(sid, steps, checkpoint_every, stream)
        pos, _, err = ctx.read_state(sid, stream)
        if err:
            raise RuntimeError(f"device error bits {err}")
        _, vbar0 = ctx.read_adjoint(sid, stream)
        mubar = ctx.read_adjoint_friction(sid, stream) if with_mu else None
    finally:
        ctx.destroy_scene(sid)
    if with_mu:
        return body_coms(sc, pos), rigid_gradient(sc, vbar0), mubar
    return body_coms(sc, pos), rigid_gradient(sc, vbar0)


try:   # the autograd wrapper needs torch; the rest of the module does not
    import torch

    class FinalCoM(torch.autograd.Function):
        """final CoMs [B, 3] = f(v_lin [B, 3], w_ang [B, 3]) through
        ``steps`` PBD-R substeps on the GPU; backward = J^T grad, with J from
        the forward-mode tangents (mode "forward") or by one adjoint run
        (mode "reverse")."""

        @staticmethod
        def forward(fctx, v_lin, w_ang, ctx, scene, steps, mode="forward"):
            v = v_lin.detach().cpu().double().numpy()
            w = w_ang.detach().cpu().double().numpy()
            fctx.B = scene.num_bodies
            fctx.mode = mode
            if mode == "forward":
                final, J = final_com_and_jacobian(ctx, scene, v, w, int(steps))
                fctx.save_for_backward(torch.from_numpy(J))
            elif mode == "reverse":
                # primal only; the one adjoint run happens in backward
                final = final_com(ctx, scene, v, w, int(steps))
                fctx.args = (ctx, scene, v, w, int(steps))
            else:
                raise ValueError("mode is 'forward' or 'reverse'")
            return torch.from_numpy(final).to(v_lin.dtype)

        @staticmethod
        def backward(fctx, grad):
            g = grad.detach().double().cpu()
            if fctx.mode == "forward":
                (J,) = fctx.saved_tensors
                gp = (J.T @ g.reshape(-1)).reshape(fctx.B, 6)
            else:
                ctx, scene, v, w, steps = fctx.args
                _, gp = com_gradient_reverse(ctx, scene, v, w, steps, g.numpy())
                gp = torch.from_numpy(gp)
            return gp[:, :3].to(grad.dtype), gp[:, 3:].to(grad.dtype), None, None, None, None

except ImportError:   # pragma: no cover
    FinalCoM = None


def c5_scene(seed: int = 0, **kw):
    """16 bodies of 5^3 resting in a 4x4 grid, 0.6 m pitch, horizontal
    velocities U[-1, 1] m/s, mu = 0.5, K = 10, dt = 1/240."""
    return _scenes.resting_grid_scene(seed=seed, **kw)
