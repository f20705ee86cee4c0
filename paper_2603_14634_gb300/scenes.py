"""Seeded synthetic scene generators for the PBD-R solver.

This module only builds *inputs*: lattice-packed rigid bodies (uniformly
spaced, non-overlapping equal spheres, the packing of Sec. IV-B "Shape
Representations"), random poses, initial velocities and the per-scene
physical parameters.  It holds none of the solver's arithmetic (no rest
offsets, no centre of mass, no contact or shape-matching math), so both the
CUDA path and the FP64 CPU oracle can consume the same arrays without sharing
any of the method's code.

Every generator is deterministic given its seed (``numpy.random.default_rng``).
Positions, velocities and inverse masses are returned as FP32 arrays because
the solver state is FP32 (Sec. IV-B "Implementation Details").
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# flag bits of pbdr_scene_desc.flags (mirrors include/pbdr.h)
STD_VELOCITY = 1 << 0   # standard PBD velocity update V = (X - X_init)/dt
NO_LINMOM = 1 << 1      # drop the linear-momentum correction
NO_ANGMOM = 1 << 2      # drop the angular-momentum correction
CONTACT_AVG = 1 << 3    # average particle-particle corrections over active contacts
SM_FROM_XI = 1 << 4     # shape matching on X_i instead of X_i + contact corrections

GRAVITY = 9.81


@dataclasses.dataclass
class Scene:
    """One independent scene: bodies are contiguous particle ranges."""
    pos: np.ndarray            # [N,3] float32
    vel: np.ndarray            # [N,3] float32
    inv_mass: np.ndarray       # [N] float32 (> 0)
    body_off: np.ndarray       # [B+1] int32, body b = [body_off[b], body_off[b+1])
    radius: float = 0.05
    friction: float = 0.5
    gravity: Sequence[float] = (0.0, 0.0, -GRAVITY)
    plane: Sequence[float] = (0.0, 0.0, 1.0, 0.0)   # n (unit), d : n.x = d
    dt: float = 1.0 / 240.0
    iterations: int = 10
    flags: int = 0
    # optional constant wrench at each body's centre of mass: [B,3] each
    force: Optional[np.ndarray] = None
    torque: Optional[np.ndarray] = None

    @property
    def num_particles(self) -> int:
        return int(self.pos.shape[0])

    @property
    def num_bodies(self) -> int:
        return int(self.body_off.shape[0] - 1)

    def copy(self) -> "Scene":
        return dataclasses.replace(
            self, pos=self.pos.copy(), vel=self.vel.copy(),
            inv_mass=self.inv_mass.copy(), body_off=self.body_off.copy(),
            force=None if self.force is None else self.force.copy(),
            torque=None if self.torque is None else self.torque.copy())


# --------------------------------------------------------------------------
# geometry helpers (input construction only)
# --------------------------------------------------------------------------

def lattice_cube(n: int, spacing: float) -> np.ndarray:
    """n^3 lattice points with the given spacing, centred at the origin.

    Point order: x fastest, then y, then z (so the bottom layer comes first).
    """
    ax = (np.arange(n, dtype=np.float64) - (n - 1) / 2.0) * spacing
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def random_rotations(rng: np.random.Generator, k: int) -> np.ndarray:
    """k uniform random rotation matrices [k,3,3] (Shoemake 1992 quaternion
    sampling)."""
    u = rng.random((k, 3))
    a, b = np.sqrt(1.0 - u[:, 0]), np.sqrt(u[:, 0])
    x, y = a * np.sin(2 * np.pi * u[:, 1]), a * np.cos(2 * np.pi * u[:, 1])
    z, w = b * np.sin(2 * np.pi * u[:, 2]), b * np.cos(2 * np.pi * u[:, 2])
    R = np.empty((k, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """One uniform random rotation matrix."""
    return random_rotations(rng, 1)[0]


def _assemble(bodies_pos, bodies_vel, mass_per_particle=1.0, **params) -> Scene:
    pos = np.concatenate(bodies_pos, axis=0).astype(np.float32)
    vel = np.concatenate(bodies_vel, axis=0).astype(np.float32)
    sizes = [b.shape[0] for b in bodies_pos]
    body_off = np.zeros(len(sizes) + 1, dtype=np.int32)
    body_off[1:] = np.cumsum(sizes)
    inv_mass = np.full(pos.shape[0], 1.0 / mass_per_particle, dtype=np.float32)
    return Scene(pos=pos, vel=vel, inv_mass=inv_mass, body_off=body_off, **params)


def _obb_separated(ca, Ra, ea, cb, Rb, eb):
    """Separating-axis test between oriented cubes (Gottschalk et al. 1996).

    ca [K,3], Ra [K,3,3] (columns = axes), ea [K]: candidate cubes;
    cb [P,3], Rb [P,3,3], eb [P]: placed cubes.  Returns a [K,P] bool array,
    True where the two cubes (half extents ea, eb) do not intersect.
    """
    eps = 1e-9
    C = np.einsum("kai,paj->kpij", Ra, Rb)                 # C_ij = A_i . B_j
    A = np.abs(C) + eps
    T = cb[None, :, :] - ca[:, None, :]
    t = np.einsum("kai,kpa->kpi", Ra, T)                   # T in A's frame
    ea = ea[:, None]
    eb = eb[None, :]
    sep = np.zeros(C.shape[:2], dtype=bool)
    for i in range(3):
        sep |= np.abs(t[..., i]) > ea + eb * A[..., i, :].sum(-1)
    tb = np.einsum("kpi,kpij->kpj", t, C)
    for j in range(3):
        sep |= np.abs(tb[..., j]) > ea * A[..., :, j].sum(-1) + eb
    for i in range(3):
        i1, i2 = (i + 1) % 3, (i + 2) % 3
        for j in range(3):
            j1, j2 = (j + 1) % 3, (j + 2) % 3
            ra = ea * (A[..., i1, j] + A[..., i2, j])
            rb = eb * (A[..., i, j1] + A[..., i, j2])
            proj = np.abs(t[..., i2] * C[..., i1, j] - t[..., i1] * C[..., i2, j])
            sep |= proj > ra + rb
    return sep


def place_bodies(rng: np.random.Generator, lattice_sizes: Sequence[int], *,
                 spacing: float = 0.1, radius: float = 0.05,
                 box_lo=(-1.0, -1.0, 0.0), box_hi=(1.0, 1.0, 2.0),
                 vmax: float = 1.0, wmax: float = 2.0,
                 max_fail: int = 256, grow_z: float = 0.5, batch: int = 64):
    """Random non-overlapping placement of n^3 lattice bodies in a box.

    Each body gets a uniform random orientation and a centre uniform in the box
    shrunk by the body's bounding radius.  A candidate is rejected when its
    cube (particle centres' extent grown by r) intersects the grown cube of an
    already placed body, which guarantees that no two particles of different
    bodies start closer than 2r.  After ``max_fail`` rejections the box grows
    by ``grow_z`` in +z.  Candidates are drawn ``batch`` at a time and the
    first valid one (in draw order) is kept.
    Linear velocity ~ U[-vmax, vmax]^3, angular velocity ~ U[-wmax, wmax]^3;
    each particle gets the rigid velocity v + w x (x - centre).
    """
    lo = np.array(box_lo, dtype=np.float64)
    hi = np.array(box_hi, dtype=np.float64)
    ctrs = np.zeros((0, 3))
    rots = np.zeros((0, 3, 3))
    halfs = np.zeros(0)
    out_pos: List[np.ndarray] = []
    vels: List[np.ndarray] = []
    for n in lattice_sizes:
        local = lattice_cube(n, spacing)
        half = (n - 1) / 2.0 * spacing + radius
        brad = math.sqrt(3.0) * half
        fails = 0
        while True:
            Rs = random_rotations(rng, batch)
            lo_c = lo + brad
            hi_c = np.maximum(hi - brad, lo_c)
            cs = lo_c + rng.random((batch, 3)) * (hi_c - lo_c)
            if ctrs.shape[0]:
                sep = _obb_separated(cs, Rs, np.full(batch, half), ctrs, rots, halfs)
                good = np.nonzero(sep.all(axis=1))[0]
            else:
                good = np.arange(1)
            if good.size:
                k = int(good[0])
                break
            fails += batch
            if fails >= max_fail:
                hi[2] += grow_z
                fails = 0
        R, ctr = Rs[k], cs[k]
        cand = local @ R.T + ctr
        v = (rng.random(3) * 2 - 1) * vmax
        w = (rng.random(3) * 2 - 1) * wmax
        ctrs = np.vstack([ctrs, ctr[None, :]])
        rots = np.concatenate([rots, R[None]], axis=0)
        halfs = np.append(halfs, half)
        out_pos.append(cand)
        vels.append(v[None, :] + np.cross(w[None, :], cand - ctr[None, :]))
    return out_pos, vels


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------

def cube_drop(n: int = 4, spacing: float = 0.1, radius: float = 0.05,
              clearance: float = 1.0, friction: float = 0.5,
              dt: float = 1.0 / 240.0, iterations: int = 10,
              mass_per_particle: float = 1.0, flags: int = 0) -> Scene:
    """One n^3 cube whose bottom surface starts ``clearance`` above z = 0.

    Default: 4x4x4 = 64 particles, r = 0.05 m, spacing 0.1 m, unit mass each,
    dropped from 1 m, friction 0.5, g = -9.81, dt = 1/240, 10 iterations.
    """
    p = lattice_cube(n, spacing)
    p[:, 2] += clearance + radius - p[:, 2].min()
    return _assemble([p], [np.zeros_like(p)], mass_per_particle, radius=radius,
                     friction=friction, dt=dt, iterations=iterations, flags=flags)


def random_bodies_scene(seed: int = 0, num_bodies: int = 64, n: int = 5,
                        friction: float = 0.5, dt: float = 1.0 / 240.0,
                        iterations: int = 20) -> Scene:
    """64 rigid 5^3 bodies (8000 particles, r = 0.05 m) with seeded uniform
    random poses in a 2x2x2 m box, linear velocity U[-1,1] m/s and angular
    velocity U[-2,2] rad/s, friction 0.5, dt = 1/240, 20 iterations."""
    rng = np.random.default_rng(seed)
    pos, vel = place_bodies(rng, [n] * num_bodies)
    return _assemble(pos, vel, 1.0, friction=friction, dt=dt, iterations=iterations)


BATCH_LATTICE_SIZES = (3, 4, 5, 7)   # 27, 64, 125, 343 particles


def batch_scene(rng: np.random.Generator, max_bodies: int = 32,
                iterations: int = 10, dt: float = 1.0 / 240.0,
                friction: float = 0.5) -> Scene:
    """One scene of the batched workload: n_b = floor(exp(U ln(max_bodies+1)))
    bodies (log-uniform in [1, max_bodies]), each an n^3 lattice body with n
    uniform in {3, 4, 5, 7}, placed and launched as in random_bodies_scene."""
    nb = int(math.floor(math.exp(rng.random() * math.log(max_bodies + 1))))
    nb = min(max(nb, 1), max_bodies)
    sizes = [BATCH_LATTICE_SIZES[i] for i in rng.integers(0, len(BATCH_LATTICE_SIZES), nb)]
    pos, vel = place_bodies(rng, sizes)
    return _assemble(pos, vel, 1.0, friction=friction, dt=dt, iterations=iterations)


def _batch_scene_from_seed(args):
    seed_seq, kw = args
    return batch_scene(np.random.default_rng(seed_seq), **kw)


def batched_scenes(num_scenes: int = 4096, seed: int = 0, workers: int = 0,
                   **kw) -> List[Scene]:
    """The batched workload: ``num_scenes`` independent uneven scenes
    (4096 scenes, 1-32 bodies of {27,64,125,343} particles, ~5M particles).

    Scene k draws from its own child stream ``SeedSequence(seed).spawn(n)[k]``,
    so the result does not depend on ``workers`` (processes used to build the
    scenes; 0 = serial).
    """
    children = np.random.SeedSequence(seed).spawn(num_scenes)
    jobs = [(c, kw) for c in children]
    if workers and workers > 1 and num_scenes > 64:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            return pool.map(_batch_scene_from_seed, jobs, chunksize=16)
    return [_batch_scene_from_seed(j) for j in jobs]


def stacked_block_scene(seed: int = 0, nb: int = 5, n: int = 4, pitch: float = 0.4,
                        tilt_deg: float = 0.5, shift: float = 0.002, friction: float = 0.5,
                        dt: float = 1.0 / 240.0, iterations: int = 20) -> Scene:
    """A contact-dense scene: nb^3 rigid n^3 bodies (spacing 0.1 m, r = 0.05 m)
    stacked in a block on the ground, at rest, with a pitch that puts the
    facing particles of neighbouring bodies one diameter apart; every body is
    tilted by up to ``tilt_deg`` about a random axis and shifted by up to
    ``shift`` m, so the faces are not exactly aligned.  Defaults: 125 bodies
    of 4^3 (8000 particles, the size of the 64-body scene), 20 iterations;
    after a tenth of a second the particles average about one neighbour."""
    rng = np.random.default_rng(seed)
    spacing = 0.1
    base = lattice_cube(n, spacing)
    base = base - base.mean(0)
    half = 0.5 * (n - 1) * spacing
    pos, vel = [], []
    for iz in range(nb):
        for iy in range(nb):
            for ix in range(nb):
                axis = rng.normal(size=3)
                axis /= np.linalg.norm(axis)
                ang = math.radians(tilt_deg) * rng.uniform(-1.0, 1.0)
                K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
                R = np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)
                c = np.array([ix * pitch, iy * pitch, 0.05 + half + iz * pitch + 0.002 * iz])
                c[:2] -= 0.5 * (nb - 1) * pitch
                c = c + rng.uniform(-shift, shift, size=3) * np.array([1.0, 1.0, 0.0])
                pos.append(base @ R.T + c)
                vel.append(np.zeros_like(base))
    return _assemble(pos, vel, 1.0, friction=friction, dt=dt, iterations=iterations)


def _stacked_from_seed(args):
    seed, kw = args
    return stacked_block_scene(seed=seed, **kw)


def stacked_block_scenes(num_scenes: int, seed: int = 0, workers: int = 0, **kw) -> List[Scene]:
    """``num_scenes`` stacked blocks (seeds seed, seed+1, ...)."""
    jobs = [(seed + k, kw) for k in range(num_scenes)]
    if workers and workers > 1 and num_scenes > 16:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            return pool.map(_stacked_from_seed, jobs, chunksize=4)
    return [_stacked_from_seed(j) for j in jobs]


def resting_grid_scene(seed: int = 0, nx: int = 4, n: int = 5, pitch: float = 0.6,
                       friction: float = 0.5, dt: float = 1.0 / 240.0,
                       iterations: int = 10, radius: float = 0.05,
                       spacing: float = 0.1) -> Scene:
    """16 rigid 5^3 bodies resting on the plane in a 4x4 grid (0.6 m pitch)
    with horizontal velocities U[-1,1] m/s (sliding regime)."""
    rng = np.random.default_rng(seed)
    local = lattice_cube(n, spacing)
    local[:, 2] += radius - local[:, 2].min()
    pos, vel = [], []
    for i in range(nx):
        for j in range(nx):
            ctr = np.array([(i - (nx - 1) / 2) * pitch, (j - (nx - 1) / 2) * pitch, 0.0])
            p = local + ctr
            v = np.zeros_like(p)
            v[:, :2] = (rng.random(2) * 2 - 1)[None, :]
            pos.append(p)
            vel.append(v)
    return _assemble(pos, vel, 1.0, friction=friction, dt=dt, iterations=iterations,
                     radius=radius)


def analytic_box(test: int, n: int = 4, box_mass: float = 4.0, spacing: float = 0.1,
                 radius: float = 0.05, dt: float = 1e-3, iterations: int = 10) -> Scene:
    """Box of the analytic physics tests (Table I) with Table II parameters.

    test 1: pushed box, F = 17 N along +x at the CoM, mu = 0.4
    test 2: box with torque, tau = 0.01 N m about +z, mu = 0
    test 3: box on a slope of pi/8, mu = 0.4 (gravity tilted; plane z = 0)
    The box rests on the plane (bottom layer centres at z = r), zero velocity.
    """
    p = lattice_cube(n, spacing)
    p[:, 2] += radius - p[:, 2].min()
    m = box_mass / p.shape[0]
    params = dict(radius=radius, dt=dt, iterations=iterations)
    B = 1
    if test == 1:
        params["friction"] = 0.4
        sc = _assemble([p], [np.zeros_like(p)], m, **params)
        sc.force = np.array([[17.0, 0.0, 0.0]] * B, dtype=np.float32)
    elif test == 2:
        params["friction"] = 0.0
        sc = _assemble([p], [np.zeros_like(p)], m, **params)
        sc.torque = np.array([[0.0, 0.0, 0.01]] * B, dtype=np.float32)
    elif test == 3:
        th = math.pi / 8
        params["friction"] = 0.4
        # the slope is expressed by tilting gravity in the plane's frame:
        # downhill = +x, normal = +z
        params["gravity"] = (GRAVITY * math.sin(th), 0.0, -GRAVITY * math.cos(th))
        sc = _assemble([p], [np.zeros_like(p)], m, **params)
    else:
        raise ValueError("analytic test must be 1, 2 or 3")
    return sc


def lattice_placement(rng: np.random.Generator, lattice_sizes: Sequence[int], *,
                      spacing: float = 0.1, radius: float = 0.05, vmax: float = 1.0,
                      wmax: float = 2.0, z0: float = 0.0):
    """Fast non-overlapping placement for large requests: bodies go to the
    cells of a cubic lattice whose pitch is the largest bounding diameter
    (+2r), in random order, each with a uniform random rotation and a random
    shift within its cell's slack; the lattice's base rests at height z0.
    Velocities as in place_bodies."""
    halfs = [(n - 1) / 2.0 * spacing for n in lattice_sizes]
    brad = max(math.sqrt(3.0) * h + radius for h in halfs)
    pitch = 2.0 * brad + 2.0 * radius
    nb = len(lattice_sizes)
    side = int(math.ceil(nb ** (1.0 / 3.0)))
    cells = rng.permutation(side ** 3)[:nb]
    Rs = random_rotations(rng, nb)
    pos, vel = [], []
    for k, n in enumerate(lattice_sizes):
        c = cells[k]
        ijk = np.array([c % side, (c // side) % side, c // (side * side)], dtype=np.float64)
        my = math.sqrt(3.0) * halfs[k] + radius
        slack = max(0.0, brad - my)
        ctr = (ijk - (side - 1) / 2.0) * pitch + (rng.random(3) * 2 - 1) * slack
        ctr[2] += z0 + (side - 1) / 2.0 * pitch + brad
        p = lattice_cube(n, spacing) @ Rs[k].T + ctr
        v = (rng.random(3) * 2 - 1) * vmax
        w = (rng.random(3) * 2 - 1) * wmax
        pos.append(p)
        vel.append(v[None, :] + np.cross(w[None, :], p - ctr[None, :]))
    return pos, vel


def serving_request(rng: np.random.Generator, min_particles: int = 1000,
                    max_particles: int = 200000, iterations: int = 10,
                    dt: float = 1.0 / 240.0, friction: float = 0.5):
    """One serving request: particle target P log-uniform in [1e3, 2e5]; n^3
    bodies with n ~ U{4..8} (64-512 particles) added until >= P, placed by
    lattice_placement; returns (scene, steps) with steps ~ U{1..100}."""
    P = math.exp(math.log(min_particles) + rng.random() *
                 (math.log(max_particles) - math.log(min_particles)))
    sizes, total = [], 0
    while total < P:
        n = int(rng.integers(4, 9))
        sizes.append(n)
        total += n ** 3
    pos, vel = lattice_placement(rng, sizes)
    sc = _assemble(pos, vel, 1.0, friction=friction, dt=dt, iterations=iterations)
    steps = int(rng.integers(1, 101))
    return sc, steps
