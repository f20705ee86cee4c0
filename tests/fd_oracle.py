"""Reference derivatives for the tangent tests: central finite differences of
the FP64 oracle's final body centres of mass with respect to per-body rigid
velocities (v_b, omega_b).  Test infrastructure only."""
import numpy as np

from paper_2603_14634_gb300 import diff, scenes


def final_coms(orc, scene, steps):
    return diff.body_coms(scene, orc.OracleScene(scene).substep(steps).x)


def rigid_fd_jacobian(orc, scene, v_lin, w_ang, steps, h=1e-4):
    """d(final CoM [3B]) / d(v, omega [6B]) by central differences (FP64)."""
    B = scene.num_bodies
    J = np.zeros((3 * B, 6 * B))
    for b in range(B):
        for k in range(6):
            out = []
            for sgn in (1.0, -1.0):
                v = np.array(v_lin, np.float64).copy()
                w = np.array(w_ang, np.float64).copy()
                (v if k < 3 else w)[b, k % 3] += sgn * h
                sc = scenes.Scene(**{**scene.__dict__})
                sc.vel = diff.rigid_velocity(scene, v, w)
                out.append(final_coms(orc, sc, steps).reshape(-1))
            J[:, 6 * b + k] = (out[0] - out[1]) / (2 * h)
    return J


def sliding_grid(seed=0, nx=2, n=4, mu=0.3, speed=(1.0, 1.5), spin=1.0):
    """nx^2 boxes of n^3 resting on the plane (0.6 m pitch), each sliding at
    a speed in ``speed`` in a random horizontal direction and spinning about
    z at up to ``spin`` rad/s: every particle slides for the first 0.2 s."""
    rng = np.random.default_rng(seed)
    sc = scenes.resting_grid_scene(seed=seed, nx=nx, n=n, friction=mu)
    B = sc.num_bodies
    ang = rng.random(B) * 2 * np.pi
    sp = speed[0] + rng.random(B) * (speed[1] - speed[0])
    v = np.stack([sp * np.cos(ang), sp * np.sin(ang), np.zeros(B)], 1)
    w = np.zeros((B, 3))
    w[:, 2] = (rng.random(B) * 2 - 1) * spin
    sc.vel = diff.rigid_velocity(sc, v, w).astype(np.float32)
    return sc, v, w


def mu_fd(orc, scene, steps, h=1e-4):
    """d(final CoM [3B]) / d(mu) by central differences (FP64)."""
    out = []
    for sgn in (1.0, -1.0):
        sc = scenes.Scene(**{**scene.__dict__})
        sc.friction = float(scene.friction) + sgn * h
        out.append(final_coms(orc, sc, steps).reshape(-1))
    return (out[0] - out[1]) / (2 * h)


def _fd_column(args):
    """One central-difference column (runs in a spawned worker)."""
    from oracle import oracle as orc
    scene_dict, v_lin, w_ang, b, k, steps, h = args
    scene = scenes.Scene(**scene_dict)
    out = []
    for sgn in (1.0, -1.0):
        if b < 0:   # the friction coefficient
            sc = scenes.Scene(**scene_dict)
            sc.friction = float(scene.friction) + sgn * h
        else:
            v = np.array(v_lin, np.float64).copy()
            w = np.array(w_ang, np.float64).copy()
            (v if k < 3 else w)[b, k % 3] += sgn * h
            sc = scenes.Scene(**scene_dict)
            sc.vel = diff.rigid_velocity(scene, v, w)
        out.append(final_coms(orc, sc, steps).reshape(-1))
    return (out[0] - out[1]) / (2 * h)


def rigid_mu_fd_jacobian_parallel(scene, v_lin, w_ang, steps, h=1e-4, workers=None):
    """d(final CoM [3B]) / d(v, omega [6B], mu) [3B, 6B + 1] by central
    differences of the FP64 oracle, one column per task on a pool of
    spawned processes (never forked: the caller may hold a CUDA context)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    B = scene.num_bodies
    d = dict(scene.__dict__)
    tasks = [(d, v_lin, w_ang, b, k, steps, h) for b in range(B) for k in range(6)]
    tasks.append((d, v_lin, w_ang, -1, 0, steps, h))
    workers = workers or min(16, os.cpu_count() or 1)
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        cols = list(ex.map(_fd_column, tasks))
    return np.stack(cols, 1)
