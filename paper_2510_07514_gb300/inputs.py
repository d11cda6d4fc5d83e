"""Seeded synthetic workloads for batched HJCD-IK.

This module is the only code shared by the FP64 oracle and the CUDA path.  It
holds configuration tables and random draws only: robot descriptions (DH
tables, joint limits, link spheres, self-collision ignore masks), obstacle
scenes, joint-space samples whose forward kinematics each side computes with
its own code, per-target seed counts, and the algorithm's parameter table.
It contains no kinematics, no residuals and no collision tests.

Workload recipe (stands in for the paper's Halton-sampled Panda targets, the
MotionBenchMaker ``box_panda`` scene and the ``foam`` sphere models, none of
which are available here; Sec. VI):

* Panda chain: modified DH (Craig), 7 revolute joints, flange Tz(0.107).
* Link spheres: ``per_body`` spheres per body on the segment from the body's
  frame origin to the next joint's origin (expressed in the body frame; the
  flange body extends 0.1 m along its z axis), radii uniform in a range.
* Scene: spheres and axis-aligned boxes uniform in a box around the base,
  none of them inside a keep-out cylinder around the base axis (a sampling
  region, not a collision test).
* Targets: the pose of a joint sample drawn uniformly inside the limits; each
  consumer computes the pose (and, with a scene, keeps only samples it finds
  collision-free) with its own kinematics.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Generator seed for workload k (1-based).
CFG_SEED = {k: 0x484A4344_00000000 + k for k in range(1, 6)}

# Parameter table of the algorithm (Alg. 2-4).  The paper names these only
# symbolically; the values are this implementation's readings.  Both the oracle
# and the CUDA library receive them explicitly.
DEFAULT_PARAMS = dict(
    # PO-CCD (Alg. 3)
    cd_max_iters=32,          # max_iters
    cd_eps_pos2=0.01 ** 2,    # epsilon: coarse break on |e_p|^2 (m^2)
    cd_eps_ori2=0.1 ** 2,     # nu: coarse break on |omega|^2 (rad^2)
    cd_gamma_pos=1e-4,        # gamma along position (m)
    cd_gamma_ori=1e-3,        # gamma along orientation (rad)
    cd_sigma=0.05,            # Sigma = sigma^2 I of the rejection perturbation (rad)
    cd_delta0=0.5,            # delta(k) = delta0 * rho^k  (Eq. ori_update)
    cd_rho=0.97,
    proj_eps=1e-4,            # projected-vector length (relative) below which Eq. theta_proj gives 0
    cd_tie=1e-4,              # greedy choice: a later joint wins only if its score is lower by this fraction
    cd_variant=0,             # 0: PO-CCD (Alg. 3); 1: position-only CCD (Alg. 1), a baseline; 2: PO-CCD, target-wide break
    # Top-K and duplication (Alg. 2)
    dup_ratio=4,              # K = max(1, floor(B / dup_ratio))
    dup_sigma=0.02,           # Sigma of the duplication perturbation (rad)
    # PJ-IK (Alg. 4)
    lm_max_iters=20,
    lm_lambda=1e-3,           # lambda of Eq. normal-eqs
    lm_trust_R=0.3,           # R (rad)
    lm_beta=2.0,              # line-search ratio beta
    lm_A=4,                   # line-search depth A
    lm_sigma=0.01,            # Sigma of the PJ-IK perturbation (rad)
    lm_gn_reg=1e-6,           # regulariser of the minimum-norm Gauss-Newton step (dogleg)
)

PARAM_ORDER = tuple(DEFAULT_PARAMS.keys())
INT_PARAMS = {"cd_max_iters", "dup_ratio", "lm_max_iters", "lm_A", "cd_variant"}

# Philox phases (third counter word, high byte) -- part of the stream layout
# both sides implement: ctr = (candidate, target, phase << 24 | iteration, block).
PHASE_SEED, PHASE_CD, PHASE_DUP, PHASE_LM = 1, 2, 3, 4


def seed_key(seed: int) -> tuple[int, int]:
    """Split a 64-bit request seed into the two Philox key words (lo, hi)."""
    seed &= (1 << 64) - 1
    return seed & 0xFFFFFFFF, seed >> 32


@dataclass
class Robot:
    """Serial revolute chain in modified DH form plus its collision model.

    Joint i (0-based) contributes Rx(alpha[i]) Tx(a[i]) Rz(theta_i + theta_off[i]) Tz(d[i]).
    Bodies: 0 = base, 1..n = the body moved by joint i, n+1 = flange frame.
    """
    n: int
    a: np.ndarray
    alpha: np.ndarray
    d: np.ndarray
    theta_off: np.ndarray
    flange: np.ndarray          # 4x4 row-major, fixed transform after joint n
    lo: np.ndarray
    hi: np.ndarray
    sph_body: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    sph_xyzr: np.ndarray = field(default_factory=lambda: np.zeros((0, 4), np.float64))
    ignore: np.ndarray | None = None   # (n+2)x(n+2) uint8, 1 = pair never checked

    @property
    def n_bodies(self) -> int:
        return self.n + 2


@dataclass
class Scene:
    sph_xyzr: np.ndarray        # (Os, 4)
    box_lohi: np.ndarray        # (Oc, 6): lo xyz, hi xyz


def _trans_z(z: float) -> np.ndarray:
    t = np.eye(4)
    t[2, 3] = z
    return t


def panda() -> Robot:
    """The 7-DoF Franka Panda chain (modified DH), flange 0.107 m along z7."""
    hp = math.pi / 2
    lo = np.full(7, -2.8)
    hi = np.full(7, 2.8)
    lo[3], hi[3] = -3.0, -0.07
    return Robot(
        n=7,
        a=np.array([0, 0, 0, 0.0825, -0.0825, 0, 0.088]),
        alpha=np.array([0, -hp, hp, hp, -hp, hp, hp]),
        d=np.array([0.333, 0, 0.316, 0, 0.384, 0, 0]),
        theta_off=np.zeros(7),
        flange=_trans_z(0.107),
        lo=lo, hi=hi,
    )


def panda_chain(copies: int) -> Robot:
    """6 x copies joints: the Panda's first six DH rows and limits repeated
    (the DoF-scaling variants of 12, 18 and 24 joints), flange 0.107 m along
    the last axis.  Repeating the rows literally puts each copy's first joint
    on the axis of the previous copy's sixth joint (a = 0, alpha = 0)."""
    p = panda()
    rep = lambda v: np.tile(np.asarray(v[:6], float), copies)
    return Robot(n=6 * copies, a=rep(p.a), alpha=rep(p.alpha), d=rep(p.d), theta_off=np.zeros(6 * copies),
                 flange=_trans_z(0.107), lo=rep(p.lo), hi=rep(p.hi))


DOF_SCALING = (7, 12, 18, 24)  # the Panda and its chained variants


def dof_scaling_robot(dof: int) -> Robot:
    return panda() if dof == 7 else panda_chain(dof // 6)


def planar(lengths) -> Robot:
    """Planar nR chain: all axes parallel to z, link i of length lengths[i]."""
    n = len(lengths)
    a = np.concatenate([[0.0], np.asarray(lengths[:-1], float)])
    fl = np.eye(4)
    fl[0, 3] = lengths[-1]
    return Robot(n=n, a=a, alpha=np.zeros(n), d=np.zeros(n), theta_off=np.zeros(n),
                 flange=fl, lo=np.full(n, -math.pi), hi=np.full(n, math.pi))


def random_chain(rng: np.random.Generator, dof: int) -> Robot:
    """Random serial revolute chain: a, d ~ U[0, 0.4] m, alpha in {0, +-pi/2},
    symmetric limits +-U[1.5, 3.1] rad, flange 0.05 m along the last axis."""
    hp = math.pi / 2
    lim = rng.uniform(1.5, 3.1, dof)
    return Robot(
        n=dof,
        a=rng.uniform(0, 0.4, dof),
        alpha=rng.choice(np.array([0.0, hp, -hp]), dof),
        d=rng.uniform(0, 0.4, dof),
        theta_off=np.zeros(dof),
        flange=_trans_z(0.05),
        lo=-lim, hi=lim,
    )


def _segment_end(robot: Robot, body: int) -> np.ndarray:
    """End point, in body `body`'s frame, of the segment its spheres lie on.

    For body i < n it is the origin of joint i+1's frame, which the DH table
    gives directly: (a, -d sin(alpha), d cos(alpha)) of joint i+1.  Body n ends
    at the flange origin; the flange body extends 0.1 m along its z axis.
    """
    n = robot.n
    if 1 <= body < n:
        j = body  # 0-based index of joint body+1
        return np.array([robot.a[j], -robot.d[j] * math.sin(robot.alpha[j]),
                         robot.d[j] * math.cos(robot.alpha[j])])
    if body == n:
        return robot.flange[:3, 3].copy()
    if body == n + 1:
        return np.array([0.0, 0.0, 0.1])
    raise ValueError(body)


def add_link_spheres(rng: np.random.Generator, robot: Robot, counts, r_lo: float, r_hi: float) -> Robot:
    """Place counts[b-1] spheres on body b (b = 1..n+1), evenly spaced on the
    body's segment (end points included), radii ~ U[r_lo, r_hi]."""
    bodies, xyzr = [], []
    for b in range(1, robot.n + 2):
        m = int(counts[b - 1])
        end = _segment_end(robot, b)
        for i in range(m):
            f = i / (m - 1) if m > 1 else 0.5
            bodies.append(b)
            xyzr.append([*(f * end), rng.uniform(r_lo, r_hi)])
    robot.sph_body = np.asarray(bodies, np.int32)
    robot.sph_xyzr = np.asarray(xyzr, np.float64).reshape(-1, 4)
    robot.ignore = default_ignore(robot)
    return robot


def default_ignore(robot: Robot, slack: float = 0.1) -> np.ndarray:
    """Self-collision pairs that are never checked.

    Adjacent bodies (|i - j| <= 1) always touch at their shared joint.  Bodies
    further apart are also ignored when the chain between them is shorter
    than the sum of their largest sphere radii plus `slack`: such pairs sit at
    a distance fixed (or nearly fixed) by the chain and overlap in every
    configuration, like the links of a spherical wrist.  The base (body 0)
    carries no spheres.
    """
    nb = robot.n_bodies
    ign = np.zeros((nb, nb), np.uint8)
    rmax = np.zeros(nb)
    for b, r in zip(robot.sph_body, robot.sph_xyzr[:, 3]):
        rmax[b] = max(rmax[b], r)
    seg = np.zeros(nb)
    for b in range(1, nb):
        seg[b] = float(np.sqrt(np.sum(_segment_end(robot, b) ** 2)))
    for i in range(nb):
        for j in range(nb):
            lo, hi = min(i, j), max(i, j)
            if hi - lo <= 1 or lo == 0:
                ign[i, j] = 1
            elif seg[lo + 1:hi].sum() < rmax[lo] + rmax[hi] + slack:
                ign[i, j] = 1
    return ign


def panda_with_spheres(rng: np.random.Generator) -> Robot:
    """Panda with 60 link spheres (r 0.04-0.08 m) on bodies 1..7 and the flange body."""
    return add_link_spheres(rng, panda(), [8, 8, 8, 8, 7, 7, 7, 7], 0.04, 0.08)


def random_scene(rng: np.random.Generator, n_sph: int, n_box: int,
                 r_range=(0.02, 0.15), half_range=(0.025, 0.10),
                 lo=(-0.75, -0.75, 0.0), hi=(0.75, 0.75, 1.5),
                 keepout_r=0.25, keepout_z=0.45) -> Scene:
    """Obstacle spheres and boxes with centres uniform in [lo, hi]; draws that
    reach into the vertical keep-out cylinder (radius keepout_r, below
    keepout_z) around the base axis are redrawn."""
    lo, hi = np.asarray(lo), np.asarray(hi)
    sph = []
    while len(sph) < n_sph:
        c = rng.uniform(lo, hi)
        r = rng.uniform(*r_range)
        if math.hypot(c[0], c[1]) < keepout_r + r and c[2] - r < keepout_z:
            continue
        sph.append([*c, r])
    box = []
    while len(box) < n_box:
        c = rng.uniform(lo, hi)
        h = rng.uniform(*half_range, 3)
        blo, bhi = c - h, c + h
        inside_xy = (blo[0] < keepout_r and bhi[0] > -keepout_r and
                     blo[1] < keepout_r and bhi[1] > -keepout_r)
        if inside_xy and blo[2] < keepout_z:
            continue
        box.append([*blo, *bhi])
    return Scene(np.asarray(sph, np.float64).reshape(-1, 4), np.asarray(box, np.float64).reshape(-1, 6))


def joint_samples(rng: np.random.Generator, robot: Robot, count: int) -> np.ndarray:
    """Joint vectors uniform inside the limits, shape (count, n)."""
    return rng.uniform(robot.lo, robot.hi, size=(count, robot.n))


def log_uniform_counts(rng: np.random.Generator, count: int, lo: int, hi: int) -> np.ndarray:
    """Per-target seed counts round(exp(U[ln lo, ln hi]))."""
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), count))).astype(np.int64)


# ----------------------------------------------------------------------------
# Named workloads.  Each returns plain arrays; the pose of every joint sample
# is computed by the consumer.

@dataclass
class Workload:
    name: str
    robot: Robot
    scene: Scene | None
    theta_gen: np.ndarray       # candidate joint samples for targets (pool; filter with a scene)
    n_targets: int
    n_samples: int              # seeds per target (M = B)
    top_k: int
    seed: int                   # request seed of the method's own random draws
    eps_pos: float = 1e-3
    eps_ori: float = 1e-2


def cfg1() -> Workload:
    """Panda, 16 targets x 64 seeds, no obstacles."""
    rng = np.random.default_rng(CFG_SEED[1])
    rob = panda()
    return Workload("panda-16x64-open", rob, None, joint_samples(rng, rob, 16), 16, 64, 4,
                    CFG_SEED[1])


def cfg2(n_targets: int = 1000, n_samples: int = 1000, pool_factor: int = 16) -> Workload:
    """Panda + 60 link spheres, scene of 200 spheres and 20 boxes,
    1000 targets x 1000 seeds (sizes overridable for reduced cases)."""
    rng = np.random.default_rng(CFG_SEED[2])
    rob = panda_with_spheres(rng)
    scene = random_scene(rng, 200, 20)
    pool = joint_samples(rng, rob, n_targets * pool_factor)
    return Workload(f"panda-{n_targets}x{n_samples}-scene200s20b", rob, scene, pool,
                    n_targets, n_samples, 1, CFG_SEED[2])


CFG3_DOFS = (6, 7, 9, 12, 16, 20, 7, 12)


def cfg3_chains() -> list[Robot]:
    """The eight random chains of the uneven workload, with 6-12 spheres per
    link (r 0.02-0.05 m)."""
    rng = np.random.default_rng(CFG_SEED[3])
    out = []
    for dof in CFG3_DOFS:
        rob = random_chain(rng, dof)
        counts = rng.integers(6, 13, dof + 1)
        out.append(add_link_spheres(rng, rob, counts, 0.02, 0.05))
    return out


@dataclass
class MultiWorkload:
    """Uneven batch: several robots, each with a pool of joint samples from
    which collision-free targets are drawn, per-target seed counts, one scene."""
    name: str
    robots: list
    scene: Scene
    pools: list                 # per robot: joint samples (filter with the scene)
    n_targets: int              # per robot
    samples: list               # per robot: seed count per target
    seed: int
    eps_pos: float = 1e-3
    eps_ori: float = 1e-2


def cfg3(n_targets: int = 500, pool_factor: int = 40, lo: int = 32, hi: int = 4096) -> MultiWorkload:
    """The eight random chains (6-20 DoF, 6-12 link spheres per body), 500
    targets each, seed counts log-uniform in [32, 4096] per target, a scene of
    100 obstacle spheres (cfg2's distributions)."""
    rng = np.random.default_rng(CFG_SEED[3] + 100)
    chains = cfg3_chains()
    scene = random_scene(rng, 100, 0)
    pools = [joint_samples(rng, r, n_targets * pool_factor) for r in chains]
    samples = [log_uniform_counts(rng, n_targets, lo, hi) for _ in chains]
    return MultiWorkload(f"8 chains x {n_targets} targets, seeds log-uniform [{lo}, {hi}], 100 obstacle spheres",
                         chains, scene, pools, n_targets, samples, CFG_SEED[3])


CFG4_ROBOTS = (1, 3, 4, 5)  # rows of cfg3_chains(): 7, 12, 16 and 20 DoF


@dataclass
class ServingTemplate:
    """One request shape of the serving trace: a robot (row of CFG4_ROBOTS),
    its own scene and a pool of joint samples to draw collision-free targets from."""
    robot: int
    scene: Scene
    pool: np.ndarray


def cfg4_templates(count: int = 64, pool: int = 256) -> list:
    """Request templates: robot uniform over the four resident chains, scene
    of U{0..500} obstacle spheres (cfg2's distributions), joint-sample pool."""
    rng = np.random.default_rng(CFG_SEED[4])
    chains = cfg3_chains()
    out = []
    for _ in range(count):
        r = int(rng.integers(0, len(CFG4_ROBOTS)))
        sc = random_scene(rng, int(rng.integers(0, 501)), 0)
        out.append(ServingTemplate(r, sc, joint_samples(rng, chains[CFG4_ROBOTS[r]], pool)))
    return out


@dataclass
class ServingTrace:
    """Poisson arrivals: time (s), template, target count (1-8), seeds per
    target (log-uniform [32, 4096], one count per request), request seed."""
    t: np.ndarray
    template: np.ndarray
    n_targets: np.ndarray
    seeds: np.ndarray
    seed: np.ndarray


def cfg4_trace(rate: float = 2000.0, duration: float = 60.0, n_templates: int = 64, salt: int = 0) -> ServingTrace:
    rng = np.random.default_rng(CFG_SEED[4] + 1 + salt)
    n = int(rng.poisson(rate * duration))
    t = np.sort(rng.uniform(0.0, duration, n))
    return ServingTrace(t, rng.integers(0, n_templates, n), rng.integers(1, 9, n), log_uniform_counts(rng, n, 32, 4096),
                        rng.integers(0, 2 ** 63 - 1, n, dtype=np.int64))


@dataclass
class LargeWorkload:
    """The large case: target configurations first, then candidate obstacle
    nodes in the order they are admitted (the consumer drops every node a
    target configuration's link spheres touch and keeps the first n_obstacles
    that remain)."""
    name: str
    robot: Robot
    target_pool: np.ndarray     # joint samples; the consumer keeps the self-collision-free ones
    nodes: np.ndarray           # (k, 4) candidate obstacle spheres, admission order
    n_targets: int
    n_samples: int
    n_obstacles: int
    top_k: int
    seed: int
    eps_pos: float = 1e-3
    eps_ori: float = 1e-2


def jittered_grid_nodes(rng: np.random.Generator, core_lo=(-0.75, -0.75, 0.0), core_hi=(0.75, 0.75, 1.5),
                        core_n=(20, 25, 10), outer_lo=(-2.0, -2.0, -0.5), outer_hi=(2.0, 2.0, 2.5),
                        jitter=0.25, r_range=(0.01, 0.03)) -> np.ndarray:
    """Obstacle spheres on a jittered 3-D grid: the core grid (core_n nodes over
    [core_lo, core_hi]) first, then the nodes of the same lattice extended over
    [outer_lo, outer_hi] in order of their distance from the core box, each
    node moved by up to +-jitter of a cell per axis, radii ~ U[r_range]."""
    core_lo, core_hi, outer_lo, outer_hi = (np.asarray(v, float) for v in (core_lo, core_hi, outer_lo, outer_hi))
    step = (core_hi - core_lo) / np.asarray(core_n, float)
    first = core_lo + 0.5 * step  # cell centres of the core grid
    lo_i = np.floor((outer_lo - first) / step).astype(int)
    hi_i = np.floor((outer_hi - first) / step).astype(int)
    axes = [np.arange(lo_i[k], hi_i[k] + 1) for k in range(3)]
    I = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
    centre = first + I * step
    # distance of each node from the core box (0 inside), ties in lattice order
    out = np.maximum(np.maximum(core_lo - centre, centre - core_hi), 0.0)
    order = np.lexsort((I[:, 2], I[:, 1], I[:, 0], np.linalg.norm(out, axis=1)))
    centre = centre[order]
    centre = centre + rng.uniform(-jitter, jitter, centre.shape) * step
    r = rng.uniform(r_range[0], r_range[1], len(centre))
    return np.concatenate([centre, r[:, None]], axis=1)


def cfg5(n_targets: int = 10000, n_samples: int = 4096, n_obstacles: int = 5000, top_k: int = 16,
         pool_factor: int = 2) -> LargeWorkload:
    """cfg2's Panda with 60 link spheres; 10 000 targets x 4096 seeds; a scene
    of 5000 obstacle spheres on a jittered grid carved around the target
    configurations; top-16 solutions per target."""
    rob = panda_with_spheres(np.random.default_rng(CFG_SEED[2]))  # the same robot as cfg2
    rng = np.random.default_rng(CFG_SEED[5])
    pool = joint_samples(rng, rob, n_targets * pool_factor)
    nodes = jittered_grid_nodes(rng)
    return LargeWorkload(f"panda-{n_targets}x{n_samples}-grid{n_obstacles}", rob, pool, nodes, n_targets,
                         n_samples, n_obstacles, top_k, CFG_SEED[5])
