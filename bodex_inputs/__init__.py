"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds input synthesis only -- hand templates, object SDF samples,
initial poses, contact geometry for standalone QP cases and the desired
wrench sets.  It contains none of the grasp-synthesis arithmetic itself
(no forward kinematics, no SDF queries, no grasp matrix, no QP): both the
CUDA path and the CPU oracle receive these arrays and do that work on
their own.

The paper (Sec. V-A) synthesises grasps for DexGraspNet objects rescaled to
0.06-0.12 m with Shadow (22 DoF) and Allegro (16 DoF) hands.  Those assets
are not available, so the generators below produce stand-ins of the same
scale and degree-of-freedom counts:

* ``hand_template(name)`` -- kinematic trees with a 6-DoF floating base
  (Sec. IV-B) and revolute finger joints; one contact sphere centre per
  fingertip (Sec. IV-C, coarse stage).
* ``sphere_object`` / ``grid_object`` -- an analytic sphere, or a seeded
  union of spheres, boxes and capsules sampled at the nodes of a cubic grid.
* ``initial_poses`` -- palm placed 2-5 cm outside the object surface along
  a random direction, palm facing the object, random roll, mildly flexed
  fingers.

All arrays are float32 (the library's element type) unless noted.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "HandTemplate", "SphereObject", "GridObject", "hand_template",
    "sphere_object", "grid_object", "initial_poses", "wrench_set",
    "default_params", "random_contacts", "HAND_NAMES", "workload", "mixed_workload",
]

DEG = math.pi / 180.0


# --------------------------------------------------------------------------
# hand templates
# --------------------------------------------------------------------------
@dataclass
class HandTemplate:
    """A hand as a list of revolute joints under a 6-DoF floating base.

    Joint j's frame is ``T_parent(j) @ offset[j] @ Rot(axis[j], q_j)``; the
    parent of a joint is an earlier joint or -1 (the root frame that the six
    virtual base joints produce).  Contact i sits at ``contact_local[i]`` in
    the frame of joint ``contact_link[i]``.
    """
    name: str
    parent: np.ndarray          # [n] int32
    offset: np.ndarray          # [n, 12] float32, row-major 3x4 [R | t]
    axis: np.ndarray            # [n, 3] float32, unit axis in the joint frame
    qmin: np.ndarray            # [6 + n] float32 (virtual joints first)
    qmax: np.ndarray            # [6 + n] float32
    contact_link: np.ndarray    # [m] int32
    contact_local: np.ndarray   # [m, 3] float32
    contact_radius: float       # alpha, the fingertip sphere radius (m)
    tip_samples: np.ndarray = field(default=None)  # [m, S, 3] float32
    # collision spheres (cuRobo-style hand geometry): link (-1 = palm/root),
    # centre in that link's frame, radius
    sphere_link: np.ndarray = field(default=None)    # [K] int32
    sphere_local: np.ndarray = field(default=None)   # [K, 3] float32
    sphere_radius: np.ndarray = field(default=None)  # [K] float32

    @property
    def n_joints(self) -> int:
        return int(self.parent.shape[0])

    @property
    def n_contacts(self) -> int:
        return int(self.contact_link.shape[0])

    @property
    def dof(self) -> int:
        return 6 + self.n_joints


def _rz(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def _offset(R, t):
    return np.concatenate([np.asarray(R, float), np.asarray(t, float).reshape(3, 1)], axis=1).reshape(12)


def _fib_sphere(n, radius):
    """n points spread over a sphere (golden-angle spiral), deterministic."""
    pts = []
    ga = math.pi * (3.0 - math.sqrt(5.0))
    for k in range(n):
        z = 1.0 - 2.0 * (k + 0.5) / n
        r = math.sqrt(max(0.0, 1.0 - z * z))
        th = ga * k
        pts.append((radius * r * math.cos(th), radius * r * math.sin(th), radius * z))
    return np.array(pts)


class _Builder:
    def __init__(self):
        self.parent, self.offset, self.axis, self.lo, self.hi = [], [], [], [], []
        self.clink, self.clocal = [], []

    def joint(self, parent, R, t, axis, lo, hi):
        self.parent.append(parent)
        self.offset.append(_offset(R, t))
        self.axis.append(np.asarray(axis, float))
        self.lo.append(lo)
        self.hi.append(hi)
        return len(self.parent) - 1

    def finger(self, base_xy, yaw, joints, tip):
        """joints: list of (axis, length_before, lo, hi); the first joint sits at
        the finger base, later joints at the end of the previous link."""
        prev = -1
        for k, (ax, length, lo, hi) in enumerate(joints):
            if k == 0:
                R, t = _rz(yaw), (base_xy[0], base_xy[1], 0.0)
            else:
                R, t = np.eye(3), (0.0, length, 0.0)
            prev = self.joint(prev, R, t, ax, lo, hi)
        self.clink.append(prev)
        self.clocal.append((0.0, tip, 0.0))

    def spheres(self, radius, palm):
        """Collision spheres: along every finger link (the +y segment from the
        joint to the next joint, or to the fingertip contact, which keeps its
        own sphere out) at a spacing of 1.5 radii, plus the palm spheres
        ``palm`` = [(x, y, z, r)] on the root."""
        n = len(self.parent)
        link, local, rad = [], [], []
        for x, y, z, r in palm:
            link.append(-1)
            local.append((x, y, z))
            rad.append(r)
        step = 1.5 * radius
        for j in range(n):
            kids = [c for c in range(n) if self.parent[c] == j]
            if kids:
                L = float(np.asarray(self.offset[kids[0]]).reshape(3, 4)[1, 3])
            else:
                L = float(self.clocal[self.clink.index(j)][1])
            k = 0
            while k * step < L - 0.5 * step:
                link.append(j)
                local.append((0.0, k * step, 0.0))
                rad.append(radius)
                k += 1
        return (np.array(link, np.int32), np.array(local, np.float32).reshape(-1, 3),
                np.array(rad, np.float32))

    def build(self, name, radius, n_tip_samples=32, palm=()):
        n = len(self.parent)
        sl, sp, sr = self.spheres(radius, palm)
        vlo = [-0.3, -0.3, -0.3, -math.pi, -math.pi, -math.pi]
        vhi = [0.3, 0.3, 0.3, math.pi, math.pi, math.pi]
        clocal = np.array(self.clocal, float)
        samples = np.stack([c + _fib_sphere(n_tip_samples, radius) for c in clocal])
        return HandTemplate(
            name=name,
            parent=np.array(self.parent, np.int32),
            offset=np.array(self.offset, np.float32).reshape(n, 12),
            axis=np.array(self.axis, np.float32).reshape(n, 3),
            qmin=np.array(vlo + self.lo, np.float32),
            qmax=np.array(vhi + self.hi, np.float32),
            contact_link=np.array(self.clink, np.int32),
            contact_local=clocal.astype(np.float32),
            contact_radius=float(radius),
            tip_samples=samples.astype(np.float32),
            sphere_link=sl,
            sphere_local=sp,
            sphere_radius=sr,
        )


X, Y, Z = (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)


def _palm(nx, ny, dx, ys, r):
    """nx x ny palm spheres of radius r centred r/2 under the palm plane."""
    xs = [(k - (nx - 1) / 2) * dx for k in range(nx)]
    y0, y1 = ys
    yy = [y0 + (y1 - y0) * k / max(1, ny - 1) for k in range(ny)]
    return [(x, y, -0.5 * r, r) for y in yy for x in xs]
HAND_NAMES = ("hand4", "hand3", "hand4x4", "hand5")


def hand_template(name: str) -> HandTemplate:
    """Synthetic hands.  The palm lies in the root x-y plane with its normal
    along root +z; fingers point along +y (thumb along -y, yawed by pi) and
    positive flexion (about the joint's local x) curls them toward +z.

    * ``hand4``: 4 fingers x 3 flexion joints (12), links 4/3/2.5 cm,
      limits +-90 deg, 4 fingertip contacts, alpha = 0.8 cm.
    * ``hand3``: 3 fingers x 3 joints (9), 3 contacts.
    * ``hand4x4``: 4 fingers x (abduction + 3 flexion) = 16 joints, 4 contacts.
    * ``hand5``: Shadow-like, joints per finger 4/4/4/5/5 = 22, 5 contacts.
    """
    b = _Builder()
    flex = lambda L: (X, L, -90 * DEG, 90 * DEG)
    if name == "hand4":
        for xb in (-0.02, 0.0, 0.02):
            b.finger((xb, 0.03), 0.0, [flex(0.0), flex(0.04), flex(0.03)], 0.025)
        b.finger((0.0, -0.03), math.pi, [flex(0.0), flex(0.04), flex(0.03)], 0.025)
        return b.build(name, 0.008, palm=_palm(3, 2, 0.02, (-0.01, 0.015), 0.011))
    if name == "hand3":
        for xb in (-0.02, 0.02):
            b.finger((xb, 0.03), 0.0, [flex(0.0), flex(0.04), flex(0.03)], 0.025)
        b.finger((0.0, -0.03), math.pi, [flex(0.0), flex(0.04), flex(0.03)], 0.025)
        return b.build(name, 0.008, palm=_palm(2, 2, 0.02, (-0.01, 0.015), 0.011))
    if name == "hand4x4":
        abd = (Z, 0.0, -20 * DEG, 20 * DEG)
        for xb in (-0.02, 0.0, 0.02):
            b.finger((xb, 0.03), 0.0, [abd, flex(0.0), flex(0.04), flex(0.03)], 0.025)
        b.finger((0.0, -0.03), math.pi, [abd, flex(0.0), flex(0.04), flex(0.03)], 0.025)
        return b.build(name, 0.008, palm=_palm(3, 2, 0.02, (-0.01, 0.015), 0.011))
    if name == "hand5":
        abd = (Z, 0.0, -20 * DEG, 20 * DEG)
        fl = lambda L, lo=0.0: (X, L, lo * DEG, 90 * DEG)
        for xb in (-0.022, 0.0, 0.022):            # index, middle, ring
            b.finger((xb, 0.04), 0.0, [abd, fl(0.0, -15), fl(0.045), fl(0.025)], 0.022)
        # little finger: metacarpal arch about the finger axis, then abduction
        b.finger((0.044, 0.03), 0.0,
                 [(Y, 0.0, 0.0, 40 * DEG), (Z, 0.01, -20 * DEG, 20 * DEG),
                  fl(0.0, -15), fl(0.04), fl(0.022)], 0.02)
        # thumb: axial rotation, abduction, three flexions; opposes the fingers
        b.finger((-0.025, -0.015), math.pi,
                 [(Y, 0.0, -60 * DEG, 60 * DEG), (Z, 0.0, -30 * DEG, 30 * DEG),
                  fl(0.0, -15), fl(0.038), fl(0.032)], 0.027)
        return b.build(name, 0.009, palm=_palm(3, 2, 0.022, (-0.005, 0.02), 0.012))
    raise ValueError(f"unknown hand template {name!r}")


# --------------------------------------------------------------------------
# objects
# --------------------------------------------------------------------------
@dataclass
class SphereObject:
    center: np.ndarray   # [3] float32
    radius: float
    kind: str = "sphere"

    def sdf(self, pts):
        """Exact distance for pose initialisation only (float64)."""
        return np.linalg.norm(np.asarray(pts, float) - self.center, axis=-1) - self.radius


@dataclass
class GridObject:
    values: np.ndarray   # [N, N, N] float32, index [iz, iy, ix] (x fastest)
    origin: np.ndarray   # [3] float32, position of node (0, 0, 0)
    h: float             # node spacing (m)
    primitives: list     # the analytic union the grid was sampled from
    kind: str = "grid"

    @property
    def n(self) -> int:
        return int(self.values.shape[0])

    def sdf(self, pts):
        return _union_sdf(self.primitives, np.asarray(pts, float))


def sphere_object(radius=0.04, center=(0.0, 0.0, 0.0)) -> SphereObject:
    return SphereObject(np.asarray(center, np.float32), float(radius))


def _rand_rot(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def _union_sdf(prims, p):
    d = np.full(p.shape[:-1], np.inf)
    for pr in prims:
        q = p - pr["c"]
        if pr["type"] == "sphere":
            di = np.linalg.norm(q, axis=-1) - pr["r"]
        elif pr["type"] == "box":
            ql = np.abs(q @ pr["R"]) - pr["he"]
            di = (np.linalg.norm(np.maximum(ql, 0.0), axis=-1)
                  + np.minimum(ql.max(axis=-1), 0.0))
        else:  # capsule: segment c +- hl * a, radius r
            s = np.clip(q @ pr["a"], -pr["hl"], pr["hl"])
            di = np.linalg.norm(q - s[..., None] * pr["a"], axis=-1) - pr["r"]
        d = np.minimum(d, di)
    return d


def grid_object(seed: int, n: int = 64, h: float = 0.002, n_prims: int = 8) -> GridObject:
    """Seeded union of spheres (r ~ U[1, 2.5] cm), boxes (half extents
    U[0.5, 2] cm, random rotation) and capsules (r ~ U[0.5, 1.5] cm, half
    length U[1, 3] cm); centres U[-2.5, 2.5] cm per axis.  The distance
    field is sampled at the nodes of an n^3 grid with spacing h, centred on
    the origin."""
    rng = np.random.default_rng(seed)
    prims = []
    for _ in range(n_prims):
        kind = ("sphere", "box", "capsule")[int(rng.integers(3))]
        c = rng.uniform(-0.025, 0.025, size=3)
        if kind == "sphere":
            prims.append(dict(type=kind, c=c, r=rng.uniform(0.01, 0.025)))
        elif kind == "box":
            prims.append(dict(type=kind, c=c, R=_rand_rot(rng), he=rng.uniform(0.005, 0.02, size=3)))
        else:
            a = rng.normal(size=3)
            a /= np.linalg.norm(a)
            prims.append(dict(type=kind, c=c, a=a, r=rng.uniform(0.005, 0.015), hl=rng.uniform(0.01, 0.03)))
    origin = np.full(3, -(n - 1) * h / 2.0)
    ax = origin[0] + h * np.arange(n)
    zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
    pts = np.stack([xx, yy, zz], axis=-1)
    vals = _union_sdf(prims, pts).astype(np.float32)
    return GridObject(vals, origin.astype(np.float32), float(h), prims)


# --------------------------------------------------------------------------
# poses
# --------------------------------------------------------------------------
def _euler_xyz(R):
    """Angles (a, b, c) with R = Rx(a) Ry(b) Rz(c)."""
    b = math.asin(max(-1.0, min(1.0, R[0, 2])))
    a = math.atan2(-R[1, 2], R[2, 2])
    c = math.atan2(-R[0, 1], R[0, 0])
    return a, b, c


def _surface_distance(obj, U):
    """For each unit direction (rows of U), the largest s with sdf(s u) <= 0
    (the outermost surface crossing along u), marched from 0.2 m inward in
    0.5 mm steps and refined by bisection, all directions at once."""
    U = np.asarray(U, float).reshape(-1, 3)
    if isinstance(obj, SphereObject):
        return np.full(len(U), obj.radius)  # centred sphere
    step = 0.0005
    s = np.full(len(U), 0.2)
    moving = np.ones(len(U), bool)
    while moving.any():
        out = obj.sdf(s[:, None] * U) > 0
        moving = out & (s > 0)
        s = np.where(moving, s - step, s)
    lo, hi = s.copy(), s + step
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        outside = obj.sdf(mid[:, None] * U) > 0
        hi = np.where(outside, mid, hi)
        lo = np.where(outside, lo, mid)
    return 0.5 * (lo + hi)


def initial_poses(hand: HandTemplate, obj, batch: int, seed: int,
                  gap=(0.02, 0.05), flex=0.3) -> np.ndarray:
    """Poses x = [t(3), r(3), q(n)] (float32 [batch, 6 + n]).

    A direction u is drawn uniformly on the sphere; the palm centre (root
    origin) is put at (surface distance along u) + U[gap] along u, its normal
    (root +z) points along -u toward the object, with a random roll; joint
    angles are U[0, flex] times their upper limits."""
    rng = np.random.default_rng(seed)
    D = hand.dof
    out = np.zeros((batch, D), np.float64)
    U = np.zeros((batch, 3))
    gaps = np.zeros(batch)
    for b in range(batch):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        U[b] = u
        gaps[b] = rng.uniform(*gap)
        zax = -u
        a = np.cross(zax, (1.0, 0.0, 0.0) if abs(zax[0]) < 0.9 else (0.0, 1.0, 0.0))
        a /= np.linalg.norm(a)
        c2 = np.cross(zax, a)
        psi = rng.uniform(0.0, 2.0 * math.pi)
        xax = math.cos(psi) * a + math.sin(psi) * c2
        yax = np.cross(zax, xax)
        R = np.stack([xax, yax, zax], axis=1)
        out[b, 3:6] = _euler_xyz(R)
        out[b, 6:] = rng.uniform(0.0, flex, size=hand.n_joints) * hand.qmax[6:]
    dist = _surface_distance(obj, U) + gaps
    out[:, 0:3] = dist[:, None] * U
    return out.astype(np.float32)


# --------------------------------------------------------------------------
# wrenches, parameters, standalone-QP geometry
# --------------------------------------------------------------------------
def wrench_set(s: int) -> np.ndarray:
    """Desired unit wrenches t_j (Sec. IV-A): s = 6 gives +-force axes with
    zero torque; s = 12 adds the +-torque axes.  Order: +e0, -e0, +e1, ..."""
    if s not in (6, 12):
        raise ValueError("s must be 6 or 12")
    T = np.zeros((s, 6), np.float32)
    for k in range(s // 2):
        T[2 * k, k] = 1.0
        T[2 * k + 1, k] = -1.0
    return T


def default_params(**kw) -> dict:
    """Hyper-parameters.  mu = 0.5 (the workloads' friction); beta = 1 and
    gamma = 0.5 (the paper leaves them open); w_Q = 1, w_d = 1000; delta =
    0.01 m (the 1 cm pre-grasp margin, Sec. IV-D); Adam lr 2e-3 for
    translation and 2e-2 for angles."""
    p = dict(mu=0.5, beta=1.0, gamma=0.5, w_q=1.0, w_d=1000.0, delta=0.01,
             eps_reg=0.0, lr_t=2e-3, lr_r=2e-2, b1=0.9, b2=0.999, adam_eps=1e-8)
    p.update(kw)
    return p


def random_contacts(batch: int, m: int, seed: int, radius=0.04, spread=1.0,
                    normal_noise=0.15) -> tuple[np.ndarray, np.ndarray]:
    """Contact positions p [batch, m, 3] near a sphere of the given radius
    (directions biased to one hemisphere by ``spread`` < 1) and unit inward
    normals n (the radial direction perturbed by ``normal_noise``)."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(batch, m, 3))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    if spread < 1.0:
        d[..., 2] = np.abs(d[..., 2]) * spread + (1 - spread)
        d /= np.linalg.norm(d, axis=-1, keepdims=True)
    p = radius * d * rng.uniform(0.95, 1.05, size=(batch, m, 1))
    n = -d + normal_noise * rng.normal(size=(batch, m, 3))
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    # keep clear of the tangent-basis branch cut at n_z = 0
    bad = np.abs(n[..., 2]) < 1e-3
    n[..., 2][bad] = np.where(n[..., 2][bad] >= 0, 1e-3, -1e-3)
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    return p.astype(np.float32), n.astype(np.float32)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
def workload(name: str, batch: int | None = None):
    """The named synthetic workloads: returns (hand, object, x0, T, params,
    steps, admm_iters).

    * ``tiny``: 64 grasps, hand4, analytic sphere r = 4 cm, s = 6,
      50 upper steps x 30 ADMM iterations, seed 1.
    * ``paper``: 4096 grasps, hand5, 64^3 grid (2 mm) union of 8 primitives,
      s = 12, 200 upper steps x 50 ADMM iterations, seed 2.
    * ``grad``: 1024 grasps on the tiny hand/object, seed 3.
    """
    if name == "tiny":
        hand, obj, B, s, seed, steps, iters = hand_template("hand4"), sphere_object(), 64, 6, 1, 50, 30
    elif name == "paper":
        hand, obj, B, s, seed, steps, iters = hand_template("hand5"), grid_object(2), 4096, 12, 2, 200, 50
    elif name == "grad":
        hand, obj, B, s, seed, steps, iters = hand_template("hand4"), sphere_object(), 1024, 6, 3, 1, 30
    else:
        raise ValueError(name)
    if batch is not None:
        B = batch
    x0 = initial_poses(hand, obj, B, seed)
    return hand, obj, x0, wrench_set(s), default_params(), steps, iters


def mixed_workload(seed: int = 4, scale: float = 1.0):
    """The mixed-template batch: 3 hand templates (3-finger 9-joint with 3
    contacts, 4-finger 16-joint with 4, 5-finger 22-joint with 5) with
    uneven counts 512 / 2048 / 6144, each split over two objects, six grids
    of 48, 56, 64, 72, 80 and 96 nodes per axis (2 mm).  Returns a list of
    (hand, object, x0) and the wrench set (s = 12).  `scale` shrinks the
    counts for tests."""
    rng_seeds = [seed * 100 + k for k in range(6)]
    grids = [grid_object(sd, n=n) for sd, n in zip(rng_seeds, (48, 56, 64, 72, 80, 96))]
    jobs = []
    for k, (name, count) in enumerate((("hand3", 512), ("hand4x4", 2048), ("hand5", 6144))):
        hand = hand_template(name)
        for half in range(2):
            obj = grids[2 * k + half]
            B = max(1, int(count * scale) // 2)
            jobs.append((hand, obj, initial_poses(hand, obj, B, seed=seed * 1000 + 2 * k + half)))
    return jobs, wrench_set(12)
