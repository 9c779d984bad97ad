"""Seeded synthetic scenes for the granular contact step.

This module only *generates inputs*: particle positions, radii, velocities and
masses, rigid-body descriptions and per-step tool twists.  It holds none of the
method's arithmetic (no binning, contact, solver or integration code), so both
the CUDA path and the FP64 oracle can consume its arrays without sharing code.

Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) turned into 53-bit uniform
doubles, then stored as float32.  Scene shapes follow the paper's workloads: a
particle column collapsing onto a plane (the column benchmark of Sec. II-D), a
particle bed dug by a kinematic scoop whose geometry is a signed distance
function (the Excavation task of Sec. III-C), and many independent copies of the
latter run side by side (the paper's "multiple independent simulations",
Sec. III-A).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Body kinds (same numbering as the C header's gg_body_kind).
PLANE = 0          # half-space below the body's local z = 0 plane
BOX = 1            # solid box, shape[0:3] = half extents
BOX_MINUS_BOX = 2  # box A (shape[0:3]) minus box B (half extents shape[3:6], centre shape[6:9])
OPEN_BOX = 3       # container: inside of a box with no lid, shape[0:3] = half extents
GRID = 4           # SDF sampled on a regular grid (trilinear), samples in Body.grid
TUBE = 5           # inside of a vertical cylinder (no caps), shape[0] = radius

DENSITY = 2500.0   # kg/m^3, used when a scene gives no density


def splitmix64(seed: int, count: int) -> np.ndarray:
    """`count` successive splitmix64 outputs for a generator started at `seed`."""
    with np.errstate(over="ignore"):
        k = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int) -> np.ndarray:
    """53-bit uniform doubles in [0, 1)."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Grid:
    """Samples of a signed distance function on a regular grid (body frame):
    values[k, j, i] = f(origin + h (i, j, k)), float32, x fastest."""
    values: np.ndarray
    origin: tuple
    spacing: float

    def __post_init__(self):
        self.values = np.ascontiguousarray(self.values, np.float32)
        assert self.values.ndim == 3 and min(self.values.shape) >= 2


@dataclass
class Body:
    kind: int
    shape: tuple = (0.0,) * 12
    pos: tuple = (0.0, 0.0, 0.0)
    quat: tuple = (1.0, 0.0, 0.0, 0.0)   # (w, x, y, z)
    lin_vel: tuple = (0.0, 0.0, 0.0)
    ang_vel: tuple = (0.0, 0.0, 0.0)
    is_free: int = 0
    mass: float = 0.0
    inertia: tuple = (0.0, 0.0, 0.0)     # principal moments in the body frame
    grid: Grid = None                    # GRID bodies: the sampled SDF

    def shape12(self):
        if self.grid is not None:        # GRID: origin of the samples, spacing
            o = self.grid.origin
            return (float(o[0]), float(o[1]), float(o[2]), float(self.grid.spacing)) + (0.0,) * 8
        s = list(self.shape) + [0.0] * (12 - len(self.shape))
        return tuple(float(v) for v in s[:12])


HEIGHT_CAMERA = 0  # orthographic, looking down: per pixel the highest particle surface point
DEPTH_CAMERA = 1   # perspective pinhole: per pixel the distance to the first surface


@dataclass
class Camera:
    """A depth observation (the paper's sky and ego cameras, Sec. III-A)."""
    kind: int = DEPTH_CAMERA
    width: int = 36
    height: int = 36
    pos: tuple = (0.0, 0.0, 0.0)
    quat: tuple = (1.0, 0.0, 0.0, 0.0)      # camera -> world; camera x right, y down, z forward
    extent: tuple = (1.0, 1.0)              # height camera: rectangle size in x, y
    fov_y: float = 1.0                      # depth camera: vertical field of view (rad)
    near: float = 0.01
    far: float = 2.0
    empty: float = 0.0                      # height camera: value where no particle is
    body_mask: int = 0xFFFFFFFF             # depth camera: bodies the rays see
    march_steps: int = 64
    march_eps: float = 1e-4


@dataclass
class Params:
    dt: float = 1e-4
    gravity: tuple = (0.0, 0.0, -9.81)
    mu: float = 0.5
    alpha: float = 0.2
    pja_iters: int = 20
    cell_size: float = 0.0      # 0 -> 2.002 * r_max
    hash_size: int = 0          # 0 -> 2 n (per environment)
    max_contacts: int = 16      # particle-particle capacity per particle
    max_body_contacts: int = 4  # particle-body capacity per particle
    cyclic_z: tuple = (0.0, 0.0)  # cyclic vertical boundary (bottom, top); off when equal
    pja_weight: int = 0         # 0 mass splitting; 1 Alg. 1 as printed (w = m_i), an ablation


@dataclass
class Scene:
    name: str
    pos_r: np.ndarray                 # float32 (n, 4): x, y, z, radius
    vel: np.ndarray                   # float32 (n, 3)
    mass: np.ndarray                  # float32 (n,)
    bodies: list                      # list[Body] (all environments, concatenated)
    params: Params
    n_steps: int
    twist: dict = field(default_factory=dict)   # global body index -> float32 (n_steps, 6)
    env_offsets: np.ndarray | None = None       # uint32 (E+1,) particle offsets, batched scenes
    body_offsets: np.ndarray | None = None      # uint32 (E+1,) body offsets, batched scenes
    info: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos_r.shape[0])


def sphere_mass(r: np.ndarray, density: float = DENSITY) -> np.ndarray:
    r = r.astype(np.float64)
    return (density * (4.0 / 3.0) * math.pi * r ** 3).astype(np.float32)


def jittered_lattice(dims, n, r0, jitter, seed, origin=(0.0, 0.0, 0.0), pitch=None):
    """First `n` sites of a dims=(nx, ny, nz) lattice, z-major (layers fill bottom up).

    Radius r_i = r0 * (1 + U(-jitter, jitter)); pitch defaults to 2 r_max * 1.02;
    each site is offset per axis by U(-(pitch/2 - r_i), +(pitch/2 - r_i)), so no
    two spheres overlap initially and every sphere stays inside its site.
    Returns float32 (n, 4) = (x, y, z, r) with the lattice's lower corner at origin.
    """
    nx, ny, nz = dims
    assert nx * ny * nz >= n
    r_max = r0 * (1.0 + jitter)
    if pitch is None:
        pitch = 2.0 * r_max * 1.02
    u = uniform(seed, 4 * n).reshape(n, 4)
    r = r0 * (1.0 + jitter * (2.0 * u[:, 0] - 1.0))
    idx = np.arange(n)
    ix = idx % nx
    iy = (idx // nx) % ny
    iz = idx // (nx * ny)
    site = np.stack([ix, iy, iz], axis=1).astype(np.float64) + 0.5
    slack = (0.5 * pitch - r)[:, None]
    off = slack * (2.0 * u[:, 1:4] - 1.0)
    p = np.asarray(origin, np.float64)[None, :] + site * pitch + off
    out = np.empty((n, 4), np.float32)
    out[:, :3] = p
    out[:, 3] = r
    return out, pitch


def _quat_from_rotvec(rv):
    rv = np.asarray(rv, np.float64)
    th = float(np.linalg.norm(rv))
    if th == 0.0:
        return (1.0, 0.0, 0.0, 0.0)
    a = rv / th
    s = math.sin(0.5 * th)
    return (math.cos(0.5 * th), a[0] * s, a[1] * s, a[2] * s)


def scoop_body(scale: float = 1.0, pos=(0.0, 0.0, 0.0), rotvec=(0.0, 0.0, 0.0)) -> Body:
    """Excavation tool: box A (0.06, 0.05, 0.04) m minus box B (0.054, 0.044, 0.04) m
    raised 0.01 m, i.e. 6 mm walls and floor with an open top, scaled by `scale`."""
    a = (0.06 * scale, 0.05 * scale, 0.04 * scale)
    b = (0.054 * scale, 0.044 * scale, 0.04 * scale)
    c = (0.0, 0.0, 0.01 * scale)
    return Body(kind=BOX_MINUS_BOX, shape=a + b + c, pos=tuple(float(v) for v in pos),
                quat=_quat_from_rotvec(rotvec))


def waypoint_twists(seed, n_steps, dt, start, dig_depth, span, n_way=6, pos_jit=0.05, rot_range=0.3,
                    seg_time=0.2):
    """Per-step world-frame twists (vx, vy, vz, wx, wy, wz) of a tool following
    `n_way` seeded waypoints along a dig path, piecewise constant per segment of
    `seg_time` seconds (the path takes (n_way - 1) seg_time s; runs shorter than
    that cover only its beginning).

    Waypoint k sits at start + (span * k/(n_way-1), 0, -dig_depth * sin(pi k/(n_way-1)))
    plus U(-pos_jit, pos_jit) per axis (k > 0), with a rotation vector drawn from
    U(-rot_range, rot_range) per axis.  The tool moves on each segment with the
    constant linear velocity that joins the two waypoint positions and the
    constant angular velocity (rotvec_{k+1} - rotvec_k) / seg_time.
    Returns (twist float32 (n_steps, 6), rotvec of waypoint 0, position of waypoint 0).
    """
    u = uniform(seed, 6 * n_way).reshape(n_way, 6)
    k = np.arange(n_way, dtype=np.float64) / (n_way - 1)
    pts = np.stack([start[0] + span * k,
                    np.full(n_way, start[1]),
                    start[2] - dig_depth * np.sin(math.pi * k)], axis=1)
    pts[1:] += pos_jit * (2.0 * u[1:, 0:3] - 1.0)
    rv = rot_range * (2.0 * u[:, 3:6] - 1.0)
    seg = max(1, int(round(seg_time / dt)))
    tw = np.zeros((n_steps, 6), np.float64)
    for s in range(n_steps):
        kseg = min(s // seg, n_way - 2)
        tw[s, 0:3] = (pts[kseg + 1] - pts[kseg]) / seg_time
        tw[s, 3:6] = (rv[kseg + 1] - rv[kseg]) / seg_time
    return tw.astype(np.float32), rv[0], pts[0]


# --------------------------------------------------------------------------- #
# Workloads shaped like the paper's tasks
# --------------------------------------------------------------------------- #

def settle_box(n=4096, seed=1000, n_steps=200):
    """4,096 spheres, r = 5 mm +-10 %, on a jittered 17x17x15 lattice inside an open
    0.2 m box (floor + 4 walls); dt = 1e-4 s, 20 PJA iterations, mu = 0.5."""
    r0, jit = 5e-3, 0.10
    pitch = 2.0 * r0 * (1 + jit) * 1.02
    dims = (17, 17, 15)
    ox = 0.5 * (0.2 - dims[0] * pitch)
    pr, _ = jittered_lattice(dims, n, r0, jit, seed, origin=(ox, ox, 0.0), pitch=pitch)
    box = Body(kind=OPEN_BOX, shape=(0.1, 0.1, 0.0), pos=(0.1, 0.1, 0.0))
    return Scene("settle_box_4096", pr, np.zeros((n, 3), np.float32), sphere_mass(pr[:, 3]), [box],
                 Params(dt=1e-4, mu=0.5, pja_iters=20), n_steps)


def column_collapse(n=262144, seed=1001, n_steps=2000, dims=None):
    """Granular column: n spheres, r = 2 mm +-10 %, on a jittered lattice 40x40 sites
    wide (1:1:4 aspect, 4.49 mm pitch) released onto a ground plane; mu = 0.6,
    dt = 5e-5 s, 20 PJA iterations."""
    r0, jit = 2e-3, 0.10
    if dims is None:
        side = 40 if n >= 40 * 40 * 4 else max(2, int(round((n / 4.0) ** (1.0 / 3.0))))
        dims = (side, side, -(-n // (side * side)))
    pitch = 2.0 * r0 * (1 + jit) * 1.02
    half = 0.5 * dims[0] * pitch
    pr, _ = jittered_lattice(dims, n, r0, jit, seed, origin=(-half, -half, 0.0), pitch=pitch)
    ground = Body(kind=PLANE, pos=(0.0, 0.0, 0.0))
    return Scene(f"column_collapse_{n}", pr, np.zeros((n, 3), np.float32), sphere_mass(pr[:, 3]),
                 [ground], Params(dt=5e-5, mu=0.6, pja_iters=20), n_steps,
                 info={"dims": dims, "pitch": pitch})


def pile_column(member=-1, n=32768, dims=(24, 24, 57), mu=0.2, n_steps=20000):
    """A column collapse that spreads into a low pile and comes to rest within
    n_steps (mu = 0.2; at mu = 0.6 a column this size stands jammed for thousands of
    steps).  Member k >= 0 of the ensemble moves the x of every particle with
    index % 8 == k by one float32 ulp towards +inf; member -1 is the unperturbed
    column.  The perturbations sample the chaotic spread of the collapse."""
    sc = column_collapse(n=n, seed=1001, n_steps=n_steps, dims=dims)
    sc.params.mu = mu
    if member >= 0:
        sel = np.arange(sc.n) % 8 == member
        sc.pos_r[sel, 0] = np.nextafter(sc.pos_r[sel, 0], np.float32(np.inf))
    sc.name = f"pile_column_{n}_m{member}"
    return sc


def pour_pile(member=-1, n=32768, mu=0.6, n_steps=20000, spread=2.0, side=24, seed=1005):
    """A pile poured onto a ground plane: n spheres (r = 2 mm +-10 %) scattered loosely
    (a jittered lattice of pitch `spread` x 2.04 r_max, sites inside the inscribed
    circle of a side x side footprint, z-major) fall, land over some 0.2 s and heap up
    at the friction of the column workload (mu = 0.6); dt = 5e-5 s, 20 PJA iterations.
    A column released at mu = 0.6 stands jammed for thousands of steps and creeps for
    longer than the oracle can follow, while a loose rain of spheres forms a heap whose
    slope has settled by 15,000 steps (0.75 s; the flank then creeps at ~2 mm/s, the
    angle by about 0.1 degree per 5,000 steps).  Member k >= 0 moves the x of every
    sphere with index % 8 == k by one float32 ulp towards +inf (-1: unperturbed)."""
    r0, jit = 2e-3, 0.10
    pitch = 2.0 * r0 * (1 + jit) * 1.02 * spread
    nz = -(-2 * n // (side * side)) + 8
    pr, _ = jittered_lattice((side, side, nz), side * side * nz, r0, jit, seed,
                             origin=(-0.5 * side * pitch, -0.5 * side * pitch, 0.0), pitch=pitch)
    rad = np.hypot(pr[:, 0], pr[:, 1])
    pr = np.ascontiguousarray(pr[rad <= 0.5 * side * pitch - 0.5 * pitch][:n])
    assert pr.shape[0] == n
    if member >= 0:
        sel = np.arange(n) % 8 == member
        pr[sel, 0] = np.nextafter(pr[sel, 0], np.float32(np.inf))
    ground = Body(kind=PLANE, pos=(0.0, 0.0, 0.0))
    return Scene(f"pour_pile_{n}_m{member}", pr, np.zeros((n, 3), np.float32), sphere_mass(pr[:, 3]), [ground],
                 Params(dt=5e-5, mu=mu, pja_iters=20), n_steps, info={"spread": spread, "side": side})


def _bed_env(n, r0, jit, seed, side=None, layers=None, n_steps=500, dt=1e-4, scoop_scale=1.0,
             tool_seed=None, margin=0.005):
    """A bed of n spheres in an open container, plus a kinematic scoop on a seeded
    dig trajectory.  Returns (pos_r, bodies, twist_of_scoop, info)."""
    if layers is None and side is None:
        layers = 16
    if side is None:
        side = int(math.ceil(math.sqrt(n / layers)))
    if layers is None:
        layers = -(-n // (side * side))
    pitch = 2.0 * r0 * (1 + jit) * 1.02
    foot = side * pitch
    half = 0.5 * foot + margin
    pr, _ = jittered_lattice((side, side, layers), n, r0, jit, seed,
                             origin=(-0.5 * foot, -0.5 * foot, 0.0), pitch=pitch)
    height = layers * pitch
    container = Body(kind=OPEN_BOX, shape=(half, half, 0.0), pos=(0.0, 0.0, 0.0))
    # the scoop starts above one side of the bed and digs across it
    ts = seed * 7 + 3 if tool_seed is None else tool_seed
    span = 0.6 * foot
    start = (-0.3 * foot, 0.0, height + 0.02 * scoop_scale)
    tw, rv0, p0 = waypoint_twists(ts, n_steps, dt, start, dig_depth=0.5 * height,
                                  span=span, pos_jit=0.02 * scoop_scale, rot_range=0.2)
    scoop = scoop_body(scoop_scale, pos=p0, rotvec=rv0)
    return pr, [container, scoop], tw, {"side": side, "layers": layers, "pitch": pitch, "height": height}


def excavation(n=1048576, seed=1002, n_steps=1000, with_cubes=True):
    """Bed of n spheres (r = 2 mm +-15 %) 128x128 sites wide in a 0.61 m container,
    one kinematic box-minus-box scoop on 6 seeded waypoints, two free 3 cm cubes;
    dt = 1e-4 s, 30 PJA iterations, mu = 0.5.  Smaller n: a 16-layer bed, scoop
    scaled with the bed's footprint."""
    r0, jit = 2e-3, 0.15
    side = 128 if n >= 128 * 128 * 64 else int(math.ceil(math.sqrt(n / 16)))
    foot = side * 2 * r0 * (1 + jit) * 1.02
    pr, bodies, tw, info = _bed_env(n, r0, jit, seed, side=side, n_steps=n_steps, dt=1e-4,
                                    margin=0.5 * (0.61 - foot) if side == 128 else 0.005,
                                    scoop_scale=min(1.0, foot / 0.6))
    if with_cubes:
        s = 0.03
        m = DENSITY * s ** 3
        inertia = m * s * s / 6.0
        zc = info["height"] + 0.5 * s + 0.001
        foot = side * info["pitch"]
        for x in (0.1 * foot, 0.3 * foot):
            bodies.append(Body(kind=BOX, shape=(0.5 * s, 0.5 * s, 0.5 * s), pos=(x, 0.2 * foot, zc), is_free=1,
                               mass=m, inertia=(inertia,) * 3))
    return Scene(f"excavation_{n}", pr, np.zeros((n, 3), np.float32), sphere_mass(pr[:, 3]), bodies,
                 Params(dt=1e-4, mu=0.5, pja_iters=30, max_body_contacts=4), n_steps, twist={1: tw},
                 info=info)


def scoop_bed(n=32768, seed=1004, n_steps=200, dims=None):
    """Differentiable workload: n spheres (32x32x32 lattice, r = 2 mm +-10 %) in a
    container plus a scoop on a seeded trajectory; dt = 1e-4 s, 20 PJA iterations."""
    r0, jit = 2e-3, 0.10
    if dims is None:
        side = int(round(n ** (1.0 / 3.0)))
        dims = (side, side, -(-n // (side * side)))
    pr, bodies, tw, info = _bed_env(n, r0, jit, seed, side=dims[0], layers=dims[2], n_steps=n_steps,
                                    dt=1e-4, scoop_scale=0.5)
    return Scene(f"scoop_bed_{n}", pr, np.zeros((n, 3), np.float32), sphere_mass(pr[:, 3]), bodies,
                 Params(dt=1e-4, mu=0.5, pja_iters=20), n_steps, twist={1: tw}, info=info)


def diff_scene(n=32768, seed=1004, n_steps=200):
    """Differentiable workload: a bed of n spheres (r = 2 mm +-10 %, cubic lattice
    footprint) in a container with a scoop (box minus box) embedded in it: the
    scoop's cavity floor sits at a third of the bed's height, and lattice sites whose
    sphere would cut the scoop's walls or floor are left empty, so the cavity starts
    full of particles and nothing overlaps the tool.  The scoop follows a seeded
    6-waypoint path (slow: 0.2 s per segment); dt = 1e-4 s, 20 PJA iterations."""
    r0, jit = 2e-3, 0.10
    side = max(4, int(round(n ** (1.0 / 3.0))))
    pitch = 2.0 * r0 * (1 + jit) * 1.02
    foot = side * pitch
    layers_total = -(-n // (side * side)) + side      # spare sites for the ones inside the walls
    cand, _ = jittered_lattice((side, side, layers_total), side * side * layers_total, r0, jit, seed,
                               origin=(-0.5 * foot, -0.5 * foot, 0.0), pitch=pitch)
    scale = 0.5 * foot / 0.12
    scoop0 = scoop_body(scale)
    ha = np.array(scoop0.shape[0:3]); hb = np.array(scoop0.shape[3:6]); cb = np.array(scoop0.shape[6:9])
    height = (-(-n // (side * side))) * pitch
    zfloor = height / 3.0                       # world height of the cavity floor
    pz = zfloor - (cb[2] - hb[2])               # scoop origin so that its cavity floor is at zfloor
    x = cand[:, :3].astype(np.float64) - np.array([0.0, 0.0, pz])
    r = cand[:, 3:4].astype(np.float64)
    in_a = np.all(np.abs(x) < ha + r, axis=1)                 # touches the outer box ...
    in_b = np.all(np.abs(x - cb) < hb - r, axis=1)            # ... but not well inside the cavity
    keep = ~(in_a & ~in_b)
    pr = cand[keep][:n].copy()
    assert pr.shape[0] == n
    half = 0.5 * foot + 0.005
    container = Body(kind=OPEN_BOX, shape=(half, half, 0.0), pos=(0.0, 0.0, 0.0))
    tw, rv0, p0 = waypoint_twists(seed * 7 + 3, n_steps, 1e-4, (0.0, 0.0, pz), dig_depth=-0.3 * height,
                                  span=0.3 * foot, pos_jit=0.1 * foot, rot_range=0.15)
    scoop = scoop_body(scale, pos=p0, rotvec=(0.0, 0.0, 0.0))
    tw = tw.copy()
    return Scene(f"diff_scene_{n}", pr, np.zeros((n, 3), np.float32), sphere_mass(pr[:, 3]), [container, scoop],
                 Params(dt=1e-4, mu=0.5, pja_iters=20), n_steps, twist={1: tw},
                 info={"side": side, "pitch": pitch, "scoop_scale": scale, "eps": 0.5 * r0,
                       "cavity_floor_z": zfloor})


def batched_beds(n_envs=256, seed=1003, n_steps=500, n_min=8192, n_max=65536):
    """n_envs independent beds with n_e = round(exp(U(ln n_min, ln n_max))) spheres,
    radius r_e ~ U(2, 4) mm (+-10 %), 16 layers, each with its own container and a
    scoop (scaled by r_e / 2 mm) on its own seeded trajectory; dt = 1e-4 s,
    20 PJA iterations, mu = 0.5.  Environments are spaced 10 m apart in x so that
    they never touch; they stay independent in any case because each has its own
    hash-bucket range."""
    u = uniform(seed, 2 * n_envs).reshape(n_envs, 2)
    ne = np.rint(np.exp(math.log(n_min) + u[:, 0] * (math.log(n_max) - math.log(n_min)))).astype(np.int64)
    re = 2e-3 + 2e-3 * u[:, 1]
    pos, bodies, twist = [], [], {}
    offs, boffs = [0], [0]
    for e in range(n_envs):
        pr, bl, tw, _ = _bed_env(int(ne[e]), float(re[e]), 0.10, seed * 65536 + e, layers=16,
                                 n_steps=n_steps, dt=1e-4, scoop_scale=float(re[e]) / 2e-3)
        dx = 10.0 * e
        pr[:, 0] += np.float32(dx)
        for b in bl:
            b.pos = (b.pos[0] + dx, b.pos[1], b.pos[2])
        twist[len(bodies) + 1] = tw
        bodies.extend(bl)
        pos.append(pr)
        offs.append(offs[-1] + pr.shape[0])
        boffs.append(len(bodies))
    pr = np.concatenate(pos, 0)
    n = pr.shape[0]
    return Scene(f"batched_{n_envs}env_{n}", pr, np.zeros((n, 3), np.float32), sphere_mass(pr[:, 3]),
                 bodies, Params(dt=1e-4, mu=0.5, pja_iters=20), n_steps, twist=twist,
                 env_offsets=np.asarray(offs, np.uint32), body_offsets=np.asarray(boffs, np.uint32),
                 info={"n_e": ne.tolist(), "r_e": re.tolist()})


def random_cloud(n, seed, box=0.05, r0=2e-3, jitter=0.1, vel_scale=0.0, overlap=1.0):
    """n spheres uniformly scattered in [0, box]^3 (overlaps allowed), for contact
    tests.  `overlap` < 1 shrinks the box relative to the given size."""
    u = uniform(seed, 7 * n).reshape(n, 7)
    pr = np.empty((n, 4), np.float32)
    pr[:, :3] = (u[:, 0:3] * box * overlap).astype(np.float32)
    pr[:, 3] = (r0 * (1.0 + jitter * (2.0 * u[:, 3] - 1.0))).astype(np.float32)
    vel = (vel_scale * (2.0 * u[:, 4:7] - 1.0)).astype(np.float32)
    return pr, vel


# --------------------------------------------------------------------------- #
# sampled SDF bodies (Sec. II-C): geometry baked onto regular grids
# --------------------------------------------------------------------------- #

def bake_grid(f, lo, hi, h):
    """Grid of f (a numpy SDF over (..., 3) body-frame points) on the box [lo, hi]
    with spacing h (the box is grown to a whole number of cells)."""
    lo = np.asarray(lo, np.float64)
    n = np.ceil((np.asarray(hi, np.float64) - lo) / h).astype(int) + 1
    n = np.maximum(n, 2)
    vals = np.empty((n[2], n[1], n[0]), np.float32)
    xs = lo[0] + h * np.arange(n[0])
    ys = lo[1] + h * np.arange(n[1])
    for k in range(n[2]):
        yy, xx = np.meshgrid(ys, xs, indexing="ij")
        pts = np.stack([xx, yy, np.full_like(xx, lo[2] + h * k)], axis=-1)
        vals[k] = f(pts)
    return Grid(vals, tuple(float(v) for v in lo), float(h))


def box_minus_box_sdf(shape):
    """numpy SDF of the scoop geometry (box A minus box B), for baking."""
    ha, hb, cb = np.array(shape[0:3]), np.array(shape[3:6]), np.array(shape[6:9])

    def box(y, half):
        q = np.abs(y) - half
        return np.linalg.norm(np.maximum(q, 0.0), axis=-1) + np.minimum(q.max(axis=-1), 0.0)

    return lambda y: np.maximum(box(y, ha), -box(y - cb, hb))


def gear_outline(teeth, module, pressure_deg=20.0, n_flank=10, n_arc=3):
    """Closed outline (counter-clockwise, (N, 2)) of an involute spur gear: pitch
    radius module * teeth / 2, addendum module, dedendum 1.25 module, involute
    flanks from the base circle (radial below it), tooth half-thickness pi / (2 teeth)
    of arc at the pitch circle."""
    a = math.radians(pressure_deg)
    rp = 0.5 * module * teeth
    rb, ra, rf = rp * math.cos(a), rp + module, max(rp - 1.25 * module, 0.2 * rp)

    def inv(r):  # involute polar angle at radius r >= rb
        al = math.acos(min(1.0, rb / r))
        return math.tan(al) - al

    half = math.pi / (2 * teeth) + inv(rp)      # flank angle offset at the base circle
    pts = []
    for k in range(teeth):
        c = 2 * math.pi * k / teeth
        r_lo = max(rb, rf)
        rr = np.linspace(r_lo, ra, n_flank)
        # right flank (rising), tip arc, left flank (falling)
        right = [(r, c - half + inv(r)) for r in rr]
        left = [(r, c + half - inv(r)) for r in rr[::-1]]
        tip0, tip1 = right[-1][1], left[0][1]
        tip = [(ra, t) for t in np.linspace(tip0, tip1, n_arc + 2)[1:-1]]
        root_a = c + half - inv(r_lo)
        root_b = c + 2 * math.pi / teeth - half + inv(r_lo)
        root = [(rf, t) for t in np.linspace(root_a, root_b, n_arc + 2)]
        seq = ([(rf, right[0][1])] if rf < rb else []) + right + tip + left + ([(rf, root_a)] if rf < rb else []) + root[1:-1]
        pts.extend(seq)
    return np.array([(r * math.cos(t), r * math.sin(t)) for r, t in pts])


def polygon_sdf2(poly):
    """numpy signed distance to a closed polygon (negative inside), over (..., 2)."""
    a = poly
    b = np.roll(poly, -1, axis=0)
    e = b - a
    ee = (e * e).sum(1)

    def f(p):
        shp = p.shape[:-1]
        q = p.reshape(-1, 2)
        out = np.empty(q.shape[0])
        for s in range(0, q.shape[0], 8192):
            w = q[s:s + 8192, None, :] - a[None]
            t = np.clip((w * e[None]).sum(-1) / ee[None], 0.0, 1.0)
            d = w - t[..., None] * e[None]
            dist = np.sqrt((d * d).sum(-1).min(1))
            # winding (crossing) test for the sign
            y = q[s:s + 8192, 1][:, None]
            cond = (a[None, :, 1] <= y) != (b[None, :, 1] <= y)
            xint = a[None, :, 0] + (y - a[None, :, 1]) * (b[None, :, 0] - a[None, :, 0]) / np.where(
                b[None, :, 1] == a[None, :, 1], 1.0, b[None, :, 1] - a[None, :, 1])
            inside = (cond & (q[s:s + 8192, 0][:, None] < xint)).sum(1) % 2 == 1
            out[s:s + 8192] = np.where(inside, -dist, dist)
        return out.reshape(shp)

    return f


def helical_gear_sdf(teeth, module, width, helix_deg=20.0):
    """numpy SDF (approximate away from the surface) of an involute helical gear about
    the body z axis: the outline twisted by tan(helix) / r_pitch per unit height,
    intersected with the slab |z| <= width / 2."""
    outline = polygon_sdf2(gear_outline(teeth, module))
    twist = math.tan(math.radians(helix_deg)) / (0.5 * module * teeth)

    def f(y):
        ang = -twist * y[..., 2]
        c, s = np.cos(ang), np.sin(ang)
        p2 = np.stack([c * y[..., 0] - s * y[..., 1], s * y[..., 0] + c * y[..., 1]], axis=-1)
        return np.maximum(outline(p2), np.abs(y[..., 2]) - 0.5 * width)

    return f


def gear_body(teeth=12, module=0.004, width=0.02, h=None, margin=0.006, pos=(0.0, 0.0, 0.0),
              quat=(1.0, 0.0, 0.0, 0.0), ang_vel=(0.0, 0.0, 0.0)):
    """A GRID body: helical gear baked with spacing h (default module / 4) on its
    bounding box grown by `margin` (>= r_max of the spheres it meets)."""
    h = h or module / 4.0
    ra = 0.5 * module * teeth + module
    lo = (-ra - margin, -ra - margin, -0.5 * width - margin)
    hi = (ra + margin, ra + margin, 0.5 * width + margin)
    g = bake_grid(helical_gear_sdf(teeth, module, width), lo, hi, h)
    return Body(kind=GRID, pos=pos, quat=quat, ang_vel=ang_vel, grid=g)


def gear_bed(n=4096, seed=1005, n_gears=1, teeth=8, module=0.003, width=0.012, omega=4.0, r0=1.5e-3,
             n_steps=200, gear=None):
    """A bed of n spheres (r0 +-10 %) in an open box with n_gears helical gears (GRID
    bodies, vertical axes, one baked grid shared by all) embedded in it, spinning at
    +-omega rad/s; lattice sites whose sphere would touch a gear are left empty.
    dt = 1e-4 s, 20 PJA iterations, mu = 0.5."""
    jit = 0.10
    pitch = 2.0 * r0 * (1 + jit) * 1.02
    ra = 0.5 * module * teeth + module
    per_row = max(1, int(math.ceil(math.sqrt(n_gears))))
    side = max(int(math.ceil(math.sqrt(n / 12.0))), int(math.ceil(per_row * 2.6 * ra / pitch)))
    foot = side * pitch
    layers = -(-n // (side * side)) + 8
    cand, _ = jittered_lattice((side, side, layers), side * side * layers, r0, jit, seed,
                               origin=(-0.5 * foot, -0.5 * foot, 0.0), pitch=pitch)
    g = gear if gear is not None else gear_body(teeth, module, width, margin=max(0.004, 2.5 * r0))
    sdf = helical_gear_sdf(teeth, module, width)
    u = uniform(seed * 31 + 7, 2 * n_gears)
    bodies = [Body(kind=OPEN_BOX, shape=(0.5 * foot + 0.004, 0.5 * foot + 0.004, 0.0))]
    keep = np.ones(cand.shape[0], bool)
    cell = foot / per_row
    zc = 0.5 * width + 2.0 * pitch
    for k in range(n_gears):
        cx = -0.5 * foot + (k % per_row + 0.5) * cell
        cy = -0.5 * foot + (k // per_row + 0.5) * cell
        w = omega if u[2 * k] < 0.5 else -omega
        pos = (cx, cy, zc)
        y = cand[:, :3].astype(np.float64) - np.array(pos)
        near = np.linalg.norm(y[:, :2], axis=1) < ra + 2 * r0
        near &= np.abs(y[:, 2]) < 0.5 * width + 2 * r0
        if near.any():
            d = sdf(y[near])
            idx = np.nonzero(near)[0]
            keep[idx[d < cand[idx, 3] + 2e-4]] = False
        bodies.append(Body(kind=GRID, pos=pos, ang_vel=(0.0, 0.0, w), grid=g.grid))
    pr = cand[keep][:n].copy()
    assert pr.shape[0] == n
    return Scene(f"gear_bed_{n}_{n_gears}", pr, np.zeros((n, 3), np.float32), sphere_mass(pr[:, 3]), bodies,
                 Params(dt=1e-4, mu=0.5, pja_iters=20), n_steps, info={"foot": foot, "ra": ra})


def gear_tower(n=65536, n_gears=10, seed=1006, radius=0.06, r0=2e-3, teeth=10, module=0.003, width=0.012,
               omega=4.0, gap=0.04, n_steps=500, gear=None):
    """The paper's helical-gear benchmark (Sec. III): n spheres (r0 +-10 %) in a tall
    vertical tube of the given radius with a cyclic vertical boundary (spheres leaving
    through the bottom re-enter at the top), and n_gears involute helical gears (GRID
    bodies sharing one baked grid) on the axis every `gap` metres, each with a seeded
    random orientation, spinning about its own axis at U(-omega, omega) rad/s.  The
    spheres start on a jittered lattice inside the tube (sites touching a gear left
    empty).  dt = 1e-4 s, 20 PJA iterations, mu = 0.5."""
    jit = 0.10
    pitch = 2.0 * r0 * (1 + jit) * 1.02
    side = int(math.floor(2.0 * (radius - 1.2 * r0) / pitch))
    foot = side * pitch
    per_layer = None
    g = gear if gear is not None else gear_body(teeth, module, width, margin=max(0.004, 2.5 * r0))
    sdf = helical_gear_sdf(teeth, module, width)
    ra = 0.5 * module * teeth + module
    u = uniform(seed * 13 + 5, 4 * max(n_gears, 1))
    gears = []
    for k in range(n_gears):
        rv = (np.array(u[4 * k:4 * k + 3]) * 2.0 - 1.0) * math.pi / math.sqrt(3.0)
        q = _quat_from_rotvec(rv)
        w = (2.0 * u[4 * k + 3] - 1.0) * omega
        qa = np.array(q, np.float64)
        a, b, c, d = qa / np.linalg.norm(qa)
        axis = np.array([2 * (b * d + a * c), 2 * (c * d - a * b), 1 - 2 * (b * b + c * c)])  # R e_z
        z = gap * (k + 1)
        gears.append((np.array([0.0, 0.0, z]), q, w * axis))
    # enough lattice layers for n spheres after removing the sites in the tube's
    # corners and around the gears
    inside = None
    layers = 8
    while True:
        cand, _ = jittered_lattice((side, side, layers), side * side * layers, r0, jit, seed,
                                   origin=(-0.5 * foot, -0.5 * foot, 0.5 * pitch), pitch=pitch)
        x = cand[:, :3].astype(np.float64)
        keep = np.hypot(x[:, 0], x[:, 1]) < radius - cand[:, 3] - 0.2 * r0
        for pos, q, _ in gears:
            qa = np.array(q, np.float64)
            a, b, c, d = qa / np.linalg.norm(qa)
            R = np.array([[1 - 2 * (c * c + d * d), 2 * (b * c - a * d), 2 * (b * d + a * c)],
                          [2 * (b * c + a * d), 1 - 2 * (b * b + d * d), 2 * (c * d - a * b)],
                          [2 * (b * d - a * c), 2 * (c * d + a * b), 1 - 2 * (b * b + c * c)]])
            y = (x - pos) @ R
            near = np.linalg.norm(y, axis=1) < ra + width + 2 * r0
            if near.any():
                idx = np.nonzero(near)[0]
                keep[idx[sdf(y[near]) < cand[idx, 3] + 2e-4]] = False
        if keep.sum() >= n:
            break
        layers = int(layers * 1.3) + 4
    pr = cand[keep][:n].copy()
    top = max(float(pr[:, 2].max()) + 2 * r0, gap * (n_gears + 1))
    bodies = [Body(kind=TUBE, shape=(radius,))]
    for pos, q, w in gears:
        bodies.append(Body(kind=GRID, pos=tuple(pos), quat=q, ang_vel=tuple(float(v) for v in w), grid=g.grid))
    return Scene(f"gear_tower_{n}_{n_gears}", pr, np.zeros((n, 3), np.float32), sphere_mass(pr[:, 3]), bodies,
                 Params(dt=1e-4, mu=0.5, pja_iters=20, cyclic_z=(0.0, top)), n_steps,
                 info={"radius": radius, "height": top, "ra": ra})
