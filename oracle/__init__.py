"""FP64 CPU oracle of the granular contact step (ctypes wrapper over gg_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import this package.  The product library
never calls it, and it shares no code with the CUDA path: the two meet only in
the seeded input arrays of paper_2306_01369_gb300.scenes.

Every value handed to the C oracle is first rounded to float32, because the
method's inputs (positions, radii, masses, body poses, twists, dt, mu, alpha,
gravity) are float32 on the device; the oracle then computes in FP64 from
exactly those values.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gg_oracle.c")
_HDR = os.path.join(_HERE, "gg_oracle.h")
_LIB = os.path.join(_HERE, "libgg_oracle.so")

CFLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile gg_oracle.c with gcc (FMA contraction off) unless up to date."""
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OrcParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("gravity", C.c_double * 3), ("mu", C.c_double), ("alpha", C.c_double),
                ("pja_iters", C.c_int32), ("n_threads", C.c_int32), ("cell_size", C.c_float),
                ("hash_size", C.c_uint32), ("cyclic_z", C.c_double * 2), ("pja_weight", C.c_int32)]


class OrcBody(C.Structure):
    _fields_ = [("kind", C.c_int32), ("is_free", C.c_int32), ("shape", C.c_double * 12), ("pos", C.c_double * 3),
                ("quat", C.c_double * 4), ("lin_vel", C.c_double * 3), ("ang_vel", C.c_double * 3),
                ("mass", C.c_double), ("inertia", C.c_double * 3), ("grid", C.c_void_p),
                ("grid_dims", C.c_uint32 * 3)]


class OrcCamera(C.Structure):
    _fields_ = [("kind", C.c_int32), ("width", C.c_int32), ("height", C.c_int32), ("pos", C.c_double * 3),
                ("quat", C.c_double * 4), ("extent", C.c_double * 2), ("fov_y", C.c_double),
                ("near_clip", C.c_double), ("far_clip", C.c_double), ("empty", C.c_double),
                ("body_mask", C.c_uint32), ("march_steps", C.c_uint32), ("march_eps", C.c_double)]


class OrcStats(C.Structure):
    _fields_ = [("n_pp", C.c_int64), ("n_body", C.c_int64), ("n_corner", C.c_int64), ("max_pp", C.c_int32),
                ("max_body", C.c_int32), ("max_psi", C.c_double), ("ncp_residual", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    """The oracle library: the one build() makes, or the build named by the environment
    variable GG_ORACLE_LIB (tests/oracle_mutations.py points it at copies of the oracle
    with one mistake planted, to check that the pins catch each)."""
    global _lib
    if _lib is None:
        L = C.CDLL(os.environ.get("GG_ORACLE_LIB") or build())
        P = C.POINTER
        L.orc_inv_cell.restype = C.c_float
        L.orc_inv_cell.argtypes = [C.c_float]
        L.orc_cell_index.restype = C.c_int32
        L.orc_cell_index.argtypes = [C.c_float, C.c_float]
        L.orc_hash.restype = C.c_uint32
        L.orc_hash.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_uint32]
        L.orc_cell_keys.argtypes = [C.c_uint32, P(C.c_double), C.c_float, C.c_uint32, P(C.c_uint32)]
        L.orc_sort_perm.argtypes = [C.c_uint32, P(C.c_uint32), P(C.c_uint32)]
        L.orc_contacts.restype = C.c_int
        L.orc_contacts.argtypes = [P(OrcParams), C.c_uint32, P(C.c_double), P(C.c_double), C.c_uint32, P(OrcBody),
                                   C.c_int, P(C.c_uint32), P(C.c_uint32), P(C.c_double), P(C.c_uint32),
                                   P(C.c_uint32), P(C.c_double), P(OrcStats)]
        L.orc_step.restype = C.c_int
        L.orc_step.argtypes = [P(OrcParams), C.c_uint32, P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_double),
                               C.c_uint32, P(OrcBody), P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_double),
                               P(OrcStats)]
        L.orc_sdf.restype = C.c_double
        L.orc_sdf.argtypes = [P(OrcBody), P(C.c_double), P(C.c_double)]
        L.orc_render.restype = None
        L.orc_render.argtypes = [P(OrcCamera), C.c_uint32, P(C.c_double), P(C.c_double), C.c_uint32, P(OrcBody),
                                 P(C.c_double)]
        L.orc_scoop_loss.restype = C.c_double
        L.orc_scoop_loss.argtypes = [C.c_uint32, P(C.c_double), P(C.c_double), P(OrcBody), C.c_double]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t)) if a is not None else None


def _f32(v):
    return float(np.float32(v))


def default_cell_size(r_max: float) -> float:
    """The documented default cell edge: float32(2.002 * r_max)."""
    return float(np.float32(2.002 * float(np.float32(r_max))))


def make_params(params, n: int, r_max: float, n_threads: int = 1) -> OrcParams:
    p = OrcParams()
    p.dt = _f32(params.dt)
    for k in range(3):
        p.gravity[k] = _f32(params.gravity[k])
    p.mu = _f32(params.mu)
    p.alpha = _f32(params.alpha)
    p.pja_iters = int(params.pja_iters)
    p.n_threads = int(n_threads)
    p.cell_size = params.cell_size if params.cell_size > 0 else default_cell_size(r_max)
    p.hash_size = params.hash_size if params.hash_size > 0 else max(1, 2 * n)
    cz = getattr(params, "cyclic_z", (0.0, 0.0))
    p.cyclic_z[0], p.cyclic_z[1] = _f32(cz[0]), _f32(cz[1])
    p.pja_weight = int(getattr(params, "pja_weight", 0))
    return p


def make_bodies(bodies) -> C.Array:
    arr = (OrcBody * max(1, len(bodies)))()
    for k, b in enumerate(bodies):
        o = arr[k]
        o.kind = int(b.kind)
        o.is_free = int(b.is_free)
        for a, v in enumerate(b.shape12()):
            o.shape[a] = _f32(v)
        for a in range(3):
            o.pos[a] = _f32(b.pos[a])
            o.lin_vel[a] = _f32(b.lin_vel[a])
            o.ang_vel[a] = _f32(b.ang_vel[a])
            o.inertia[a] = _f32(b.inertia[a])
        for a in range(4):
            o.quat[a] = _f32(b.quat[a])
        o.mass = _f32(b.mass)
        g = getattr(b, "grid", None)
        if g is not None:   # the caller keeps b (and so the samples) alive while arr is used
            assert g.values.dtype == np.float32 and g.values.flags["C_CONTIGUOUS"]
            o.grid = g.values.ctypes.data
            nz, ny, nx = g.values.shape
            o.grid_dims[0], o.grid_dims[1], o.grid_dims[2] = nx, ny, nz
    return arr


def inv_cell(cell_size: float) -> float:
    return lib().orc_inv_cell(cell_size)


def cell_index(x: float, inv_c: float) -> int:
    return lib().orc_cell_index(x, inv_c)


def hash_cell(k0: int, k1: int, k2: int, n_h: int) -> int:
    return lib().orc_hash(k0, k1, k2, n_h)


def cell_keys(x: np.ndarray, cell_size: float, n_h: int) -> np.ndarray:
    x = np.ascontiguousarray(x[:, :3], np.float64)
    out = np.empty(x.shape[0], np.uint32)
    lib().orc_cell_keys(x.shape[0], _p(x, C.c_double), inv_cell(cell_size), n_h, _p(out, C.c_uint32))
    return out


def sort_perm(keys: np.ndarray) -> np.ndarray:
    keys = np.ascontiguousarray(keys, np.uint32)
    out = np.empty(keys.shape[0], np.uint32)
    lib().orc_sort_perm(keys.shape[0], _p(keys, C.c_uint32), _p(out, C.c_uint32))
    return out


def contacts(x, r, bodies, params, brute=False, n_threads=1):
    """Contact lists of the state (x: (n,3), r: (n,)) as CSR arrays by particle id."""
    x = np.ascontiguousarray(np.asarray(x, np.float64)[:, :3])
    r = np.ascontiguousarray(r, np.float64)
    n = x.shape[0]
    p = make_params(params, n, float(r.max()) if n else 0.0, n_threads)
    ba = make_bodies(bodies)
    st = OrcStats()
    L = lib()
    pp_off = np.zeros(n + 1, np.uint32)
    bc_off = np.zeros(n + 1, np.uint32)
    rc = L.orc_contacts(C.byref(p), n, _p(x, C.c_double), _p(r, C.c_double), len(bodies), ba, int(brute),
                        _p(pp_off, C.c_uint32), None, None, _p(bc_off, C.c_uint32), None, None, C.byref(st))
    if rc != 0:
        raise RuntimeError("oracle contact build overflowed")
    npp, nbc = int(pp_off[-1]), int(bc_off[-1])
    pp_j = np.zeros(max(npp, 1), np.uint32)
    pp_geom = np.zeros((max(npp, 1), 4), np.float64)
    bc_b = np.zeros(max(nbc, 1), np.uint32)
    bc_geom = np.zeros((max(nbc, 1), 7), np.float64)
    L.orc_contacts(C.byref(p), n, _p(x, C.c_double), _p(r, C.c_double), len(bodies), ba, int(brute),
                   _p(pp_off, C.c_uint32), _p(pp_j, C.c_uint32), _p(pp_geom, C.c_double), _p(bc_off, C.c_uint32),
                   _p(bc_b, C.c_uint32), _p(bc_geom, C.c_double), C.byref(st))
    return {"pp_off": pp_off, "pp_j": pp_j[:npp], "pp_geom": pp_geom[:npp], "bc_off": bc_off,
            "bc_b": bc_b[:nbc], "bc_geom": bc_geom[:nbc], "stats": st.as_dict()}


def render(cam, x, r, bodies) -> np.ndarray:
    """Depth observation (height, width) of spheres (x: (n, 3), r: (n,)) and bodies."""
    c = OrcCamera()
    c.kind, c.width, c.height = int(cam.kind), int(cam.width), int(cam.height)
    for k in range(3):
        c.pos[k] = _f32(cam.pos[k])
    for k in range(4):
        c.quat[k] = _f32(cam.quat[k])
    c.extent[0], c.extent[1] = _f32(cam.extent[0]), _f32(cam.extent[1])
    c.fov_y, c.near_clip, c.far_clip, c.empty = _f32(cam.fov_y), _f32(cam.near), _f32(cam.far), _f32(cam.empty)
    c.body_mask, c.march_steps, c.march_eps = int(cam.body_mask) & 0xFFFFFFFF, int(cam.march_steps), _f32(cam.march_eps)
    x = np.ascontiguousarray(np.asarray(x, np.float64)[:, :3])
    r = np.ascontiguousarray(r, np.float64)
    ba = make_bodies(bodies)
    out = np.zeros((c.height, c.width), np.float64)
    lib().orc_render(C.byref(c), x.shape[0], _p(x, C.c_double), _p(r, C.c_double), len(bodies), ba,
                     _p(out, C.c_double))
    return out


def sdf(body, xw) -> tuple:
    ba = make_bodies([body])
    xw = np.ascontiguousarray(xw, np.float64)
    nrm = np.zeros(3, np.float64)
    f = lib().orc_sdf(ba, _p(xw, C.c_double), _p(nrm, C.c_double))
    return f, nrm


class Sim:
    """FP64 oracle simulation of one scene (all float32 inputs widened exactly)."""

    def __init__(self, pos_r, vel, mass, bodies, params, twist=None, n_threads=1):
        pos_r = np.asarray(pos_r, np.float32)
        self.n = pos_r.shape[0]
        self.x = np.ascontiguousarray(pos_r[:, :3], np.float64)
        self.r = np.ascontiguousarray(pos_r[:, 3], np.float64)
        self.v = np.ascontiguousarray(np.asarray(vel, np.float32)[:, :3], np.float64)
        self.m = np.ascontiguousarray(np.asarray(mass, np.float32), np.float64)
        self.body_list = list(bodies)
        self.nb = len(self.body_list)
        self.bodies = make_bodies(self.body_list)
        self.params = params
        self.p = make_params(params, self.n, float(self.r.max()) if self.n else 0.0, n_threads)
        self.twist = {int(k): np.asarray(v, np.float32) for k, v in (twist or {}).items()}
        self.step_index = 0
        self.wrench = np.zeros((max(self.nb, 1), 6), np.float64)
        self.stats = OrcStats()

    def _twist_now(self):
        if not self.twist:
            return None
        t = np.zeros((max(self.nb, 1), 6), np.float64)
        for b in range(self.nb):
            o = self.bodies[b]
            t[b, :3] = list(o.lin_vel)
            t[b, 3:] = list(o.ang_vel)
            tab = self.twist.get(b)
            if tab is not None and self.step_index < tab.shape[0] and not o.is_free:
                t[b] = tab[self.step_index].astype(np.float64)
        return t

    def step(self, n_steps=1, pp_lam=None, bc_lam=None):
        L = lib()
        for _ in range(n_steps):
            tw = self._twist_now()
            rc = L.orc_step(C.byref(self.p), self.n, _p(self.x, C.c_double), _p(self.v, C.c_double),
                            _p(self.r, C.c_double), _p(self.m, C.c_double), self.nb, self.bodies,
                            _p(tw, C.c_double), _p(self.wrench, C.c_double), _p(pp_lam, C.c_double),
                            _p(bc_lam, C.c_double), C.byref(self.stats))
            if rc == -2:
                raise RuntimeError("oracle step: pja_weight = 1 (Alg. 1 as printed) with a free body")
            if rc != 0:
                raise RuntimeError("oracle step failed (contact overflow)")
            self.step_index += 1
        return self

    def body_pose(self, b):
        o = self.bodies[b]
        return np.array(list(o.pos) + list(o.quat), np.float64)

    def body_twist(self, b):
        o = self.bodies[b]
        return np.array(list(o.lin_vel) + list(o.ang_vel), np.float64)

    def set_state(self, x, v):
        self.x[:] = x
        self.v[:] = v

    def contacts(self, brute=False):
        return contacts_from(self, brute)

    def scoop_loss(self, body_index, eps):
        return lib().orc_scoop_loss(self.n, _p(self.x, C.c_double), _p(self.m, C.c_double),
                                    C.byref(self.bodies[body_index]), eps)


def contacts_from(sim: Sim, brute=False):
    """Contact lists of a Sim's current state (its own bodies, params and radii)."""
    n = sim.n
    L = lib()
    st = OrcStats()
    pp_off = np.zeros(n + 1, np.uint32)
    bc_off = np.zeros(n + 1, np.uint32)
    rc = L.orc_contacts(C.byref(sim.p), n, _p(sim.x, C.c_double), _p(sim.r, C.c_double), sim.nb, sim.bodies,
                        int(brute), _p(pp_off, C.c_uint32), None, None, _p(bc_off, C.c_uint32), None, None,
                        C.byref(st))
    if rc != 0:
        raise RuntimeError("oracle contact build overflowed")
    npp, nbc = int(pp_off[-1]), int(bc_off[-1])
    pp_j = np.zeros(max(npp, 1), np.uint32)
    pp_geom = np.zeros((max(npp, 1), 4), np.float64)
    bc_b = np.zeros(max(nbc, 1), np.uint32)
    bc_geom = np.zeros((max(nbc, 1), 7), np.float64)
    L.orc_contacts(C.byref(sim.p), n, _p(sim.x, C.c_double), _p(sim.r, C.c_double), sim.nb, sim.bodies,
                   int(brute), _p(pp_off, C.c_uint32), _p(pp_j, C.c_uint32), _p(pp_geom, C.c_double),
                   _p(bc_off, C.c_uint32), _p(bc_b, C.c_uint32), _p(bc_geom, C.c_double), C.byref(st))
    return {"pp_off": pp_off, "pp_j": pp_j[:npp], "pp_geom": pp_geom[:npp], "bc_off": bc_off,
            "bc_b": bc_b[:nbc], "bc_geom": bc_geom[:nbc], "stats": st.as_dict()}
