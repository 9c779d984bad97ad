"""Thin ctypes binding of libgg.so (include/gg.h): argument marshalling only.

Every step of the contact pipeline runs in the library's CUDA kernels.  Inputs
may be numpy arrays (host) or CUDA torch tensors (device); outputs come back as
numpy arrays unless a CUDA tensor is given as `out`.  If libgg.so is missing the
import of this module still works, but creating a simulation raises: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# GG_DEBUG=1 in the environment loads the checked build (libgg_debug.so: device-side
# index checks that report GG_ERR_INTERNAL instead of touching memory out of range)
LIB_PATH = os.path.join(_PKG, "libgg_debug.so" if os.environ.get("GG_DEBUG") == "1" else "libgg.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_CONTACT_OVERFLOW, ERR_DEVICE_TIMEOUT, ERR_NONFINITE, \
    ERR_UNSUPPORTED, ERR_NO_DEVICE = range(9)

FIELD = {"POS": 0, "VEL": 1, "BODY_STATE": 2, "BODY_WRENCH": 3, "CELL_KEY": 4, "SORT_PERM": 5, "CELL_START": 6,
         "CONTACTS": 7, "CONTACT_GEOM": 8, "CONTACT_IMPULSE": 9, "BODY_CONTACT_GEOM": 10,
         "BODY_CONTACT_IMPULSE": 11, "STATS": 12, "STATE": 13, "POS_VEL": 14}

# exported functions: name -> (restype, argtypes)
_P = C.c_void_p
SIGNATURES = {
    "gg_abi_version": (C.c_uint32, []),
    "gg_status_string": (C.c_char_p, [C.c_int]),
    "gg_create": (C.c_int, [_P, C.c_uint32, _P, _P, _P, C.c_int, C.POINTER(C.c_void_p)]),
    "gg_create_batch": (C.c_int, [_P, C.c_uint32, _P, _P, _P, _P, C.c_int, C.POINTER(C.c_void_p)]),
    "gg_set_bodies": (C.c_int, [_P, C.c_uint32, C.c_uint32, _P]),
    "gg_set_trajectory": (C.c_int, [_P, C.c_uint32, C.c_uint32, C.c_uint32, _P, C.c_int]),
    "gg_set_body_grid": (C.c_int, [_P, C.c_uint32, C.c_uint32, _P, _P, C.c_float, _P, C.c_int]),
    "gg_render": (C.c_int, [_P, C.c_uint32, _P, _P, C.c_int, _P]),
    "gg_autotune": (C.c_int, [_P, _P]),
    "gg_set_particles": (C.c_int, [_P, _P, _P, C.c_int, _P]),
    "gg_step": (C.c_int, [_P, C.c_uint32, _P]),
    "gg_sync": (C.c_int, [_P, _P]),
    "gg_step_io": (C.c_int, [_P, _P, _P, _P, _P]),
    "gg_field_bytes": (C.c_size_t, [_P, C.c_int]),
    "gg_readback": (C.c_int, [_P, C.c_int, _P, C.c_size_t, C.c_int, _P]),
    "gg_set_state": (C.c_int, [_P, _P, C.c_size_t, C.c_int, _P]),
    "gg_tuning_count": (C.c_uint32, []),
    "gg_hash_size": (C.c_uint32, [_P, C.c_uint32]),
    "gg_cell_size": (C.c_float, [_P, C.c_uint32]),
    "gg_tuning_flags": (C.c_uint32, [C.c_uint32]),
    "gg_enable_timing": (C.c_int, [_P, C.c_int]),
    "gg_stage_ms": (C.c_int, [_P, C.POINTER(C.c_float)]),
    "gg_kernels_per_step": (C.c_uint32, [_P]),
    "gg_tuning_selected": (C.c_uint32, [_P]),
    "gg_last_error": (C.c_char_p, [_P]),
    "gg_destroy": (None, [_P]),
    "gg_bin_sort_noalloc": (C.c_int, [_P, C.c_uint32, C.c_float, C.c_uint32, _P, _P, _P, _P]),
    "gg_tape_reserve": (C.c_int, [_P, C.c_uint32, C.c_uint32]),
    "gg_step_taped": (C.c_int, [_P, C.c_uint32, C.c_uint32, _P]),
    "gg_backward": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_int, _P]),
}


class GGParams(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("dt", C.c_float), ("gravity", C.c_float * 3), ("mu", C.c_float),
                ("alpha", C.c_float), ("pja_iters", C.c_uint32), ("cell_size", C.c_float),
                ("hash_factor", C.c_uint32), ("hash_size", C.c_uint32), ("max_contacts", C.c_uint32),
                ("max_body_contacts", C.c_uint32), ("max_bodies", C.c_uint32), ("density", C.c_float),
                ("tuning", C.c_uint32), ("wrench_history", C.c_uint32), ("max_free_bodies", C.c_uint32),
                ("free_contact_capacity", C.c_uint32), ("barrier_test_phantoms", C.c_uint32),
                ("binning", C.c_uint32), ("cyclic_z", C.c_float * 2), ("wait_limit_us", C.c_uint32),
                ("hash_tune", C.c_uint32), ("pja_weight", C.c_uint32)]


class GGBody(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("is_free", C.c_uint32), ("shape", C.c_float * 12), ("pos", C.c_float * 3),
                ("quat", C.c_float * 4), ("lin_vel", C.c_float * 3), ("ang_vel", C.c_float * 3),
                ("mass", C.c_float), ("inertia", C.c_float * 3)]


class GGCamera(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("kind", C.c_uint32), ("width", C.c_uint32), ("height", C.c_uint32),
                ("pos", C.c_float * 3), ("quat", C.c_float * 4), ("extent", C.c_float * 2), ("fov_y", C.c_float),
                ("near_clip", C.c_float), ("far_clip", C.c_float), ("empty", C.c_float), ("body_mask", C.c_uint32),
                ("march_steps", C.c_uint32), ("march_eps", C.c_float)]


def make_camera(cam) -> GGCamera:
    c = GGCamera()
    c.struct_size = C.sizeof(GGCamera)
    c.kind, c.width, c.height = int(cam.kind), int(cam.width), int(cam.height)
    for k in range(3):
        c.pos[k] = cam.pos[k]
    for k in range(4):
        c.quat[k] = cam.quat[k]
    c.extent[0], c.extent[1] = cam.extent
    c.fov_y, c.near_clip, c.far_clip, c.empty = cam.fov_y, cam.near, cam.far, cam.empty
    c.body_mask, c.march_steps, c.march_eps = int(cam.body_mask) & 0xFFFFFFFF, int(cam.march_steps), cam.march_eps
    return c


class GGStats(C.Structure):
    _fields_ = [("steps", C.c_uint64), ("n_pp", C.c_uint32), ("n_body", C.c_uint32), ("max_pp", C.c_uint32),
                ("max_body", C.c_uint32), ("status_flags", C.c_uint32), ("max_psi", C.c_float),
                ("n_active", C.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load():
    """Load libgg.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgg.so not built ({LIB_PATH}); run __graft_entry__.build() first")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


TUNE_BITS = {"lists": 1, "fused": 2, "lean": 4, "half": 8, "detect": 16, "serp": 32, "preload": 64, "oneloop": 128}   # GG_TUNE_* of gg.h


def tuning_flags(k):
    """Names of the GG_TUNE_* bits of launch-shape set k."""
    bits = load().gg_tuning_flags(k)
    return {name for name, b in TUNE_BITS.items() if bits & b}


class GGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status}: {load().gg_status_string(status).decode()})")
        self.status = status


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, on_device) of a numpy array or torch tensor (None -> (None, 0))."""
    if x is None:
        return None, 0
    if _is_torch(x):
        assert x.is_contiguous()
        return C.c_void_p(x.data_ptr()), int(x.is_cuda)
    assert isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"]
    return C.c_void_p(x.__array_interface__["data"][0]), 0   # (ndarray.ctypes is slow to build)


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def make_params(p, tuning=0, wrench_history=1, max_bodies=8, hash_factor=0, max_free_bodies=0,
                barrier_test_phantoms=0, binning=0, wait_limit_us=0, hash_tune=0) -> GGParams:
    q = GGParams()
    q.struct_size = C.sizeof(GGParams)
    q.dt = p.dt
    for k in range(3):
        q.gravity[k] = p.gravity[k]
    q.mu = p.mu
    q.alpha = p.alpha
    q.pja_iters = p.pja_iters
    q.cell_size = p.cell_size
    q.hash_factor = hash_factor
    q.hash_size = p.hash_size
    q.max_contacts = p.max_contacts
    q.max_body_contacts = p.max_body_contacts
    q.max_bodies = max_bodies
    q.density = 0.0
    q.tuning = tuning
    q.wrench_history = wrench_history
    q.max_free_bodies = max_free_bodies
    q.free_contact_capacity = 0
    q.barrier_test_phantoms = barrier_test_phantoms
    q.binning = binning
    q.wait_limit_us = wait_limit_us
    q.hash_tune = hash_tune
    q.pja_weight = int(getattr(p, "pja_weight", 0))
    cz = getattr(p, "cyclic_z", (0.0, 0.0))
    q.cyclic_z[0], q.cyclic_z[1] = cz[0], cz[1]
    return q


def make_bodies(bodies):
    arr = (GGBody * max(1, len(bodies)))()
    for k, b in enumerate(bodies):
        o = arr[k]
        o.kind = b.kind
        o.is_free = b.is_free
        for a, v in enumerate(b.shape12()):
            o.shape[a] = v
        for a in range(3):
            o.pos[a] = b.pos[a]
            o.lin_vel[a] = b.lin_vel[a]
            o.ang_vel[a] = b.ang_vel[a]
            o.inertia[a] = b.inertia[a]
        for a in range(4):
            o.quat[a] = b.quat[a]
        o.mass = b.mass
    return arr


class Sim:
    """One libgg simulation (single environment, or batched when env_offsets is given)."""

    def __init__(self, pos_r, vel=None, mass=None, params=None, env_offsets=None, tuning=0, wrench_history=1,
                 max_bodies=8, hash_factor=0, max_free_bodies=0, barrier_test_phantoms=0, binning=0,
                 wait_limit_us=0, hash_tune=0):
        L = load()
        self._L = L
        self.params = params
        self.gp = make_params(params, tuning, wrench_history, max_bodies, hash_factor, max_free_bodies,
                              barrier_test_phantoms, binning, wait_limit_us, hash_tune)
        n = int(pos_r.shape[0])
        self.n = n
        pp, dev = _ptr(pos_r)
        vp, dv = _ptr(vel)
        mp, dm = _ptr(mass)
        assert vel is None or dv == dev
        assert mass is None or dm == dev
        h = C.c_void_p()
        if env_offsets is None:
            st = L.gg_create(C.byref(self.gp), n, pp, vp, mp, dev, C.byref(h))
            self.n_envs = 1
        else:
            offs = np.ascontiguousarray(env_offsets, np.uint32)
            self.n_envs = len(offs) - 1
            st = L.gg_create_batch(C.byref(self.gp), self.n_envs, C.c_void_p(offs.ctypes.data), pp, vp, mp, dev,
                                   C.byref(h))
        if st != OK:
            raise GGError(st, "gg_create failed")
        self.h = h
        self._field_bytes = {}
        self.max_bodies = max_bodies
        self.K = self.gp.max_contacts or 16
        self.Kb = self.gp.max_body_contacts or 4
        self.H = max(1, wrench_history)

    # ------------------------------------------------------------------ setup
    def _check(self, st, what):
        if st != OK:
            raise GGError(st, f"{what}: {self._L.gg_last_error(self.h).decode()}")

    def set_bodies(self, bodies, env=0):
        """Bodies of environment env; the samples of GRID bodies (Body.grid) follow."""
        arr = make_bodies(bodies)
        self._check(self._L.gg_set_bodies(self.h, env, len(bodies), arr), "gg_set_bodies")
        for b, body in enumerate(bodies):
            if getattr(body, "grid", None) is not None:
                self.set_body_grid(b, body.grid, env)

    def set_body_grid(self, body, grid, env=0):
        """Samples of GRID body `body`: grid.values float32 (nz, ny, nx), grid.origin, grid.spacing."""
        v = grid.values
        if _is_torch(v):
            p, dev = _ptr(v.contiguous())
            nz, ny, nx = v.shape
        else:
            v = np.ascontiguousarray(v, np.float32)
            p, dev = _ptr(v)
            nz, ny, nx = v.shape
        dims = (C.c_uint32 * 3)(nx, ny, nz)
        org = (C.c_float * 3)(*[float(o) for o in grid.origin])
        self._check(self._L.gg_set_body_grid(self.h, env, body, dims, org, float(grid.spacing), p, dev),
                    "gg_set_body_grid")

    def set_trajectory(self, body, twist, env=0):
        tw = twist if _is_torch(twist) else np.ascontiguousarray(twist, np.float32)
        p, dev = _ptr(tw)
        self._check(self._L.gg_set_trajectory(self.h, env, body, int(tw.shape[0]), p, dev), "gg_set_trajectory")

    def step_io(self, pos_r, vel, out, stream=None):
        """gg_step_io: state in from host buffers, one step, the new state (POS_VEL
        layout, float[7 n]) into `out`, waited for."""
        pp, d0 = _ptr(pos_r)
        vp, d1 = _ptr(vel)
        op, d2 = _ptr(out)
        assert not (d0 or d1 or d2), "gg_step_io takes host buffers"
        self._check(self._L.gg_step_io(self.h, pp, vp, op, _stream(stream)), "gg_step_io")
        return out

    def set_particles(self, pos_r, vel=None, stream=None):
        pp, dev = _ptr(pos_r)
        vp, _ = _ptr(vel)
        self._check(self._L.gg_set_particles(self.h, pp, vp, dev, _stream(stream)), "gg_set_particles")

    @classmethod
    def from_scene(cls, scene, tuning=0, wrench_history=1, max_bodies=8, hash_factor=0, device_inputs=None,
                   binning=0, hash_tune=0):
        args = (scene.pos_r, scene.vel, scene.mass) if device_inputs is None else device_inputs
        n_free = sum(1 for b in scene.bodies if b.is_free)
        sim = cls(*args, params=scene.params, env_offsets=scene.env_offsets, tuning=tuning,
                  wrench_history=wrench_history, max_bodies=max_bodies, hash_factor=hash_factor,
                  max_free_bodies=n_free, binning=binning, hash_tune=hash_tune)
        if scene.body_offsets is None:
            if scene.bodies:
                sim.set_bodies(scene.bodies, 0)
            for b, tw in scene.twist.items():
                sim.set_trajectory(b, tw, 0)
        else:
            bo = scene.body_offsets
            for e in range(len(bo) - 1):
                sim.set_bodies(scene.bodies[bo[e]:bo[e + 1]], e)
            for gb, tw in scene.twist.items():
                e = int(np.searchsorted(bo, gb, side="right") - 1)
                sim.set_trajectory(gb - int(bo[e]), tw, e)
        return sim

    # ------------------------------------------------------------------ run
    def step(self, n_steps=1, stream=None):
        self._check(self._L.gg_step(self.h, n_steps, _stream(stream)), "gg_step")

    def sync(self, stream=None):
        self._check(self._L.gg_sync(self.h, _stream(stream)), "gg_sync")

    def enable_timing(self, on=True):
        self._check(self._L.gg_enable_timing(self.h, int(on)), "gg_enable_timing")

    STAGES = ("bin_sort", "contacts", "pja", "integrate_wrench")

    def stage_ms(self):
        """Device milliseconds per stage of the last enqueued step (timing must be on)."""
        out = (C.c_float * 4)()
        self._check(self._L.gg_stage_ms(self.h, out), "gg_stage_ms")
        return dict(zip(self.STAGES, [float(v) for v in out]))

    @property
    def kernels_per_step(self):
        return self._L.gg_kernels_per_step(self.h)

    def autotune(self, stream=None):
        """Re-time the launch-shape sets on the current state and keep the fastest."""
        self._check(self._L.gg_autotune(self.h, _stream(stream)), "gg_autotune")

    @property
    def tuning_selected(self):
        return self._L.gg_tuning_selected(self.h)

    @property
    def tuning_flags(self):
        """Names of the GG_TUNE_* bits of the selected set ("lists", "fused", "lean", "half")."""
        return tuning_flags(self.tuning_selected)

    # ------------------------------------------------------------------ readback
    def field_bytes(self, field):
        if field == "CELL_START":   # n_h + 1 entries: changes when the autotuner picks n_h
            return self._L.gg_field_bytes(self.h, FIELD[field])
        nb = self._field_bytes.get(field)   # the others are fixed for the simulation's lifetime
        if nb is None:
            nb = self._field_bytes[field] = self._L.gg_field_bytes(self.h, FIELD[field])
        return nb

    def hash_size(self, env=0):
        """n_h in use for environment `env` (Eq. 6's modulus)."""
        return self._L.gg_hash_size(self.h, env)

    def cell_size(self, env=0):
        """Cell edge in use for environment `env` (the grid of Eq. 6's keys)."""
        return float(self._L.gg_cell_size(self.h, env))

    def read(self, field, dtype=np.float32, shape=None, out=None, stream=None, check=True):
        nb = self.field_bytes(field)
        if out is None:
            out = np.empty(nb // np.dtype(dtype).itemsize, dtype)
            if shape is not None:
                out = out.reshape(shape)
        p, dev = _ptr(out)
        st = self._L.gg_readback(self.h, FIELD[field], p, nb, dev, _stream(stream))
        if check:
            self._check(st, f"gg_readback({field})")
        return out

    def pos(self):
        return self.read("POS", shape=(self.n, 4))

    def vel(self):
        return self.read("VEL", shape=(self.n, 3))

    def render(self, camera, env=0, out=None, stream=None):
        """Depth observation (height, width) of environment env (gg_render): into `out`
        (a CUDA tensor: asynchronous) or a new numpy array."""
        c = make_camera(camera)
        if out is None:
            out = np.empty((c.height, c.width), np.float32)
        p, dev = _ptr(out)
        self._check(self._L.gg_render(self.h, env, C.byref(c), p, dev, _stream(stream)), "gg_render")
        return out

    def pos_vel(self, out=None, stream=None):
        """Positions (n, 4) and velocities (n, 3) in one copy (and one wait, to the host):
        `out` holds 7 n floats, positions first."""
        buf = self.read("POS_VEL", out=out, stream=stream)
        flat = buf.reshape(-1)
        return flat[:4 * self.n].reshape(self.n, 4), flat[4 * self.n:].reshape(self.n, 3)

    def body_state(self):
        return self.read("BODY_STATE", shape=(self.n_envs * self.max_bodies, 16))

    def wrench(self):
        return self.read("BODY_WRENCH", shape=(self.H, self.n_envs * self.max_bodies, 6))

    def cell_keys(self):
        return self.read("CELL_KEY", np.uint32)

    def sort_perm(self):
        return self.read("SORT_PERM", np.uint32)

    def cell_start(self):
        return self.read("CELL_START", np.uint32)

    def contacts(self):
        """Contact lists of the last step as CSR arrays by particle id (like the oracle's)."""
        W = 2 + self.K + self.Kb
        rows = self.read("CONTACTS", np.uint32, shape=(self.n, W))
        geom = self.read("CONTACT_GEOM", shape=(self.n, self.K, 4))
        lam = self.read("CONTACT_IMPULSE", shape=(self.n, self.K, 3))
        bgeom = self.read("BODY_CONTACT_GEOM", shape=(self.n, self.Kb, 8))
        blam = self.read("BODY_CONTACT_IMPULSE", shape=(self.n, self.Kb, 3))
        npp = rows[:, 0].astype(np.int64)
        nbc = rows[:, 1].astype(np.int64)
        mpp = np.arange(self.K)[None, :] < npp[:, None]
        mb = np.arange(self.Kb)[None, :] < nbc[:, None]
        pp_off = np.concatenate([[0], np.cumsum(npp)]).astype(np.uint32)
        bc_off = np.concatenate([[0], np.cumsum(nbc)]).astype(np.uint32)
        return {"pp_off": pp_off, "pp_j": rows[:, 2:2 + self.K][mpp], "pp_geom": geom[mpp], "pp_lam": lam[mpp],
                "bc_off": bc_off, "bc_b": rows[:, 2 + self.K:][mb], "bc_geom": bgeom[mb][:, :7],
                "bc_lam": blam[mb]}

    # ------------------------------------------------------------------ adjoint
    def tape_reserve(self, n_steps, checkpoint_every):
        self._check(self._L.gg_tape_reserve(self.h, n_steps, checkpoint_every), "gg_tape_reserve")

    def step_taped(self, tool_body, n_steps, stream=None):
        self._check(self._L.gg_step_taped(self.h, tool_body, n_steps, _stream(stream)), "gg_step_taped")
        self._taped = n_steps

    def backward(self, dpos, dvel=None, dpose=None, stream=None):
        """Gradients (dL/dtwist float32 (T, 6), dL/dmu float) of a loss whose gradient
        w.r.t. the final positions (n, 3), velocities (n, 3) and tool pose (7,) is given.
        numpy in -> numpy out; CUDA tensors in -> CUDA tensors out."""
        if _is_torch(dpos):
            import torch
            dev = dpos.device
            dtw = torch.empty((self._taped, 6), dtype=torch.float32, device=dev)
            dmu = torch.empty((1,), dtype=torch.float32, device=dev)
            args = [t.contiguous() if t is not None else None for t in (dpos, dvel, dpose)]   # keep alive
            ptrs = [C.c_void_p(t.data_ptr()) if t is not None else None for t in args]
            st = self._L.gg_backward(self.h, ptrs[0], ptrs[1], ptrs[2], C.c_void_p(dtw.data_ptr()),
                                     C.c_void_p(dmu.data_ptr()), 1, _stream(stream))
            self._check(st, "gg_backward")
            return dtw, dmu
        dpos = np.ascontiguousarray(dpos, np.float32)
        dvel = None if dvel is None else np.ascontiguousarray(dvel, np.float32)
        dpose = None if dpose is None else np.ascontiguousarray(dpose, np.float32)
        dtw = np.empty((self._taped, 6), np.float32)
        dmu = np.empty(1, np.float32)
        st = self._L.gg_backward(self.h, _ptr(dpos)[0], _ptr(dvel)[0], _ptr(dpose)[0], C.c_void_p(dtw.ctypes.data),
                                 C.c_void_p(dmu.ctypes.data), 0, _stream(stream))
        self._check(st, "gg_backward")
        return dtw, float(dmu[0])

    def stats(self):
        s = GGStats()
        p = C.c_void_p(C.addressof(s))
        st = self._L.gg_readback(self.h, FIELD["STATS"], p, C.sizeof(s), 0, None)
        d = s.as_dict()
        d["status"] = st
        return d

    def state(self):
        return self.read("STATE", np.uint8)

    def set_state(self, blob, stream=None):
        p, dev = _ptr(blob)
        self._check(self._L.gg_set_state(self.h, p, int(blob.nbytes), dev, _stream(stream)), "gg_set_state")

    def close(self):
        if getattr(self, "h", None):
            self._L.gg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
