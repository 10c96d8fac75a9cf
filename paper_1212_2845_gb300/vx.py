"""ctypes binding of the C ABI in ``include/vx.h`` (argument marshalling only).

Every step of the simulation runs in the CUDA library ``_build/libvx.so``.
There is no CPU path: if the library is missing or no GPU is visible, calls
raise.  Functions keep the C names; :class:`Sim` wraps one ``vx_sim``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build_san" if os.environ.get("VX_HOST_SANITIZE") == "1" else
                        ("_build_bc" if os.environ.get("VX_BOUNDS_CHECK") == "1" else "_build"), "libvx.so")

VX_OK = 0
ERRORS = {-1: "VX_ERR_ARG", -2: "VX_ERR_CUDA", -3: "VX_ERR_OOM", -4: "VX_ERR_UNSTABLE",
          -5: "VX_ERR_TIMEOUT", -6: "VX_ERR_STATE", -7: "VX_ERR_CAPACITY", -8: "VX_ERR_BOUNDS"}
FLAG_FIXED = 1
FLAG_STATIC = 2
GROUPS_RESIDENT = -1    # vx_set_batching: the shared-memory-resident form (split chosen automatically)
GROUPS_RESIDENT_BOND = -2   # ... with one thread per bond in the bond phase
GROUPS_RESIDENT_VOXEL = -3  # ... with one thread per voxel in the bond phase


class VxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Material(C.Structure):
    _fields_ = [(n, C.c_float) for n in ("E", "nu", "rho", "cte", "mu_s", "mu_k")]


class Desc(C.Structure):
    _fields_ = [("n_bodies", C.c_int32), ("dims", C.POINTER(C.c_int32)), ("grid", C.POINTER(C.c_uint8)),
                ("voxel_size", C.c_float), ("palette", C.POINTER(Material)), ("n_materials", C.c_int32),
                ("origin", C.POINTER(C.c_float))]


class StateView(C.Structure):
    _fields_ = [("offset", C.c_void_p), ("quat", C.c_void_p), ("vel", C.c_void_p), ("angvel", C.c_void_p),
                ("flags", C.c_void_p)]


_P = C.c_void_p
_i32, _i64, _f32 = C.c_int32, C.c_int64, C.c_float
_pi64 = C.POINTER(C.c_int64)
_pd = C.POINTER(C.c_double)
_pf = C.POINTER(C.c_float)
_pu8 = C.POINTER(C.c_uint8)
_pi32 = C.POINTER(C.c_int32)
_pdesc = C.POINTER(Desc)

SIGNATURES = {
    "vx_version": (C.c_char_p, []),
    "vx_last_error": (C.c_char_p, []),
    "vx_plan_counts": (C.c_int, [_pdesc, _pi64, _pi64, _pi64]),
    "vx_plan_dt": (C.c_int, [_pdesc, _pf, _f32, _pd]),
    "vx_region_mask": (C.c_int, [_pdesc, _i32, _pf, _pf, _pu8, _pi64]),
    "vx_plan_tiles": (C.c_int, [_pdesc, _i32, _pi64, _pi64, _pi64, _pi32, _pi32]),
    "vx_set_step_form": (C.c_int, [_P, _i32, _i32]),
    "vx_get_tiling": (C.c_int, [_P, _pi32, _pi64, _pi32, _pi64]),
    "vx_set_batching": (C.c_int, [_P, _i64]),
    "vx_set_multistep": (C.c_int, [_P, _i32]),
    "vx_set_barrier_limits": (C.c_int, [_P, _i64, _i32]),
    "vx_create": (C.c_int, [_pdesc, C.POINTER(_P)]),
    "vx_destroy": (None, [_P]),
    "vx_get_counts": (C.c_int, [_P, _pi64, _pi64, _pi64]),
    "vx_get_anchors": (C.c_int, [_P, _pd]),
    "vx_set_materials": (C.c_int, [_P, C.POINTER(Material), _i32]),
    "vx_set_voxel_params": (C.c_int, [_P, _pf, _pf]),
    "vx_set_fixed_mask": (C.c_int, [_P, _pu8]),
    "vx_add_fixed_region": (C.c_int, [_P, _i32, _pf, _pf, _pi64]),
    "vx_add_forced_region": (C.c_int, [_P, _i32, _pf, _pf, _pf, _pi64]),
    "vx_set_forces": (C.c_int, [_P, _pf]),
    "vx_set_damping": (C.c_int, [_P, _f32, _f32, _f32]),
    "vx_set_environment": (C.c_int, [_P, _f32, _i32, _i32]),
    "vx_set_actuation": (C.c_int, [_P, _f32, _i64, _f32]),
    "vx_set_initial_velocity": (C.c_int, [_P, _pf]),
    "vx_set_material_actuation": (C.c_int, [_P, _pf, _pf, _pf]),
    "vx_set_dt_factor": (C.c_int, [_P, _f32]),
    "vx_get_dt": (C.c_int, [_P, _pd]),
    "vx_set_dt": (C.c_int, [_P, _pd]),
    "vx_reset": (C.c_int, [_P, _pf]),
    "vx_read_state": (C.c_int, [_P, C.POINTER(StateView), _i32, _P]),
    "vx_write_state": (C.c_int, [_P, C.POINTER(StateView), _i32, _P]),
    "vx_write_state_async": (C.c_int, [_P, C.POINTER(StateView), _i32, _P]),
    "vx_get_step": (C.c_int, [_P, _pi64]),
    "vx_set_step": (C.c_int, [_P, _i64]),
    "vx_step": (C.c_int, [_P, _i64, _P]),
    "vx_step_async": (C.c_int, [_P, _i64, _P]),
    "vx_get_status": (C.c_int, [_P, _P, _pi32, _pi64, _pi64]),
    "vx_rebuild_collisions": (C.c_int, [_P, _P]),
    "vx_get_collision_pairs": (C.c_int, [_P, _pi32, _i64, _pi64]),
    "vx_collision_stats": (C.c_int, [_P, _pi64, _pd]),
    "vx_collision_candidates_static": (C.c_int, [_P, _P, _P, _i32, _i32, _f32, _P, _P, _P]),
    "vx_rollout_forward": (C.c_int, [_P, _i64, _i32, _pf, _P]),
    "vx_graph_capture": (C.c_int, [_P, _i64, _P]),
    "vx_audit": (C.c_int, [_P, _pd, _P]),
    "vx_set_collision_scheme": (C.c_int, [_P, _i32, _i32]),
    "vx_relax": (C.c_int, [_P, _i64, C.c_double, _i32, _pi64, _pd, _pi32, _P]),
    "vx_graph_launch": (C.c_int, [_P, _P]),
    "vx_autotune_batching": (C.c_int, [_P, _i32, _pi32, _pi64, _pd, _P]),
    "vx_rollout_backward": (C.c_int, [_P, _pf, _P, _P, _P]),
}
STATIC_MAX_SURFACE = 65536
STATIC_MAX_BODIES = 4096
CAND_CAP = 48


def collision_candidates_static(lat, offset_planes, body, n_surface, n_bodies, voxel_size, cand_count, cand,
                                stream=None):
    """vx_collision_candidates_static on caller-owned device buffers (torch
    CUDA tensors): lat int32 [S], offset_planes float32 [3, S], body int32 [S]
    or None, cand_count int32 [S], cand int32 [S, 48]."""
    _check(lib().vx_collision_candidates_static(
        lat.data_ptr(), offset_planes.data_ptr(), None if body is None else body.data_ptr(), int(n_surface),
        int(n_bodies), float(voxel_size), cand_count.data_ptr(), cand.data_ptr(), _stream_ptr(stream)))

_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} missing "
                              "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != VX_OK:
        raise VxError(rc, lib().vx_last_error().decode())


def _ptr(a, t):
    return None if a is None else a.ctypes.data_as(C.POINTER(t))


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


class _DescHolder:
    """vx_desc built from a scene dictionary (keeps the arrays alive)."""

    def __init__(self, sc):
        self.dims = np.ascontiguousarray(sc["dims"], dtype=np.int32).reshape(-1, 3)
        self.grid = np.ascontiguousarray(sc["grid"], dtype=np.uint8).ravel()
        pal = np.asarray(sc["palette"], dtype=np.float64).reshape(-1, 6)
        self.pal = (Material * pal.shape[0])(*[Material(*map(float, row)) for row in pal])
        self.origin = np.ascontiguousarray(sc["origin"], dtype=np.float32).reshape(-1, 3)
        self.desc = Desc(self.dims.shape[0], self.dims.ctypes.data_as(_pi32), self.grid.ctypes.data_as(_pu8),
                         float(sc["voxel_size"]), self.pal, pal.shape[0], self.origin.ctypes.data_as(_pf))


def plan_counts(sc):
    h = _DescHolder(sc)
    n = [C.c_int64() for _ in range(3)]
    _check(lib().vx_plan_counts(C.byref(h.desc), *[C.byref(x) for x in n]))
    return tuple(x.value for x in n)


def plan_dt(sc, log_E=None, dt_factor=None):
    h = _DescHolder(sc)
    le = None if log_E is None else np.ascontiguousarray(log_E, dtype=np.float32)
    out = np.zeros(h.dims.shape[0])
    f = sc["dt_factor"] if dt_factor is None else dt_factor
    _check(lib().vx_plan_dt(C.byref(h.desc), _ptr(le, C.c_float), float(f), _ptr(out, C.c_double)))
    return out


def plan_tiles(sc, tile_max=256):
    h = _DescHolder(sc)
    n = [C.c_int64() for _ in range(3)]
    ml, mh = C.c_int32(), C.c_int32()
    _check(lib().vx_plan_tiles(C.byref(h.desc), int(tile_max), *[C.byref(x) for x in n], C.byref(ml), C.byref(mh)))
    return dict(n_tiles=n[0].value, n_halo=n[1].value, n_tile_bonds=n[2].value, max_local=ml.value,
                max_halo_bonds=mh.value)


FORM_FUSED = 0
FORM_TWO_PASS = 1
FORM_PIPELINED = 2


def region_mask(sc, body, loc, size):
    h = _DescHolder(sc)
    n = int(np.count_nonzero(h.grid))
    m = np.zeros(n, dtype=np.uint8)
    lo = np.ascontiguousarray(loc, dtype=np.float32)
    sz = np.ascontiguousarray(size, dtype=np.float32)
    cnt = C.c_int64()
    _check(lib().vx_region_mask(C.byref(h.desc), int(body), _ptr(lo, C.c_float), _ptr(sz, C.c_float),
                                _ptr(m, C.c_uint8), C.byref(cnt)))
    return m


class Sim:
    """One simulator instance on the current CUDA device."""

    def __init__(self, sc, apply_scene=True):
        L = lib()
        self._L = L
        self._d = _DescHolder(sc)
        h = C.c_void_p()
        _check(L.vx_create(C.byref(self._d.desc), C.byref(h)))
        self.h = h
        n = [C.c_int64() for _ in range(3)]
        _check(L.vx_get_counts(self.h, *[C.byref(x) for x in n]))
        self.N, self.n_bonds, self.n_surface = (x.value for x in n)
        self.n_bodies = self._d.dims.shape[0]
        self.n_materials = int(np.asarray(sc["palette"]).reshape(-1, 6).shape[0])
        self.l = float(np.float32(sc["voxel_size"]))
        if apply_scene:
            self.apply(sc)

    def close(self):
        if getattr(self, "h", None):
            self._L.vx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- configuration -----------------------------------------------------
    def apply(self, sc):
        self.set_damping(sc["zeta_bond"], sc["zeta_ground"], sc["zeta_collision"])
        self.set_actuation(sc["act_amplitude"], sc["act_period"], sc["act_offset"])
        if any(sc.get(k) is not None for k in ("mat_act_amplitude", "mat_act_offset", "mat_act_phase")):
            self.set_material_actuation(sc.get("mat_act_amplitude"), sc.get("mat_act_offset"),
                                        sc.get("mat_act_phase"))
        if sc.get("log_E") is not None or sc.get("phase") is not None:
            self.set_voxel_params(sc.get("log_E"), sc.get("phase"))
        self.set_dt_factor(sc["dt_factor"])
        if sc.get("fixed") is not None:
            self.set_fixed_mask(sc["fixed"])
        if sc.get("force") is not None:
            self.set_forces(sc["force"])
        self.set_environment(sc["gravity_z"], sc["floor"], sc["collide"])
        self.reset(sc.get("v0"))

    def set_damping(self, zb, zg, zc):
        _check(self._L.vx_set_damping(self.h, zb, zg, zc))

    def set_environment(self, gravity_z, floor, collide):
        # collide: False/0 off, True/1 within each body, 2 one shared world
        _check(self._L.vx_set_environment(self.h, float(gravity_z), int(bool(floor)), int(collide)))

    def set_actuation(self, amplitude, period, offset=0.0):
        _check(self._L.vx_set_actuation(self.h, float(amplitude), int(period), float(offset)))

    def set_material_actuation(self, amplitude=None, offset=None, phase=None):
        """Per-material temperature signals on the common period (Sec 2.3);
        None keeps the global amplitude / offset, or a zero phase shift."""
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float32).reshape(-1)
                for a in (amplitude, offset, phase)]
        for a in arrs:
            if a is not None and a.size != self.n_materials:
                raise ValueError("one value per material expected")
        ptr = [None if a is None else a.ctypes.data_as(_pf) for a in arrs]
        _check(self._L.vx_set_material_actuation(self.h, *ptr))

    def set_voxel_params(self, log_E=None, phase=None):
        le = None if log_E is None else np.ascontiguousarray(log_E, dtype=np.float32)
        ph = None if phase is None else np.ascontiguousarray(phase, dtype=np.float32)
        _check(self._L.vx_set_voxel_params(self.h, _ptr(le, C.c_float), _ptr(ph, C.c_float)))

    def set_fixed_mask(self, mask):
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        _check(self._L.vx_set_fixed_mask(self.h, _ptr(m, C.c_uint8)))

    def set_forces(self, F):
        f = None if F is None else np.ascontiguousarray(F, dtype=np.float32).reshape(-1, 3)
        _check(self._L.vx_set_forces(self.h, _ptr(f, C.c_float)))

    def add_fixed_region(self, body, loc, size):
        lo, sz = (np.ascontiguousarray(x, dtype=np.float32) for x in (loc, size))
        n = C.c_int64()
        _check(self._L.vx_add_fixed_region(self.h, int(body), _ptr(lo, C.c_float), _ptr(sz, C.c_float),
                                           C.byref(n)))
        return n.value

    def add_forced_region(self, body, loc, size, F):
        lo, sz, f = (np.ascontiguousarray(x, dtype=np.float32) for x in (loc, size, F))
        n = C.c_int64()
        _check(self._L.vx_add_forced_region(self.h, int(body), _ptr(lo, C.c_float), _ptr(sz, C.c_float),
                                            _ptr(f, C.c_float), C.byref(n)))
        return n.value

    def set_step_form(self, form, tile_max=0):
        _check(self._L.vx_set_step_form(self.h, int(form), int(tile_max)))

    def set_batching(self, group_voxels):
        _check(self._L.vx_set_batching(self.h, int(group_voxels)))

    def set_multistep(self, on):
        """0: one launch per step; 1 (default): multi-step launches (the
        resident form on small lattices); 2: the cooperative grid launch."""
        _check(self._L.vx_set_multistep(self.h, int(on)))

    def set_barrier_limits(self, max_spins=0, phantom_ctas=0):
        _check(self._L.vx_set_barrier_limits(self.h, int(max_spins), int(phantom_ctas)))

    def tiling(self):
        tm, ml = C.c_int32(), C.c_int32()
        nt, sm = C.c_int64(), C.c_int64()
        _check(self._L.vx_get_tiling(self.h, C.byref(tm), C.byref(nt), C.byref(ml), C.byref(sm)))
        return dict(tile_max=tm.value, n_tiles=nt.value, max_local=ml.value, smem_bytes=sm.value)

    def set_dt_factor(self, f):
        _check(self._L.vx_set_dt_factor(self.h, float(f)))

    def dt(self):
        out = np.zeros(self.n_bodies)
        _check(self._L.vx_get_dt(self.h, _ptr(out, C.c_double)))
        return out

    def set_dt(self, dt):
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (self.n_bodies,)))
        _check(self._L.vx_set_dt(self.h, _ptr(d, C.c_double)))

    def anchors(self):
        out = np.zeros((self.N, 3))
        _check(self._L.vx_get_anchors(self.h, _ptr(out, C.c_double)))
        return out

    # -- state -------------------------------------------------------------
    def set_initial_velocity(self, v):
        """Linear velocity of every non-fixed voxel now, and of later resets without one."""
        a = np.ascontiguousarray(v, dtype=np.float32).reshape(3)
        _check(self._L.vx_set_initial_velocity(self.h, a.ctypes.data_as(_pf)))

    def reset(self, v0=None):
        v = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float32)
        _check(self._L.vx_reset(self.h, _ptr(v, C.c_float)))

    def read_state(self, stream=None):
        N = self.N
        out = dict(offset=np.zeros((N, 3), np.float32), quat=np.zeros((N, 4), np.float32),
                   vel=np.zeros((N, 3), np.float32), angvel=np.zeros((N, 3), np.float32),
                   flags=np.zeros(N, np.uint8))
        v = StateView(*[out[k].ctypes.data for k in ("offset", "quat", "vel", "angvel", "flags")])
        _check(self._L.vx_read_state(self.h, C.byref(v), 0, _stream_ptr(stream)))
        return out

    def state(self):
        """Host state with absolute positions (anchor + offset, float64)."""
        s = self.read_state()
        s["pos"] = self.anchors() + s["offset"].astype(np.float64)
        s["static"] = (s["flags"] & FLAG_STATIC) >> 1
        return s

    def read_state_into(self, offset=None, quat=None, vel=None, angvel=None, flags=None, stream=None,
                        on_device=True):
        """Copy the state into caller buffers: torch CUDA tensors (on_device)
        or pinned/pageable host tensors / numpy arrays."""
        def p(x):
            if x is None:
                return None
            return x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data
        v = StateView(p(offset), p(quat), p(vel), p(angvel), p(flags))
        _check(self._L.vx_read_state(self.h, C.byref(v), int(bool(on_device)), _stream_ptr(stream)))

    def write_state_from(self, offset=None, quat=None, vel=None, angvel=None, flags=None, stream=None,
                         on_device=True, wait=True):
        """Overwrite the state from caller buffers; wait=False returns once the
        copies are enqueued (keep the buffers unchanged until the stream is done)."""
        def p(x):
            if x is None:
                return None
            return x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data
        v = StateView(p(offset), p(quat), p(vel), p(angvel), p(flags))
        fn = self._L.vx_write_state if wait else self._L.vx_write_state_async
        _check(fn(self.h, C.byref(v), int(bool(on_device)), _stream_ptr(stream)))

    def write_state(self, offset=None, quat=None, vel=None, angvel=None, flags=None, stream=None):
        arrs = [None if x is None else np.ascontiguousarray(x, dtype=np.float32) for x in (offset, quat, vel, angvel)]
        fl = None if flags is None else np.ascontiguousarray(flags, dtype=np.uint8)
        v = StateView(*[None if a is None else a.ctypes.data for a in arrs], None if fl is None else fl.ctypes.data)
        _check(self._L.vx_write_state(self.h, C.byref(v), 0, _stream_ptr(stream)))

    @property
    def step_count(self):
        n = C.c_int64()
        _check(self._L.vx_get_step(self.h, C.byref(n)))
        return n.value

    def set_step(self, n):
        _check(self._L.vx_set_step(self.h, int(n)))

    # -- stepping ----------------------------------------------------------
    def step(self, n=1, stream=None):
        _check(self._L.vx_step(self.h, int(n), _stream_ptr(stream)))

    def step_async(self, n=1, stream=None):
        _check(self._L.vx_step_async(self.h, int(n), _stream_ptr(stream)))

    def relax(self, max_steps, v_tol, check_every=100, stream=None):
        """Step until the largest voxel speed is <= v_tol [m/s] (checked every
        check_every steps) or max_steps; returns (steps, max speed, converged)."""
        n, v, c = C.c_int64(), C.c_double(), C.c_int32()
        _check(self._L.vx_relax(self.h, int(max_steps), float(v_tol), int(check_every), C.byref(n), C.byref(v),
                                C.byref(c), _stream_ptr(stream)))
        return n.value, v.value, bool(c.value)

    def status(self, stream=None):
        st, bs, bv = C.c_int32(), C.c_int64(), C.c_int64()
        _check(self._L.vx_get_status(self.h, _stream_ptr(stream), C.byref(st), C.byref(bs), C.byref(bv)))
        return st.value, bs.value, bv.value

    def audit(self, stream=None):
        """FP64 audit: dict of momentum P (3), angular momentum L (3), kinetic
        (linear, rotational), elastic and gravitational energy."""
        out = np.zeros(10)
        _check(self._L.vx_audit(self.h, _ptr(out, C.c_double), _stream_ptr(stream)))
        return dict(P=out[0:3], L=out[3:6], ke_lin=out[6], ke_rot=out[7], u_elastic=out[8], u_gravity=out[9])

    # -- captured launches and autotuning (batched form) -------------------
    def graph_capture(self, n_steps, stream=None):
        _check(self._L.vx_graph_capture(self.h, int(n_steps), _stream_ptr(stream)))

    def graph_launch(self, stream=None):
        _check(self._L.vx_graph_launch(self.h, _stream_ptr(stream)))

    def autotune_batching(self, sample_steps=20, stream=None):
        """Pick tile and group size by timing (cached per size class); returns
        (tile_max, group_voxels, sampled voxel-steps/s)."""
        tm, gv, r = C.c_int32(), C.c_int64(), C.c_double()
        _check(self._L.vx_autotune_batching(self.h, int(sample_steps), C.byref(tm), C.byref(gv), C.byref(r),
                                            _stream_ptr(stream)))
        return tm.value, gv.value, r.value

    # -- collisions --------------------------------------------------------
    def set_collision_scheme(self, all_voxels=False, every_step=False):
        _check(self._L.vx_set_collision_scheme(self.h, int(bool(all_voxels)), int(bool(every_step))))

    def rebuild_collisions(self, stream=None):
        _check(self._L.vx_rebuild_collisions(self.h, _stream_ptr(stream)))

    def collision_pairs(self):
        n = C.c_int64()
        _check(self._L.vx_get_collision_pairs(self.h, None, 0, C.byref(n)))
        p = np.zeros((max(n.value, 1), 2), dtype=np.int32)
        _check(self._L.vx_get_collision_pairs(self.h, _ptr(p, C.c_int32), n.value, C.byref(n)))
        return p[:n.value]

    def collision_stats(self):
        n, a = C.c_int64(), C.c_double()
        _check(self._L.vx_collision_stats(self.h, C.byref(n), C.byref(a)))
        return n.value, a.value

    # -- adjoint form ------------------------------------------------------
    def rollout_forward(self, n_steps, checkpoint_every=100, stream=None):
        """Run n_steps from the current state keeping checkpoints; returns the
        per-body centre-of-mass x travel (float32 [n_bodies])."""
        loss = np.zeros(self.n_bodies, dtype=np.float32)
        _check(self._L.vx_rollout_forward(self.h, int(n_steps), int(checkpoint_every), _ptr(loss, C.c_float),
                                          _stream_ptr(stream)))
        return loss

    def rollout_backward(self, grad_logE=None, grad_phase=None, w_body=None, stream=None):
        """Gradients of sum_b w_b L_b for the last rollout into caller device
        buffers (torch CUDA float32 tensors [N], canonical order)."""
        w = None if w_body is None else np.ascontiguousarray(w_body, dtype=np.float32).reshape(self.n_bodies)
        _check(self._L.vx_rollout_backward(
            self.h, _ptr(w, C.c_float), None if grad_logE is None else grad_logE.data_ptr(),
            None if grad_phase is None else grad_phase.data_ptr(), _stream_ptr(stream)))
