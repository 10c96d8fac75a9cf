"""FP64 reference simulator (test infrastructure only).

Loads ``oracle/_build/liboracle.so`` (compiled from ``voxel_oracle.cpp``) with
ctypes.  Only the tests, the package smoke check and the CPU-baseline leg of
the benchmark import this module; the CUDA library never does.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "voxel_oracle.cpp")
# VX_HOST_SANITIZE=1: built with AddressSanitizer and UndefinedBehaviorSanitizer
# into a separate file (load the runtimes with LD_PRELOAD)
_SANITIZE = os.environ.get("VX_HOST_SANITIZE") == "1"
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle_san.so" if _SANITIZE else "liboracle.so")
_lib = None

_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_U8 = C.POINTER(C.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain -O2, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        san = ["-g", "-fsanitize=address,undefined", "-fno-omit-frame-pointer"] if _SANITIZE else []
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", *san, "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        sig = {
            "orc_create": (_P, [C.c_int, _I32, _U8, C.c_double, _D, C.c_int, _D]),
            "orc_destroy": (None, [_P]),
            "orc_n_voxels": (C.c_int, [_P]),
            "orc_n_bonds": (C.c_int, [_P]),
            "orc_topology": (None, [_P, _I32, _I32, _U8]),
            "orc_bonds": (None, [_P, _I32]),
            "orc_set_params": (None, [_P, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int,
                                      C.c_double, C.c_long, C.c_double, C.c_double]),
            "orc_set_voxel_params": (None, [_P, _D, _D]),
            "orc_set_fixed": (None, [_P, _U8]),
            "orc_set_force": (None, [_P, _D]),
            "orc_region_mask": (C.c_int, [_P, C.c_int, _D, _D, _U8]),
            "orc_reset": (None, [_P, _D]),
            "orc_get_dt": (C.c_double, [_P, C.c_int]),
            "orc_reset_candidates": (None, [_P]),
            "orc_set_dt": (None, [_P, C.c_int, C.c_double]),
            "orc_get_step": (C.c_long, [_P]),
            "orc_step": (C.c_int, [_P, C.c_long]),
            "orc_get_state": (None, [_P, _D, _D, _D, _D, _U8]),
            "orc_set_state": (None, [_P, _D, _D, _D, _D, _U8]),
            "orc_set_step_counter": (None, [_P, C.c_long]),
            "orc_bond_force": (None, [_P, C.c_int, _D]),
            "orc_energy": (None, [_P, _D]),
            "orc_momentum": (None, [_P, _D]),
            "orc_candidate_pairs": (C.c_long, [_P, _I32, C.c_long]),
            "orc_n_rebuilds": (C.c_long, [_P]),
            "orc_event_signature": (C.c_uint64, [_P]),
            "orc_accumulator": (C.c_double, [_P, C.c_int]),
            "orc_pairs_from_offsets": (C.c_long, [_P, _D, _I32, C.c_long]),
            "orc_partners_of": (C.c_long, [_P, _D, C.c_int, _I32, C.c_long]),
            "orc_quant_params": (None, [C.c_double, _I32, C.POINTER(C.c_int64)]),
            "orc_rollout_jvp": (C.c_int, [_P, C.c_long, _D, _D, _D, _D]),
            "orc_linear_static": (C.c_int, [_P, _D, _D]),
            "orc_stiffness": (None, [_P, _D, _D]),
            "orc_set_collision_scheme": (None, [_P, C.c_int, C.c_int]),
            "orc_set_brute_search": (None, [_P, C.c_int]),
            "orc_set_material_actuation": (None, [_P, _D, _D, _D]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class Oracle:
    """Plain FP64 simulator built from a scene dictionary (see the package's scenes module)."""

    def __init__(self, sc, apply_scene=True):
        L = lib()
        self._L = L
        dims = np.ascontiguousarray(sc["dims"], dtype=np.int32).reshape(-1, 3)
        grid = np.ascontiguousarray(sc["grid"], dtype=np.uint8)
        pal = _f64(sc["palette"]).reshape(-1, 6)
        origin = _f64(sc["origin"]).reshape(-1, 3)
        self._keep = (dims, grid, pal, origin)
        self.h = L.orc_create(dims.shape[0], dims.ctypes.data_as(_I32), grid.ctypes.data_as(_U8),
                              float(sc["voxel_size"]), _dp(pal), pal.shape[0], _dp(origin))
        if not self.h:
            raise ValueError("oracle: invalid scene")
        self.n_bodies = dims.shape[0]
        self.n_materials = pal.shape[0]
        self.N = L.orc_n_voxels(self.h)
        self.n_bonds = L.orc_n_bonds(self.h)
        self.l = float(sc["voxel_size"])
        if apply_scene:
            self.apply(sc)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self._L.orc_destroy(h)
            self.h = None

    # -- configuration -----------------------------------------------------
    def apply(self, sc):
        self.set_params(sc)
        if sc.get("log_E") is not None or sc.get("phase") is not None:
            self.set_voxel_params(sc.get("log_E"), sc.get("phase"))
        if sc.get("fixed") is not None:
            self.set_fixed(sc["fixed"])
        if sc.get("force") is not None:
            self.set_force(sc["force"])
        self.reset(sc.get("v0"))

    def set_params(self, sc):
        self._L.orc_set_params(self.h, sc["zeta_bond"], sc["zeta_ground"], sc["zeta_collision"],
                               sc["gravity_z"], int(sc["floor"]), int(sc["collide"]),
                               sc["act_amplitude"], int(sc["act_period"]), sc["act_offset"],
                               sc["dt_factor"])
        ks = ("mat_act_amplitude", "mat_act_offset", "mat_act_phase")
        self.set_material_actuation(*[sc.get(k) for k in ks])

    def set_material_actuation(self, amplitude=None, offset=None, phase=None):
        """Per-material temperature signals on the common period (Sec 2.3);
        None: the global amplitude / offset, a zero phase shift."""
        arrs = [None if a is None else _f64(a) for a in (amplitude, offset, phase)]
        for a in arrs:
            if a is not None and a.size != self.n_materials:
                raise ValueError("one value per material expected")
        self._L.orc_set_material_actuation(self.h, *[_dp(a) for a in arrs])

    def set_voxel_params(self, log_E=None, phase=None):
        le = None if log_E is None else _f64(log_E)
        ph = None if phase is None else _f64(phase)
        self._L.orc_set_voxel_params(self.h, _dp(le), _dp(ph))

    def set_collision_scheme(self, all_voxels=False, every_step=False):
        """The paper's collision-scheme comparison: candidates among all
        voxels (not only surface voxels); rebuild every step (not on the
        horizon trigger)."""
        self._L.orc_set_collision_scheme(self.h, int(bool(all_voxels)), int(bool(every_step)))

    def set_brute_search(self, on=True):
        """Search candidate pairs by testing every pair of searched voxels
        (the definition) instead of the x-sorted sweep; both give one set."""
        self._L.orc_set_brute_search(self.h, int(bool(on)))

    def set_fixed(self, mask):
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        self._L.orc_set_fixed(self.h, m.ctypes.data_as(_U8))

    def set_force(self, F):
        f = _f64(F, (-1, 3))
        self._L.orc_set_force(self.h, _dp(f))

    def region_mask(self, body, loc, size):
        m = np.zeros(self.N, dtype=np.uint8)
        lo, sz = _f64(loc), _f64(size)
        self._L.orc_region_mask(self.h, body, _dp(lo), _dp(sz), m.ctypes.data_as(_U8))
        return m

    def reset(self, v0=None):
        v = None if v0 is None else _f64(v0)
        self._L.orc_reset(self.h, _dp(v))

    def reset_candidates(self):
        self._L.orc_reset_candidates(self.h)

    # -- stepping ----------------------------------------------------------
    def dt(self, body=0):
        return self._L.orc_get_dt(self.h, body)

    def set_dt(self, dt, body=None):
        bodies = range(self.n_bodies) if body is None else [body]
        for b in bodies:
            self._L.orc_set_dt(self.h, b, float(dt if np.isscalar(dt) else dt[b]))

    @property
    def step_count(self):
        return self._L.orc_get_step(self.h)

    def step(self, n=1):
        rc = self._L.orc_step(self.h, int(n))
        if rc != 0:
            raise FloatingPointError("oracle: non-finite state")

    # -- state -------------------------------------------------------------
    def state(self):
        N = self.N
        pos, quat = np.zeros((N, 3)), np.zeros((N, 4))
        vel, w = np.zeros((N, 3)), np.zeros((N, 3))
        st = np.zeros(N, dtype=np.uint8)
        self._L.orc_get_state(self.h, _dp(pos), _dp(quat), _dp(vel), _dp(w), st.ctypes.data_as(_U8))
        return dict(pos=pos, quat=quat, vel=vel, angvel=w, static=st)

    def set_state(self, pos=None, quat=None, vel=None, angvel=None, static=None):
        a = [None if x is None else _f64(x) for x in (pos, quat, vel, angvel)]
        st = None if static is None else np.ascontiguousarray(static, dtype=np.uint8)
        self._L.orc_set_state(self.h, *[_dp(x) for x in a], None if st is None else st.ctypes.data_as(_U8))

    def set_step_counter(self, n):
        self._L.orc_set_step_counter(self.h, int(n))

    def topology(self):
        N = self.N
        bijk = np.zeros((N, 4), dtype=np.int32)
        nbr = np.zeros((N, 6), dtype=np.int32)
        surf = np.zeros(N, dtype=np.uint8)
        self._L.orc_topology(self.h, bijk.ctypes.data_as(_I32), nbr.ctypes.data_as(_I32), surf.ctypes.data_as(_U8))
        return bijk, nbr, surf

    def bonds(self):
        b = np.zeros((self.n_bonds, 3), dtype=np.int32)
        self._L.orc_bonds(self.h, b.ctypes.data_as(_I32))
        return b

    def anchors(self, sc):
        bijk, _, _ = self.topology()
        org = np.asarray(sc["origin"], dtype=np.float64).reshape(-1, 3)[bijk[:, 0]]
        return org + (bijk[:, 1:].astype(np.float64) + 0.5) * self.l

    def bond_force(self, bond_id):
        out = np.zeros(12)
        self._L.orc_bond_force(self.h, int(bond_id), _dp(out))
        return out.reshape(4, 3)

    def energy(self):
        out = np.zeros(4)
        self._L.orc_energy(self.h, _dp(out))
        return out

    def momentum(self):
        out = np.zeros(6)
        self._L.orc_momentum(self.h, _dp(out))
        return out

    # -- collisions --------------------------------------------------------
    def candidate_pairs(self):
        n = self._L.orc_candidate_pairs(self.h, None, 0)
        p = np.zeros((max(n, 1), 2), dtype=np.int32)
        self._L.orc_candidate_pairs(self.h, p.ctypes.data_as(_I32), n)
        return p[:n]

    def event_signature(self):
        """Hash of every discrete decision since the last reset (floor contact
        and its stick/slip branch per voxel and step, voxel-voxel contacts):
        equal for two runs that take the same branches."""
        return self._L.orc_event_signature(self.h)

    def n_rebuilds(self):
        return self._L.orc_n_rebuilds(self.h)

    def accumulator(self, body=0):
        return self._L.orc_accumulator(self.h, body)

    def pairs_from_offsets(self, off):
        o = _f64(off, (-1, 3))
        n = self._L.orc_pairs_from_offsets(self.h, _dp(o), None, 0)
        p = np.zeros((max(n, 1), 2), dtype=np.int32)
        self._L.orc_pairs_from_offsets(self.h, _dp(o), p.ctypes.data_as(_I32), n)
        return p[:n]

    def partners_of(self, off, i):
        o = _f64(off, (-1, 3))
        n = self._L.orc_partners_of(self.h, _dp(o), int(i), None, 0)
        p = np.zeros(max(n, 1), dtype=np.int32)
        self._L.orc_partners_of(self.h, _dp(o), int(i), p.ctypes.data_as(_I32), n)
        return p[:n]

    @staticmethod
    def quant_params(l):
        K = C.c_int32()
        Q = C.c_int64()
        lib().orc_quant_params(float(l), C.byref(K), C.byref(Q))
        return K.value, Q.value

    # -- derivatives and statics -------------------------------------------
    def rollout_jvp(self, n_steps, dlogE=None, dphase=None):
        dl = None if dlogE is None else _f64(dlogE)
        dp = None if dphase is None else _f64(dphase)
        loss, dloss = C.c_double(), C.c_double()
        rc = self._L.orc_rollout_jvp(self.h, int(n_steps), _dp(dl), _dp(dp), C.byref(loss), C.byref(dloss))
        if rc != 0:
            raise FloatingPointError("oracle: non-finite state in dual rollout")
        return loss.value, dloss.value

    def stiffness(self):
        """Global stiffness K (6N x 6N, per voxel x, y, z, rx, ry, rz) of the
        lattice at rest assembled from the printed beam matrix, and the lumped
        mass of every DOF (m, m, m, I, I, I)."""
        n = 6 * self.N
        K = np.zeros((n, n))
        m = np.zeros(n)
        self._L.orc_stiffness(self.h, _dp(K), _dp(m))
        return K, m

    def linear_static(self, f):
        f = _f64(f, (-1, 6))
        u = np.zeros_like(f)
        if self._L.orc_linear_static(self.h, _dp(f), _dp(u)) != 0:
            raise np.linalg.LinAlgError("singular stiffness")
        return u
