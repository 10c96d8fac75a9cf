"""Seeded synthetic scenes (inputs only).

Every scene is plain data: lattice dimensions, a uint8 material grid
(x fastest, 0 = empty, k > 0 = palette entry k-1), a material palette, the
lattice dimension l, per-body origins, per-voxel actuation phases and the
simulation settings.  Nothing here evaluates the simulator's physics; both the
CUDA library and the FP64 checker consume these dictionaries.

The workloads follow the lattice sizes, material mixes and boundary conditions
of the paper's experiments (Section 3, Section 4.1) and of the five benchmark
configurations of this project (cantilever, heterogeneous actuated block,
hollow ball drop, batched population, design-gradient population).  Randomness
comes only from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import math

import numpy as np

# material tuple order used everywhere: (E [Pa], nu, rho [kg/m^3], cte [1/K], mu_s, mu_k)
MAT_FIELDS = ("E", "nu", "rho", "cte", "mu_s", "mu_k")


def material(E, nu=0.35, rho=1000.0, cte=0.0, mu_s=1.0, mu_k=0.5):
    return (float(E), float(nu), float(rho), float(cte), float(mu_s), float(mu_k))


def f32(x):
    """Round to the nearest float32 value, kept as float64: the CUDA library
    takes FP32 inputs, so scenes carry values both sides read identically."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def _base(dims, grid, l, palette, **kw):
    """Assemble a scene dict with the defaults used when a setting is not stated."""
    dims = np.asarray(dims, dtype=np.int32).reshape(-1, 3)
    sc = dict(
        dims=dims,
        grid=np.ascontiguousarray(grid, dtype=np.uint8).ravel(),
        voxel_size=float(f32(l)),
        palette=f32(np.asarray(palette, dtype=np.float64).reshape(-1, 6)),
        origin=np.zeros((dims.shape[0], 3), dtype=np.float64),
        phase=None,           # per-voxel actuation phase (canonical order) or None
        log_E=None,           # per-voxel log stiffness override or None
        fixed=None,           # per-voxel uint8 mask or None
        force=None,           # per-voxel external force [N][3] or None
        zeta_bond=1.0, zeta_ground=0.0, zeta_collision=1.0,
        gravity_z=0.0, floor=False, collide=False,
        act_amplitude=0.0, act_period=0, act_offset=0.0,
        # per-material temperature signals (amplitude, offset, phase shift per
        # palette entry) or None for the global signal
        mat_act_amplitude=None, mat_act_offset=None, mat_act_phase=None,
        v0=(0.0, 0.0, 0.0), dt_factor=0.9, steps=1,
        name="scene",
    )
    sc.update(kw)
    return normalize(sc)


FLOAT_KEYS = ("zeta_bond", "zeta_ground", "zeta_collision", "gravity_z", "act_amplitude", "act_offset",
              "dt_factor")


def normalize(sc):
    """Round every floating-point setting to a float32 value (see f32)."""
    for k in FLOAT_KEYS:
        sc[k] = float(f32(sc[k]))
    sc["v0"] = tuple(float(x) for x in f32(sc["v0"]))
    sc["origin"] = f32(sc["origin"])
    for k in ("phase", "log_E", "force", "mat_act_amplitude", "mat_act_offset", "mat_act_phase"):
        if sc.get(k) is not None:
            sc[k] = f32(sc[k])
    return sc


def n_occupied(sc):
    return int(np.count_nonzero(sc["grid"]))


def canonical_coords(sc):
    """(body, i, j, k) of every occupied site in canonical order.

    Canonical order: bodies in order, then sites x-fastest, then y, then z,
    skipping empty sites.  This is pure indexing, no physics.
    """
    out = []
    off = 0
    for b, (nx, ny, nz) in enumerate(sc["dims"]):
        n = int(nx) * int(ny) * int(nz)
        g = sc["grid"][off:off + n].reshape(int(nz), int(ny), int(nx))
        k, j, i = np.nonzero(g)          # C order over (z, y, x) == x fastest
        out.append(np.stack([np.full_like(i, b), i, j, k], axis=1))
        off += n
    return np.concatenate(out, axis=0).astype(np.int64)


# ---------------------------------------------------------------------------
# Configurations
# ---------------------------------------------------------------------------

def cantilever(n=(10, 10, 10), l=1e-3, E=1e6, rho=1000.0, nu=0.35, zeta_bond=0.1,
               steps=1000, gravity_z=-9.81):
    """Solid block cantilevered at its x=0 face, sagging under gravity (deterministic)."""
    nx, ny, nz = n
    grid = np.ones((nz, ny, nx), dtype=np.uint8)
    sc = _base([n], grid, l, [material(E, nu, rho)], zeta_bond=zeta_bond,
               gravity_z=gravity_z, steps=steps, name=f"cantilever_{nx}x{ny}x{nz}")
    ijk = canonical_coords(sc)
    sc["fixed"] = (ijk[:, 1] == 0).astype(np.uint8)
    return sc


def hetero_block(dims=(64, 64, 32), seed=2, steps=10000):
    """Heterogeneous actuated block on a floor.

    Sites: empty 10 %, soft 50 % (E 1 MPa, rho 1000, cte 0.01/K),
    stiff 40 % (E 1 GPa, rho 1200, cte 0).  Per-voxel phase U[0, 2 pi),
    sinusoidal temperature amplitude 20 K with a period of 2000 steps.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = dims
    u = rng.random((nz, ny, nx))
    grid = np.where(u < 0.10, 0, np.where(u < 0.60, 1, 2)).astype(np.uint8)
    pal = [material(1e6, 0.35, 1000.0, 0.01), material(1e9, 0.35, 1200.0, 0.0)]
    sc = _base([dims], grid, 1e-3, pal, gravity_z=-9.81, floor=True,
               act_amplitude=20.0, act_period=2000, steps=steps,
               name=f"hetero_block_{nx}x{ny}x{nz}")
    sc["phase"] = f32(rng.uniform(0.0, 2.0 * math.pi, size=n_occupied(sc)))
    return sc


def hollow_ball(R=100, t=8, drop=5, l=1e-3, v0=-2.0, steps=20000, collide=True):
    """Spherical shell: sites whose centre lies at distance r, R-t <= r < R
    (voxel units) from the sphere centre; lowest voxel's bottom face `drop`
    voxels above the floor; initial downward velocity v0."""
    n = 2 * R
    c2 = (2 * np.arange(n, dtype=np.int64) + 1 - n) ** 2      # (2 x)^2 of the site centres, exact
    s = c2[:, None, None] + c2[None, :, None] + c2[None, None, :]
    grid = ((s >= 4 * (R - t) ** 2) & (s < 4 * R * R)).astype(np.uint8)
    del s
    kmin = int(np.nonzero(grid.any(axis=(1, 2)))[0][0])
    sc = _base([(n, n, n)], grid, l, [material(0.5e6, 0.45, 1100.0)],
               gravity_z=-9.81, floor=True, collide=collide, v0=(0.0, 0.0, v0),
               steps=steps, name=f"hollow_ball_R{R}_t{t}")
    sc["origin"][0] = f32((0.0, 0.0, (drop - kmin) * l))
    return sc


def population(n_bodies=4096, seed=4, lo=4, hi=24, steps=20000):
    """Batched population of independent bodies with edges U{lo..hi} per axis.

    Sites: empty 20 %, soft 1 MPa 40 %, stiff 100 MPa 20 %, actuated soft
    (1 MPa, cte 0.01/K) 20 %; rho 1000; per-voxel phase U[0, 2 pi).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = rng.integers(lo, hi + 1, size=(n_bodies, 3)).astype(np.int32)
    grids = []
    for d in dims:
        u = rng.random((d[2], d[1], d[0]))
        g = np.where(u < 0.2, 0, np.where(u < 0.6, 1, np.where(u < 0.8, 2, 3)))
        grids.append(g.astype(np.uint8).ravel())
    pal = [material(1e6), material(1e8), material(1e6, cte=0.01)]
    sc = _base(dims, np.concatenate(grids), 1e-3, pal, gravity_z=-9.81, floor=True,
               act_amplitude=20.0, act_period=2000, steps=steps,
               name=f"population_{n_bodies}")
    sc["phase"] = f32(rng.uniform(0.0, 2.0 * math.pi, size=n_occupied(sc)))
    return sc


def design_population(n_bodies=1024, n=12, seed=5, steps=2000):
    """Design-gradient population: n^3 bodies with per-voxel log-stiffness
    U[ln 1e5, ln 1e8] and phase U[0, 2 pi); cte 0.01/K everywhere."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = np.tile(np.array([n, n, n], dtype=np.int32), (n_bodies, 1))
    grid = np.ones(n_bodies * n ** 3, dtype=np.uint8)
    sc = _base(dims, grid, 1e-3, [material(1e6, cte=0.01)], gravity_z=-9.81,
               floor=True, act_amplitude=20.0, act_period=2000, steps=steps,
               name=f"design_{n_bodies}x{n}^3")
    nv = n_bodies * n ** 3
    sc["log_E"] = f32(rng.uniform(math.log(1e5), math.log(1e8), size=nv))
    sc["phase"] = f32(rng.uniform(0.0, 2.0 * math.pi, size=nv))
    # bodies side by side along x, 2 voxels apart (independent worlds anyway)
    sc["origin"][:, 0] = f32(np.arange(n_bodies) * (n + 2) * 1e-3)
    return sc


def random_blob(dims=(6, 5, 4), seed=0, fill=0.8, n_mat=3):
    """Small random heterogeneous lattice for parity tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = dims
    u = rng.random((nz, ny, nx))
    m = rng.integers(1, n_mat + 1, size=(nz, ny, nx))
    grid = np.where(u < fill, m, 0).astype(np.uint8)
    pal = [material(1e6 * 10 ** (k % 3), 0.3 + 0.05 * k, 1000.0 + 100 * k, 0.01 * (k % 2),
                    0.8, 0.4) for k in range(n_mat)]
    sc = _base([dims], grid, 1e-3, pal, name=f"blob_{nx}x{ny}x{nz}_s{seed}")
    sc["phase"] = f32(rng.uniform(0.0, 2.0 * math.pi, size=n_occupied(sc)))
    return sc


def clapper(scale=1, period=4000, amplitude=10.0):
    """Synthetic stand-in for the paper's collision test geometry (its exact
    shape is not given): a fixed base slab and two upright arms, each a
    bilayer of an expanding (cte +0.02/K) and a contracting (cte -0.02/K)
    layer of 1 MPa voxels, the contracting layers facing each other.  The
    temperature swings +-amplitude, so the arms bend toward each other and
    apart again and their tips collide periodically (with the default 10 K
    the tips meet after ~700 steps and touch for ~1,000; the paper's 30 K,
    60 % strain, drives the arms through each other in this small-strain
    beam model).  scale multiplies every dimension (scale 1: 880 voxels)."""
    c = int(scale)
    nx, ny, nz = 20 * c, 4 * c, 23 * c
    g = np.zeros((nz, ny, nx), dtype=np.uint8)
    g[: 3 * c, :, :] = 1                                   # base (passive)
    arm = slice(3 * c, nz)
    g[arm, :, 0: 2 * c] = 2                                # left arm: outer expanding
    g[arm, :, 2 * c: 4 * c] = 3                            #           inner contracting
    g[arm, :, 16 * c: 18 * c] = 3                          # right arm: inner contracting
    g[arm, :, 18 * c: 20 * c] = 2                          #            outer expanding
    pal = [material(1e6), material(1e6, cte=0.02), material(1e6, cte=-0.02)]
    sc = _base([(nx, ny, nz)], g.ravel(), 1e-3, pal, collide=True, act_amplitude=amplitude,
               act_period=period, steps=period, name=f"clapper_x{c}")
    ijk = canonical_coords(sc)
    sc["fixed"] = (ijk[:, 3] == 0).astype(np.uint8)        # bottom layer of the base
    return sc


CONFIGS = {
    "cantilever": cantilever,
    "hetero_block": hetero_block,
    "hollow_ball": hollow_ball,
    "population": population,
    "design_population": design_population,
}
