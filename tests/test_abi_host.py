"""CPU checks of the C ABI: the library loads, exports every declared entry
point, and its host-side lattice logic (counts, stable timestep, region
selection, argument validation) agrees with the FP64 oracle."""
import os
import re

import numpy as np
import pytest

from oracle import Oracle
from paper_1212_2845_gb300 import scenes
from paper_1212_2845_gb300 import vx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "vx.h")).read()
    return set(re.findall(r"^VX_API [^\n(]*?\b(vx_\w+)\(", txt, flags=re.M))


def test_library_exports_every_declared_symbol():
    L = vx.lib()
    names = declared_symbols()
    assert len(names) >= 30
    for n in names:
        assert hasattr(L, n), n
    assert set(vx.SIGNATURES) == names
    assert L.vx_version().decode().startswith("voxsim-gb300")


SCENES = [
    lambda: scenes.cantilever(),
    lambda: scenes.hetero_block(dims=(12, 10, 8), seed=3),
    lambda: scenes.hollow_ball(R=12, t=3),
    lambda: scenes.population(n_bodies=7, seed=11, lo=2, hi=6),
    lambda: scenes.random_blob((7, 5, 4), seed=2, fill=0.6),
]


@pytest.mark.parametrize("mk", SCENES)
def test_plan_counts_match_oracle(mk):
    sc = mk()
    o = Oracle(sc, apply_scene=False)
    n, nb, ns = vx.plan_counts(sc)
    _, _, surf = o.topology()
    assert (n, nb, ns) == (o.N, o.n_bonds, int(surf.sum()))


@pytest.mark.parametrize("mk", SCENES)
def test_plan_dt_matches_oracle(mk):
    sc = mk()
    o = Oracle(sc)
    dt = vx.plan_dt(sc, log_E=sc.get("log_E"))
    ref = np.array([o.dt(b) for b in range(o.n_bodies)])
    assert np.allclose(dt, ref, rtol=1e-13, atol=0)


def test_plan_dt_with_per_voxel_stiffness():
    sc = scenes.design_population(n_bodies=3, n=4, seed=9)
    o = Oracle(sc)
    dt = vx.plan_dt(sc, log_E=sc["log_E"])
    assert np.allclose(dt, [o.dt(b) for b in range(3)], rtol=1e-13, atol=0)


def test_region_masks_match_oracle():
    rng = np.random.default_rng(3)
    sc = scenes.population(n_bodies=3, seed=5, lo=3, hi=9)
    o = Oracle(sc, apply_scene=False)
    for _ in range(40):
        b = int(rng.integers(0, 3))
        loc = scenes.f32(rng.uniform(0, 1, 3))
        size = scenes.f32(rng.uniform(0, 0.6, 3) * (rng.random(3) < 0.8))
        assert np.array_equal(vx.region_mask(sc, b, loc, size), o.region_mask(b, loc, size))


def test_appendix_a_regions():
    sc = scenes._base([(5, 10, 5)], np.ones(250, np.uint8), 1e-3, [scenes.material(1e7, 0.3)])
    ijk = scenes.canonical_coords(sc)
    assert np.array_equal(vx.region_mask(sc, 0, (0, 0, 0), (1, 0.01, 1)).astype(bool), ijk[:, 2] == 0)
    assert np.array_equal(vx.region_mask(sc, 0, (0, 0.99, 0), (1, 0.01, 1)).astype(bool), ijk[:, 2] == 9)


@pytest.mark.parametrize("bad", ["material", "empty", "dims", "E", "nu", "size"])
def test_invalid_descriptions_are_rejected(bad):
    sc = scenes.random_blob((4, 3, 2), seed=1)
    if bad == "material":
        sc["grid"] = sc["grid"].copy()
        sc["grid"][0] = 9
    elif bad == "empty":
        sc["grid"] = np.zeros_like(sc["grid"])
    elif bad == "dims":
        sc["dims"] = np.array([[0, 3, 2]], np.int32)
    elif bad == "E":
        sc["palette"] = sc["palette"].copy()
        sc["palette"][0, 0] = -1.0
    elif bad == "nu":
        sc["palette"] = sc["palette"].copy()
        sc["palette"][1, 1] = 0.5
    elif bad == "size":
        sc["voxel_size"] = 0.0
    with pytest.raises(vx.VxError) as e:
        vx.plan_counts(sc)
    assert e.value.code == -1
    assert vx.lib().vx_last_error().decode()


@pytest.mark.parametrize("mk", SCENES)
@pytest.mark.parametrize("tile_max", [128, 256, 512])
def test_tile_plan_invariants(mk, tile_max):
    sc = mk()
    n, nb, _ = vx.plan_counts(sc)
    t = vx.plan_tiles(sc, tile_max)
    assert t["n_tiles"] >= (n + tile_max - 1) // tile_max
    # every bond is evaluated by each tile that owns one of its voxels: once
    # inside a tile, twice when it crosses a tile border; crossing bonds are
    # bounded by the halo entries
    assert nb <= t["n_tile_bonds"] <= nb + t["n_halo"] * 6
    assert 0 < t["max_local"] <= 2 * tile_max
    assert 0 <= t["max_halo_bonds"] <= 2 * tile_max


@pytest.mark.parametrize("tile_max", [128, 256])
def test_sparse_lattice_halo_bond_lists_fit_the_staging(tile_max):
    """A sparse random lattice (many tile faces per voxel) still gets tiles
    whose halo-bond lists fit the kernels' staging of 2 tile_max entries."""
    sc = scenes.random_blob((24, 24, 24), seed=11, fill=0.55, n_mat=2)
    t = vx.plan_tiles(sc, tile_max)
    assert 0 < t["max_halo_bonds"] <= 2 * tile_max
    assert 0 < t["max_local"] <= 2 * tile_max
