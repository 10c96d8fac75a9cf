"""The stable timestep of a simulator (Sec 2.1.4): every body's largest
w^2 = k / m over its voxels' own contact springs and its bonds is reduced on
the device (warp shuffle, shared memory across warps, one atomicMax per CTA).
It must equal the host planner's FP64 loop to the bit for palette materials,
agree within the rounding of exp for per-voxel moduli, and match the FP64
oracle within 1e-13."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1212_2845_gb300 import scenes
from paper_1212_2845_gb300 import vx

pytestmark = pytest.mark.gpu


def _hetero_moduli(sc, seed):
    """Per-voxel log moduli spread over six decades, so that the maximum
    falls on a bond in some bodies and on a voxel's own spring in others."""
    rng = np.random.default_rng(seed)
    n = scenes.n_occupied(sc)
    return scenes.f32(rng.uniform(np.log(1e3), np.log(1e9), n))


SCENES = {
    "cantilever": lambda: scenes.cantilever(),
    "hetero_block": lambda: scenes.hetero_block(dims=(40, 36, 20), seed=3),
    "hollow_ball_R40": lambda: scenes.hollow_ball(R=40, t=8),
    "population_512": lambda: scenes.population(n_bodies=512, seed=11, lo=2, hi=20),
    "random_blob": lambda: scenes.random_blob((9, 7, 6), seed=2, fill=0.6, n_mat=4),
}


@pytest.mark.parametrize("name", sorted(SCENES))
def test_device_dt_equals_host_planner_bitwise(name):
    sc = SCENES[name]()
    s = vx.Sim(sc)
    try:
        dt = s.dt()
        ref = vx.plan_dt(sc)
        assert np.array_equal(dt, ref), np.max(np.abs(dt / ref - 1))
        for f in (0.25, 1.0):
            s.set_dt_factor(f)
            assert np.array_equal(s.dt(), vx.plan_dt(sc, dt_factor=f))
    finally:
        s.close()


def test_device_dt_matches_oracle_on_a_population():
    sc = scenes.population(n_bodies=64, seed=7, lo=2, hi=9)
    s = vx.Sim(sc)
    try:
        o = Oracle(sc)
        ref = np.array([o.dt(b) for b in range(o.n_bodies)])
        assert np.allclose(s.dt(), ref, rtol=1e-13, atol=0)
    finally:
        s.close()


@pytest.mark.parametrize("name", ["hetero_block", "population_512"])
def test_device_dt_with_per_voxel_moduli(name):
    sc = SCENES[name]()
    le = _hetero_moduli(sc, seed=5)
    s = vx.Sim(sc)
    try:
        s.set_voxel_params(log_E=le)
        dt = s.dt()
        ref = vx.plan_dt(sc, log_E=le)
        # the device's and the host's exp may differ in the last bit
        assert np.allclose(dt, ref, rtol=4e-16 * 8, atol=0), np.max(np.abs(dt / ref - 1))
        sc2 = dict(sc, log_E=le)
        o = Oracle(sc2)
        for b in range(0, o.n_bodies, max(1, o.n_bodies // 16)):
            assert dt[b] == pytest.approx(o.dt(b), rel=1e-13, abs=0)
    finally:
        s.close()


def test_shared_world_takes_the_smallest_body_timestep():
    sc = scenes.population(n_bodies=40, seed=3, lo=2, hi=8)
    s = vx.Sim(sc)
    try:
        ref = vx.plan_dt(sc)
        s.set_environment(0.0, False, 2)
        assert np.array_equal(s.dt(), np.full_like(ref, ref.min()))
        s.set_environment(0.0, False, 1)
        assert np.array_equal(s.dt(), ref)
    finally:
        s.close()
