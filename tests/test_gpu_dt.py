"""The stable timestep of a simulator (Sec 2.1.4): every body's largest
w^2 = k / m over its voxels' own contact springs and its bonds is reduced on
the device in FP32 (warp shuffle, shared memory across warps, one atomicMax
per CTA); the host takes dt = f / (2 pi sqrt(w^2)).

Error bound against the FP64 planner and the oracle: a candidate w^2 takes at
most six FP32 roundings (the bond's E_c l / min(m): 2 E_v E_u, E_v + E_u, the
quotient, the product with l, the rounded mass rho l^3, the last quotient),
so it is within 6 x 2^-24 = 3.6e-7 of its exact value, and so is the maximum
of the candidates; dt goes as (w^2)^(-1/2), half of that: 1.8e-7.  With
per-voxel moduli each of the two exp values adds at most 2 ulp (2.4e-7
relative) and the harmonic mean passes at most the sum of their relative
errors, so w^2 is within 6e-7 and dt within 3e-7."""
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


RTOL = 2e-7      # palette moduli (see the bound above)
RTOL_EXP = 3.5e-7  # per-voxel moduli


@pytest.mark.parametrize("name", sorted(SCENES))
def test_device_dt_matches_host_planner(name):
    sc = SCENES[name]()
    s = vx.Sim(sc)
    try:
        dt = s.dt()
        ref = vx.plan_dt(sc)
        assert np.all(dt > 0)
        assert np.allclose(dt, ref, rtol=RTOL, atol=0), np.max(np.abs(dt / ref - 1))
        for f in (0.25, 1.0):
            s.set_dt_factor(f)
            d2 = s.dt()
            assert np.allclose(d2, vx.plan_dt(sc, dt_factor=f), rtol=RTOL, atol=0)
            # the factor scales the reduced value and nothing else
            assert np.allclose(d2, dt * (float(np.float32(f)) / float(np.float32(sc["dt_factor"]))), rtol=1e-15, atol=0)
    finally:
        s.close()


def test_device_dt_matches_oracle_on_a_population():
    sc = scenes.population(n_bodies=64, seed=7, lo=2, hi=9)
    s = vx.Sim(sc)
    try:
        o = Oracle(sc)
        ref = np.array([o.dt(b) for b in range(o.n_bodies)])
        assert np.allclose(s.dt(), ref, rtol=RTOL, atol=0)
    finally:
        s.close()


def test_device_dt_takes_the_stiffest_term():
    """Two-voxel bodies whose maximum is, in turn, the bond (a stiff heavy
    voxel bonded to a soft light one: 2 E_soft / m_light beats both own
    springs) and a voxel's own spring (a stiff light voxel bonded to a soft
    heavy one): the reduction must pick the right candidate in each."""
    l = float(np.float32(1e-3))
    for (E1, r1), (E2, r2), expect in (((1e6, 8000.0), (1e5, 100.0), "bond"),
                                       ((1e7, 1000.0), (1e3, 8000.0), "own")):
        pal = [scenes.material(E1, rho=r1), scenes.material(E2, rho=r2)]
        sc = scenes._base([(2, 1, 1)], np.array([1, 2], dtype=np.uint8), l, pal)
        s = vx.Sim(sc)
        try:
            dt = s.dt()[0]
        finally:
            s.close()
        m1, m2 = r1 * l ** 3, r2 * l ** 3
        own = max(E1 * l / m1, E2 * l / m2)
        bond = 2 * E1 * E2 / (E1 + E2) * l / min(m1, m2)
        assert (bond > own) == (expect == "bond")
        w = np.sqrt(max(own, bond))
        assert dt == pytest.approx(float(np.float32(0.9)) / (2 * np.pi * w), rel=RTOL)


@pytest.mark.parametrize("name", ["hetero_block", "population_512"])
def test_device_dt_with_per_voxel_moduli(name):
    sc = SCENES[name]()
    le = _hetero_moduli(sc, seed=5)
    s = vx.Sim(sc)
    try:
        s.set_voxel_params(log_E=le)
        dt = s.dt()
        ref = vx.plan_dt(sc, log_E=le)
        assert np.allclose(dt, ref, rtol=RTOL_EXP, atol=0), np.max(np.abs(dt / ref - 1))
        sc2 = dict(sc, log_E=le)
        o = Oracle(sc2)
        for b in range(0, o.n_bodies, max(1, o.n_bodies // 16)):
            assert dt[b] == pytest.approx(o.dt(b), rel=RTOL_EXP, abs=0)
    finally:
        s.close()


def test_shared_world_takes_the_smallest_body_timestep():
    sc = scenes.population(n_bodies=40, seed=3, lo=2, hi=8)
    s = vx.Sim(sc)
    try:
        ref = s.dt()
        assert np.allclose(ref, vx.plan_dt(sc), rtol=RTOL, atol=0)
        s.set_environment(0.0, False, 2)
        assert np.array_equal(s.dt(), np.full_like(ref, ref.min()))
        s.set_environment(0.0, False, 1)
        assert np.array_equal(s.dt(), ref)
    finally:
        s.close()
