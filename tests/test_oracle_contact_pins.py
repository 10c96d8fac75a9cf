"""Pins of the oracle's voxel-voxel contact law, both terms of the stable
timestep, the ground damper, and the candidate search.

The paper gives no force law for voxel-voxel contact (Sec 2.2.2 only says
collisions are damped and must keep the shell from being penetrated).  The
reading used here is a penalty spring k_c = 2 E_i E_j / (E_i + E_j) l on the
overlap of the two current half sizes, along the centre line, plus a normal
damper 2 zeta_c sqrt(m_min k_c) on the relative normal velocity, both only
while the voxels overlap.  These tests fix each part of it by closed forms of
mechanics that a wrong stiffness, mass, sign or damper would fail:

* the force on two overlapping free voxels after one step from rest
  (magnitude, direction, which voxel's mass takes it, unequal moduli);
* the rest overlap of a voxel lying on a fixed unbonded voxel under gravity:
  k_c delta = m g;
* the restitution and contact time of a head-on damped collision, against the
  damped linear oscillator of the relative coordinate (reduced mass mu,
  stiffness k_c, damper c = 2 zeta_c sqrt(m_min k_c)):
  y'' + c / mu y' + k_c / mu y = 0, so the effective damping ratio is
  zeta = c / (2 sqrt(mu k_c)) = zeta_c sqrt(m_min / mu) (sqrt(2) zeta_c for
  equal masses); a contact that starts and ends at zero overlap lasts
  pi / w_d and returns the relative speed times e = exp(-pi zeta / sqrt(1 - zeta^2)).
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_1212_2845_gb300 import scenes

L = float(np.float32(1e-3))   # the scenes round the voxel size to FP32


def pair_scene(axis, mats, zeta_c=0.0, gravity=0.0):
    """Two voxels of one body, 5 sites apart along `axis` (no bond between
    them, lattice Manhattan distance 5 > 3): voxel 0 of material 0, voxel 1 of
    material 1."""
    dims = [1, 1, 1]
    dims[axis] = 6
    grid = np.array([1, 0, 0, 0, 0, 2], np.uint8)
    pal = [scenes.material(E, 0.35, rho) for E, rho in mats]
    return scenes._base([dims], grid, L, pal, collide=True, zeta_collision=zeta_c, zeta_bond=0.0,
                        gravity_z=gravity)


def k_contact(E0, E1):
    return 2.0 * E0 * E1 / (E0 + E1) * L


@pytest.mark.parametrize("E0,E1,rho0,rho1", [(1e6, 1e6, 1000.0, 1000.0), (1e6, 5e6, 1000.0, 2500.0),
                                             (3e7, 2e5, 1500.0, 900.0)])
def test_overlap_force_is_the_harmonic_penalty_spring(E0, E1, rho0, rho1):
    """Two free voxels overlapping by delta along a skew direction n: after one
    step from rest each has taken the impulse -+ k_c delta n dt (no damping, no
    gravity), k_c the harmonic composite of the two moduli times l."""
    sc = pair_scene(0, [(E0, rho0), (E1, rho1)])
    o = Oracle(sc)
    sc_l = o.l
    n = np.array([1.0, 2.0, 2.0]) / 3.0
    delta = 0.1 * sc_l
    pos = o.state()["pos"].copy()
    pos[1] = pos[0] + (sc_l - delta) * n
    o.set_state(pos=pos)
    o.reset_candidates()
    assert [tuple(p) for p in o.candidate_pairs()] == [(0, 1)]
    dt = o.dt()
    o.step(1)
    v = o.state()["vel"]
    m0, m1 = rho0 * sc_l ** 3, rho1 * sc_l ** 3
    F = k_contact(E0, E1) * delta
    assert np.allclose(v[0], -F * dt / m0 * n, rtol=1e-12, atol=1e-15 * F * dt / m0)
    assert np.allclose(v[1], F * dt / m1 * n, rtol=1e-12, atol=1e-15 * F * dt / m1)


def test_contact_starts_at_the_sum_of_current_half_sizes():
    """The contact distance is the sum of the two current half sizes
    l (1 + alpha dT) / 2 (a voxel expanded by a temperature offset touches
    earlier): just outside it nothing happens, just inside the spring acts."""
    sc = pair_scene(0, [(1e6, 1000.0), (1e6, 1000.0)])
    sc["palette"][0, 3] = 0.01                 # voxel 0 expands: cte 0.01 / K
    sc["act_offset"] = 5.0                     # constant +5 K: h0 = l (1 + 0.05) / 2
    c = 0.5 * L * 1.05 + 0.5 * L
    for r, touching in ((c * (1 + 1e-9), False), (c * (1 - 1e-6), True)):
        o = Oracle(sc)
        pos = o.state()["pos"].copy()
        pos[1] = pos[0] + np.array([r, 0.0, 0.0])
        o.set_state(pos=pos)
        o.reset_candidates()
        o.step(1)
        v = o.state()["vel"]
        if touching:
            assert v[0, 0] < 0 < v[1, 0]
            dt = o.dt()
            assert v[1, 0] == pytest.approx(k_contact(1e6, 1e6) * (c - r) * dt / (1000 * L ** 3), rel=1e-6)
        else:
            assert np.all(v == 0.0)


@pytest.mark.parametrize("E0,E1,rho1", [(1e6, 1e6, 1000.0), (4e6, 1e6, 2000.0)])
def test_voxel_resting_on_a_fixed_unbonded_voxel(E0, E1, rho1):
    """A voxel lying on a fixed voxel it is not bonded to (same column, five
    sites apart in the lattice) settles at overlap m g / k_c."""
    sc = pair_scene(2, [(E0, 1000.0), (E1, rho1)], zeta_c=1.0, gravity=-9.81)
    o = Oracle(sc)
    o.set_fixed(np.array([1, 0], np.uint8))
    pos = o.state()["pos"].copy()
    pos[1] = pos[0] + np.array([0.0, 0.0, L])          # touching, at rest
    o.set_state(pos=pos)
    o.reset_candidates()
    prev = None
    for _ in range(200):
        o.step(2000)
        z = o.state()["pos"][1, 2]
        if prev is not None and abs(z - prev) < 1e-15:
            break
        prev = z
    overlap = L - (z - pos[0, 2])
    m = rho1 * L ** 3
    assert overlap == pytest.approx(m * 9.81 / k_contact(E0, E1), rel=1e-9)
    assert [tuple(p) for p in o.candidate_pairs()] == [(0, 1)]


@pytest.mark.parametrize("zeta_c,E0,E1,rho0,rho1", [(0.2, 1e6, 1e6, 1000.0, 1000.0),
                                                     (0.3, 1e6, 3e6, 1000.0, 3000.0),
                                                     (0.05, 2e6, 1e6, 2000.0, 1000.0)])
def test_head_on_collision_restitution_and_contact_time(zeta_c, E0, E1, rho0, rho1):
    """Head-on collision of two free voxels: the relative speed comes back
    multiplied by exp(-pi zeta / sqrt(1 - zeta^2)) after a contact of
    pi / w_d, with zeta = zeta_c sqrt(m_min / mu) and w_0^2 = k_c / mu (mu the
    reduced mass).  The timestep is 1/200 of the stable one so that the
    explicit integration resolves the contact (about 3,000 steps)."""
    sc = pair_scene(0, [(E0, rho0), (E1, rho1)], zeta_c=zeta_c)
    o = Oracle(sc)
    m0, m1 = rho0 * L ** 3, rho1 * L ** 3
    u = 0.05                                            # approach speed [m/s]
    pos = o.state()["pos"].copy()
    pos[1] = pos[0] + np.array([L, 0.0, 0.0])           # touching
    vel = np.array([[u * m1 / (m0 + m1), 0, 0], [-u * m0 / (m0 + m1), 0, 0]])
    o.set_state(pos=pos, vel=vel)
    o.reset_candidates()
    dt = o.dt() / 200
    o.set_dt(dt)
    in_contact = 0
    for _ in range(20000):
        o.step(1)
        s = o.state()
        r = s["pos"][1, 0] - s["pos"][0, 0]
        if r < L:
            in_contact += 1
        elif in_contact:
            break
    rel_out = s["vel"][1, 0] - s["vel"][0, 0]
    mu = m0 * m1 / (m0 + m1)
    kc = k_contact(E0, E1)
    zeta = zeta_c * math.sqrt(min(m0, m1) / mu)
    w0 = math.sqrt(kc / mu)
    wd = w0 * math.sqrt(1 - zeta * zeta)
    e = math.exp(-math.pi * zeta / math.sqrt(1 - zeta * zeta))
    assert rel_out / u == pytest.approx(e, rel=2e-3)
    assert in_contact * dt == pytest.approx(math.pi / wd, rel=2e-3)
    assert np.abs(s["vel"][0] * m0 + s["vel"][1] * m1).max() < 1e-12 * u * m0   # momentum


# ---------------------------------------------------------------------------
# stable timestep (Sec 2.1.4; reading: max over bonds and over each voxel's
# own floor / contact spring, k = E l on its own mass)
# ---------------------------------------------------------------------------

def test_stable_timestep_bond_term_dominates():
    """Stiff heavy voxel bonded to a softer light one: the bond's
    sqrt(E_c l / m_min) (harmonic E_c, the smaller mass) exceeds both voxels'
    own sqrt(E l / m) and sets dt."""
    o = Oracle(scenes._base([(2, 1, 1)], np.array([1, 2], np.uint8), L,
                            [scenes.material(1e7, rho=10000.0), scenes.material(1e6, rho=1000.0)]))
    Ec = 2 * 1e7 * 1e6 / (1e7 + 1e6)
    w_bond = math.sqrt(Ec * L / (1000.0 * L ** 3))
    assert w_bond > math.sqrt(1e7 * L / (10000.0 * L ** 3)) and w_bond > math.sqrt(1e6 * L / (1000.0 * L ** 3))
    assert o.dt() == pytest.approx(0.9 / (2 * math.pi * w_bond), rel=1e-13)


def test_stable_timestep_own_spring_term_dominates():
    """A very stiff voxel bonded only to a very soft one: the bond is soft
    (harmonic E_c ~ 2 E_soft), so the stiff voxel's own floor / contact spring
    sqrt(E l / m) sets dt."""
    o = Oracle(scenes._base([(2, 1, 1)], np.array([1, 2], np.uint8), L,
                            [scenes.material(1e8), scenes.material(1e5)]))
    Ec = 2 * 1e8 * 1e5 / (1e8 + 1e5)
    w_own = math.sqrt(1e8 * L / (1000.0 * L ** 3))
    assert w_own > 10 * math.sqrt(Ec * L / (1000.0 * L ** 3))
    assert o.dt() == pytest.approx(0.9 / (2 * math.pi * w_own), rel=1e-13)


def test_ground_damping_rotational_rate_equals_translational():
    """Damping to ground (Sec 2.1.5) on a lone voxel: the linear and angular
    velocities decay by the same factor 1 - 2 zeta_g sqrt(k_v / m) dt per step
    (the rotational damper on I = m l^2 / 6 with stiffness k_v l^2 / 6 has the
    translational rate), with nothing else acting."""
    zg = 0.4
    sc = scenes._base([(1, 1, 1)], np.ones(1, np.uint8), L, [scenes.material(2e6, rho=1300.0)], zeta_ground=zg)
    o = Oracle(sc)
    v0, w0 = np.array([[0.01, -0.02, 0.005]]), np.array([[3.0, 1.0, -2.0]])
    o.set_state(vel=v0, angvel=w0)
    n = 25
    o.step(n)
    s = o.state()
    rate = 2 * sc["zeta_ground"] * math.sqrt(2e6 * L / (1300.0 * L ** 3))   # zeta_g as rounded to FP32
    f = (1 - rate * o.dt()) ** n
    assert np.allclose(s["vel"], f * v0, rtol=1e-12, atol=0)
    assert np.allclose(s["angvel"], f * w0, rtol=1e-12, atol=0)


# ---------------------------------------------------------------------------
# candidate search: the x-sorted sweep finds exactly the brute-force set
# ---------------------------------------------------------------------------

def scrambled_state(o, seed, amp=0.45):
    rng = np.random.default_rng(seed)
    s = o.state()
    o.set_state(pos=s["pos"] + rng.uniform(-amp, amp, size=s["pos"].shape) * o.l)


@pytest.mark.parametrize("which", ["ball", "world", "clapper_all"])
def test_sweep_search_equals_brute_force(which):
    if which == "ball":
        sc = scenes.hollow_ball(R=9, t=3)
    elif which == "world":
        sc = scenes.population(n_bodies=6, seed=11, lo=3, hi=6)
        sc["collide"] = 2
    else:
        sc = scenes.clapper()
    for seed in (1, 2, 3):
        sets, from_off = [], []
        for brute in (True, False):
            o = Oracle(sc, apply_scene=False)
            if which == "clapper_all":
                o.set_collision_scheme(True, False)
            o.apply(sc)
            o.set_brute_search(brute)
            scrambled_state(o, seed)
            o.reset_candidates()
            sets.append({tuple(p) for p in o.candidate_pairs()})
            off = np.random.default_rng(seed + 10).uniform(-0.45, 0.45, size=(o.N, 3)) * o.l
            from_off.append([tuple(p) for p in o.pairs_from_offsets(off)])
        assert len(sets[0]) > 30 and len(from_off[0]) > 30
        assert sets[0] == sets[1]
        assert from_off[0] == from_off[1] == sorted(set(from_off[0]))
