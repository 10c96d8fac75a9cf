"""Pins of the FP64 oracle against values the paper prints and closed forms.

Each test checks the oracle against something other than itself: numbers the
paper prints (tests/golden/paper_values.json), textbook closed forms
(Euler-Bernoulli cantilever, harmonic series springs, symplectic-Euler free
fall), invariants (momentum, frame indifference, zero modes) and brute force.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import Oracle
from paper_1212_2845_gb300 import scenes

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def qexp(w):
    a = np.linalg.norm(w)
    if a == 0:
        return np.array([1.0, 0, 0, 0])
    return np.concatenate([[math.cos(a / 2)], math.sin(a / 2) * np.asarray(w) / a])


def qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def rotm(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def two_voxel(axis=0, mats=((1e6, 0.35, 1000.0),), grid=(1, 1), zeta_bond=0.0, **kw):
    dims = [1, 1, 1]
    dims[axis] = 2
    pal = [scenes.material(*m) for m in mats]
    return scenes._base([dims], np.array(grid, np.uint8), 1e-3, pal, zeta_bond=zeta_bond, **kw)


def printed_K(a1, a2, b1, b2, b3):
    """The 12x12 beam matrix exactly as printed in Sec 2.1.2 (upper triangle, symmetric)."""
    up = {(0, 0): a1, (0, 6): -a1,
          (1, 1): b1, (1, 5): b2, (1, 7): -b1, (1, 11): b2,
          (2, 2): b1, (2, 4): -b2, (2, 8): -b1, (2, 10): -b2,
          (3, 3): a2, (3, 9): -a2,
          (4, 4): 2 * b3, (4, 8): b2, (4, 10): b3,
          (5, 5): 2 * b3, (5, 7): -b2, (5, 11): b3,
          (6, 6): a1, (7, 7): b1, (7, 11): -b2, (8, 8): b1, (8, 10): b2,
          (9, 9): a2, (10, 10): 2 * b3, (11, 11): 2 * b3}
    K = np.zeros((12, 12))
    for (r, c), v in up.items():
        K[r, c] = v
        K[c, r] = v
    return K


def bond_jacobian(o, h=1e-9):
    """-(d force on voxels)/(d DOFs) of bond 0 by central differences, world frame."""
    s0 = o.state()
    J = np.zeros((12, 12))
    for d in range(12):
        cols = []
        for sgn in (1, -1):
            pos, quat = s0["pos"].copy(), s0["quat"].copy()
            node, w = divmod(d, 6)
            if w < 3:
                pos[node, w] += sgn * h
            else:
                r = np.zeros(3)
                r[w - 3] = sgn * h
                quat[node] = qexp(r)
            o.set_state(pos=pos, quat=quat)
            cols.append(o.bond_force(0).ravel())
        J[:, d] = -(cols[0] - cols[1]) / (2 * h)
    o.set_state(pos=s0["pos"], quat=s0["quat"])
    return J


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_bond_linearisation_equals_printed_matrix(axis):
    """Around the rest state, the co-rotational bond force linearises to the
    paper's [K] (Sec 2.1.2), for every lattice axis after the axis permutation."""
    E, nu, l = 1e6, 0.35, 1e-3
    o = Oracle(two_voxel(axis, mats=((E, nu, 1000.0),)))
    J = bond_jacobian(o)
    perm = [(i + axis) % 3 for i in range(3)]
    P = np.zeros((12, 12))
    for blk in range(4):
        for i in range(3):
            P[3 * blk + i, 3 * blk + perm[i]] = 1
    Kl = P @ J @ P.T
    G = E / (2 * (1 + nu))
    A, I, Jt = l * l, l ** 4 / 12, l ** 4 / 6
    K = printed_K(E * A / l, G * Jt / l, 12 * E * I / l ** 3, 6 * E * I / l ** 2, 2 * E * I / l)
    scale = np.sqrt(np.outer(np.diag(K), np.diag(K)))
    assert np.max(np.abs(Kl - K) / scale) < 1e-6


def test_printed_matrix_symmetric_psd_six_rigid_modes():
    o = Oracle(two_voxel(0))
    J = bond_jacobian(o)
    # mass-weight to make the spectrum scale-free
    D = np.diag(1 / np.sqrt(np.abs(np.diag(J))))
    S = D @ J @ D
    assert np.max(np.abs(S - S.T)) < 1e-6
    ev = np.linalg.eigvalsh(0.5 * (S + S.T))
    assert ev.min() > -1e-6
    assert np.sum(ev < 1e-6) == 6


def relax(o, probe, tol=1e-12, chunk=2000, max_chunks=400):
    prev = None
    for _ in range(max_chunks):
        o.step(chunk)
        cur = probe()
        if prev is not None and abs(cur - prev) <= tol * max(abs(cur), 1e-30):
            return cur
        prev = cur
    raise AssertionError("did not converge")


@pytest.mark.parametrize("E1,E2", [(1e6, 1e6), (1e6, 4e6), (2e7, 5e5)])
def test_single_bond_axial_series_springs(E1, E2):
    """Two voxels, voxel 1 fixed, axial force F on voxel 2: static extension
    F / (E_c l) with E_c the series (harmonic) composite of Sec 2.1.1."""
    F = 1e-3
    sc = two_voxel(0, mats=((E1, 0.35, 1000.0), (E2, 0.35, 1000.0)), grid=(1, 2),
                   zeta_bond=1.0, zeta_ground=0.05)
    sc["fixed"] = np.array([1, 0], np.uint8)
    sc["force"] = np.array([[0, 0, 0], [F, 0, 0]], float)
    o = Oracle(sc)
    x0 = o.state()["pos"][1, 0]
    ext = relax(o, lambda: o.state()["pos"][1, 0] - x0)
    Ec = 2 * E1 * E2 / (E1 + E2)
    assert ext == pytest.approx(F / (Ec * 1e-3), rel=1e-6)


def test_single_bond_lateral_cantilever():
    """Two-voxel cantilever, lateral tip force: F L^3 / (3 E I) with L = l (small load)."""
    E, F, l = 1e6, 1e-6, 1e-3
    sc = two_voxel(0, mats=((E, 0.35, 1000.0),), zeta_bond=1.0, zeta_ground=0.05)
    sc["fixed"] = np.array([1, 0], np.uint8)
    sc["force"] = np.array([[0, 0, 0], [0, 0, -F]], float)
    o = Oracle(sc)
    z0 = o.state()["pos"][1, 2]
    dz = relax(o, lambda: o.state()["pos"][1, 2] - z0)
    assert -dz == pytest.approx(F * l ** 3 / (3 * E * l ** 4 / 12), rel=1e-5)


def beam_scene(n, Ftot, zeta_ground):
    nx, ny, nz = n
    sc = scenes._base([n], np.ones(nx * ny * nz, np.uint8), 1e-3, [scenes.material(1e6, 0.35, 1000.0)],
                      zeta_bond=1.0, zeta_ground=zeta_ground)
    ijk = scenes.canonical_coords(sc)
    sc["fixed"] = (ijk[:, 1] == 0).astype(np.uint8)
    tip = ijk[:, 1] == nx - 1
    F = np.zeros((len(ijk), 3))
    F[tip, 2] = Ftot / tip.sum()
    sc["force"] = F
    return sc, tip


def test_thin_cantilever_matches_paper_and_closed_form():
    g = GOLD["thin_cantilever"]
    sc, tip = beam_scene(tuple(g["voxels"]), -g["tip_force_N"], 0.0025)
    o = Oracle(sc)
    E, l = g["E_Pa"], sc["voxel_size"]   # l: the paper's 1 mm as the scene's FP32 value
    assert l == pytest.approx(g["voxel_size_m"], rel=1e-7)
    L = (g["voxels"][0] - 1) * l  # fixed-voxel centre to tip-voxel centre
    closed = g["tip_force_N"] * L ** 3 / (3 * E * l ** 4 / 12)
    assert closed * 1e3 == pytest.approx(g["analytical_mm"], abs=5e-4)
    f6 = np.zeros((o.N, 6))
    f6[:, :3] = sc["force"]
    u = o.linear_static(f6)
    assert -u[tip, 2][0] == pytest.approx(closed, rel=1e-9)  # Hermite beams are nodally exact
    z0 = o.state()["pos"][tip, 2][0]
    dz = -relax(o, lambda: o.state()["pos"][tip, 2][0] - z0, tol=1e-10, chunk=5000)
    assert round(dz * 1e3, 3) == pytest.approx(g["mass_spring_mm"], abs=1e-9)
    assert dz == pytest.approx(closed, rel=5e-3)


def test_thin_cantilever_small_load_is_linear():
    g = GOLD["thin_cantilever"]
    sc, tip = beam_scene(tuple(g["voxels"]), -g["tip_force_N"] / 10, 0.0025)
    o = Oracle(sc)
    l = sc["voxel_size"]
    closed = g["tip_force_N"] / 10 * (19 * l) ** 3 / (3 * g["E_Pa"] * l ** 4 / 12)
    z0 = o.state()["pos"][tip, 2][0]
    dz = -relax(o, lambda: o.state()["pos"][tip, 2][0] - z0, tol=1e-10, chunk=5000)
    assert dz == pytest.approx(closed, rel=1e-3)


def test_thick_cantilever_soft_check():
    g = GOLD["thick_cantilever"]
    sc, tip = beam_scene(tuple(g["voxels"]), -g["tip_force_N"], 0.01)
    o = Oracle(sc)
    f6 = np.zeros((o.N, 6))
    f6[:, :3] = sc["force"]
    u = o.linear_static(f6)
    assert -u[tip, 2].min() * 1e3 == pytest.approx(g["direct_stiffness_mm"], abs=5e-4)
    z0 = o.state()["pos"][tip, 2]
    o.step(20000)
    dz = -(o.state()["pos"][tip, 2] - z0).mean()
    assert dz * 1e3 == pytest.approx(g["mass_spring_mm"], rel=0.03)
    assert dz < -u[tip, 2].mean()  # geometric stiffening: below the linear solve


def test_free_expansion_zero_stress_state():
    """Uniform CTE and temperature offset: every bond relaxes to l (1 + a dT)."""
    a, dT, n = 0.01, 7.0, 3
    sc = scenes._base([(n, n, n)], np.ones(n ** 3, np.uint8), 1e-3,
                      [scenes.material(1e6, 0.35, 1000.0, a)], zeta_bond=1.0, zeta_ground=0.02,
                      act_offset=dT)
    o = Oracle(sc)
    ext = lambda: np.ptp(o.state()["pos"][:, 0])
    e = relax(o, ext, tol=1e-13)
    l, a, dT = sc["voxel_size"], sc["palette"][0, 3], sc["act_offset"]
    assert e == pytest.approx((n - 1) * l * (1 + a * dT), rel=1e-9)
    s = o.state()
    assert np.abs(s["vel"]).max() < 1e-9


def test_rigid_motion_gives_zero_bond_force():
    rng = np.random.default_rng(0)
    for axis in range(3):
        o = Oracle(two_voxel(axis, zeta_bond=1.0))
        s = o.state()
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        Rm = rotm(q)
        c = s["pos"].mean(axis=0)
        pos = (s["pos"] - c) @ Rm.T + c + rng.normal(size=3) * 1e-3
        w = rng.normal(size=3) * 50.0
        V = rng.normal(size=3)
        vel = V + np.cross(w, pos - pos.mean(axis=0))
        o.set_state(pos=pos, quat=np.tile(q, (2, 1)), vel=vel, angvel=np.tile(w, (2, 1)))
        f = o.bond_force(0)
        assert np.abs(f[[0, 2]]).max() < 1e-12 * 1e6 * 1e-3 * 1e-3
        assert np.abs(f[[1, 3]]).max() < 1e-15


def test_axis_permutation_equivariance():
    """A local deformation applied along x, y and z bonds gives the same local forces."""
    rng = np.random.default_rng(1)
    dp = rng.normal(size=3) * 1e-5
    th = rng.normal(size=3) * 1e-2
    out = []
    for axis in range(3):
        o = Oracle(two_voxel(axis))
        s = o.state()
        pos = s["pos"].copy()
        gl = np.zeros(3)
        for i in range(3):
            gl[(i + axis) % 3] = dp[i]
        pos[1] += gl
        tw = np.zeros(3)
        for i in range(3):
            tw[(i + axis) % 3] = th[i]
        quat = s["quat"].copy()
        quat[1] = qexp(tw)
        o.set_state(pos=pos, quat=quat)
        f = o.bond_force(0)
        out.append(np.stack([[v[(i + axis) % 3] for i in range(3)] for v in f]))
    assert np.allclose(out[0], out[1], rtol=1e-12, atol=1e-18)
    assert np.allclose(out[0], out[2], rtol=1e-12, atol=1e-18)


def free_block(seed=3, n=(4, 3, 3), zeta=0.0):
    sc = scenes.random_blob(n, seed=seed, fill=1.0)
    sc.update(zeta_bond=zeta, zeta_ground=0.0, gravity_z=0.0)
    return sc


def test_momentum_conserved_and_energy_bounded():
    sc = free_block()
    o = Oracle(sc)
    rng = np.random.default_rng(2)
    s = o.state()
    o.set_state(vel=rng.normal(size=(o.N, 3)) * 1e-3, angvel=rng.normal(size=(o.N, 3)) * 1.0,
                pos=s["pos"] + rng.normal(size=(o.N, 3)) * 1e-7)
    P0 = o.momentum()[:3]
    e0 = o.energy()[:3].sum()
    es = []
    for _ in range(50):
        o.step(200)
        es.append(o.energy()[:3].sum())
    P1 = o.momentum()[:3]
    mass_scale = np.abs(P0).max() + 1e-3 * 1e-6 * o.N
    assert np.abs(P1 - P0).max() < 1e-12 * mass_scale
    es = np.array(es)
    # Symplectic Euler keeps a shadow energy: the true energy oscillates by
    # O(omega dt) (omega dt reaches ~0.7 for the stiffest rotational modes)
    # but does not drift.  Bounds set empirically in FP64.
    assert np.abs(es - e0).max() / e0 < 0.1
    assert abs(es[-25:].mean() - es[:25].mean()) / e0 < 1e-2


def test_bond_damping_dissipates_and_conserves_momentum():
    """Bond damping forces are equal and opposite (momentum exact) and remove
    the internal vibration energy that the undamped lattice keeps."""
    rng = np.random.default_rng(4)
    v = rng.normal(size=(36, 3)) * 1e-3
    ends = []
    for zeta in (0.0, 1.0):
        o = Oracle(free_block(zeta=zeta))
        o.set_state(vel=v[:o.N])
        P0 = o.momentum()[:3]
        e0 = o.energy()[:3].sum()
        o.step(3000)
        assert np.abs(o.momentum()[:3] - P0).max() < 1e-15
        ends.append(o.energy()[:3].sum() / e0)
    # the damped lattice keeps only (roughly) its rigid-body motion
    assert ends[0] > 0.5
    assert 0.0 < ends[1] < 0.1 * ends[0]


def test_stable_timestep_closed_form():
    """dt = f / (2 pi sqrt(k / m)) with k = E l, m = rho l^3 (Sec 2.1.4)."""
    o = Oracle(scenes.cantilever())
    assert o.dt() == pytest.approx(0.9 / (2 * math.pi * math.sqrt(1e6 * 1e-3 / (1000 * 1e-9))), rel=1e-14)


def test_free_fall_symplectic_euler():
    """One voxel under gravity: v_n = n g dt, z_n = z_0 + g dt^2 n (n + 1) / 2."""
    sc = scenes._base([(1, 1, 1)], np.ones(1, np.uint8), 1e-3, [scenes.material(1e6)], gravity_z=-9.81)
    o = Oracle(sc)
    dt, g = o.dt(), sc["gravity_z"]
    z0 = o.state()["pos"][0, 2]
    o.step(100)
    s = o.state()
    assert s["vel"][0, 2] == pytest.approx(g * 100 * dt, rel=1e-12)
    assert s["pos"][0, 2] - z0 == pytest.approx(g * dt * dt * 100 * 101 / 2, rel=1e-10)


def test_floor_rest_penetration():
    """A voxel resting on the floor sinks until k_v pen = m g (k_v = E l)."""
    sc = scenes._base([(1, 1, 1)], np.ones(1, np.uint8), 1e-3, [scenes.material(1e6)],
                      gravity_z=-9.81, floor=True, zeta_collision=1.0)
    o = Oracle(sc)
    z = relax(o, lambda: o.state()["pos"][0, 2], tol=1e-13)
    l = sc["voxel_size"]
    pen = 0.5 * l - z
    assert pen == pytest.approx(1000 * l ** 3 * -sc["gravity_z"] / (1e6 * l), rel=1e-9)


def test_static_friction_threshold_and_sliding_deceleration():
    """Coulomb model of Sec 2.2.1: no motion while |F_l| <= mu_s F_n; once it
    slides with the push removed, it decelerates at mu_d g and halts."""
    def scene(Fx):
        sc = scenes._base([(1, 1, 1)], np.ones(1, np.uint8), 1e-3,
                          [scenes.material(1e6, mu_s=0.8, mu_k=0.4)],
                          gravity_z=-9.81, floor=True, zeta_collision=1.0)
        sc["force"] = np.array([[Fx, 0.0, 0.0]])
        return sc
    sc0 = scene(0.0)
    mu_s, mu_k = sc0["palette"][0, 4], sc0["palette"][0, 5]
    m, g = 1000.0 * sc0["voxel_size"] ** 3, -sc0["gravity_z"]
    # settle first without lateral load, then push
    for frac, moves in [(0.98, False), (1.02, True)]:
        o = Oracle(scene(0.0))
        o.step(3000)
        x0 = o.state()["pos"][0, 0]
        o.set_force(np.array([[frac * mu_s * m * g, 0, 0]]))
        o.step(2000)
        dx = o.state()["pos"][0, 0] - x0
        assert (abs(dx) > 1e-9) == moves
    # sliding with no push: deceleration mu_k g (F_n = m g at rest on the floor)
    o = Oracle(scene(0.0))
    o.step(3000)
    s = o.state()
    v0 = 0.05
    o.set_state(vel=np.array([[v0, 0.0, s["vel"][0, 2]]]), static=np.array([0], np.uint8))
    dt = o.dt()
    o.step(200)
    v1 = o.state()["vel"][0, 0]
    assert (v0 - v1) / (200 * dt) == pytest.approx(mu_k * g, rel=2e-3)
    o.step(int(v1 / (mu_k * g * dt)) + 50)
    s = o.state()
    assert s["vel"][0, 0] == 0.0 and s["static"][0] == 1


def test_region_selection_appendix_a():
    g = GOLD["appendix_a_regions"]
    nx, ny, nz = g["workspace"]
    sc = scenes._base([(nx, ny, nz)], np.ones(nx * ny * nz, np.uint8), 1e-3, [scenes.material(1e7, 0.3)])
    o = Oracle(sc)
    ijk = scenes.canonical_coords(sc)
    m = o.region_mask(0, g["fixed_loc"], g["fixed_size"])
    assert np.array_equal(m.astype(bool), ijk[:, 2] == g["fixed_layer_y"])
    m = o.region_mask(0, g["forced_loc"], g["forced_size"])
    assert np.array_equal(m.astype(bool), ijk[:, 2] == g["forced_layer_y"])


# ---------------------------------------------------------------------------
# collision candidates (Sec 2.2.2)
# ---------------------------------------------------------------------------

def test_candidates_empty_for_undeformed_lattice():
    """On the undeformed lattice every site pair closer than 2 voxels has
    Manhattan distance <= 3, so the horizon list is empty."""
    sc = scenes.random_blob((6, 5, 4), seed=5, fill=0.7)
    sc["collide"] = True
    o = Oracle(sc)
    assert len(o.candidate_pairs()) == 0
    assert len(o.pairs_from_offsets(np.zeros((o.N, 3)))) == 0


def test_candidates_folded_line():
    """Line of voxels 0..7 along x; move voxel 7 next to voxel 0 (a fold)."""
    l = 1e-3
    sc = scenes._base([(8, 1, 1)], np.ones(8, np.uint8), l, [scenes.material(1e6)], collide=True)
    o = Oracle(sc)
    off = np.zeros((8, 3))
    # voxel 7 moved to 1.5 l above voxel 0: only (0,7) and (1,7) are within 2 l?
    # voxel 7 rest centre is 7 l along x; put it at x = 0.5 l, z = +1.5 l from voxel 0
    off[7] = [-7 * l + 0.5 * l, 0.0, 1.5 * l]
    pairs = {tuple(p) for p in o.pairs_from_offsets(off)}
    # distances from voxel 7 (at (0.5, 0, 1.5)) to voxel i at (i, 0, 0): sqrt((i-0.5)^2 + 2.25)
    expect = {(i, 7) for i in range(8) if abs(i - 7) > 3 and (i - 0.5) ** 2 + 2.25 < 4.0}
    assert pairs == expect == {(0, 7), (1, 7)}


def test_candidate_distance_threshold_is_strict():
    l = 1e-3
    K, Q = Oracle.quant_params(l)
    sc = scenes._base([(5, 1, 1)], np.array([1, 0, 0, 0, 1], np.uint8), l, [scenes.material(1e6)],
                      collide=True)
    o = Oracle(sc)
    # rest distance 4 l; move voxel 1 by -2 l + delta (in quantisation units)
    for dq, inside in [(0, False), (1, True), (-1, False)]:
        off = np.zeros((2, 3))
        # quantised x difference = 4Q + rint(o * 2^K) = 2Q - dq  -> o = (-2Q - dq) / 2^K
        off[1, 0] = (-2 * Q - dq) / 2.0 ** K
        assert (len(o.pairs_from_offsets(off)) == 1) == inside


def test_contact_bounce_conserves_momentum_and_energy():
    """Two unbonded voxels of one body approach head-on: the penalty contact is
    repulsive, exactly antisymmetric (momentum) and, undamped, elastic."""
    l = 1e-3
    sc = scenes._base([(6, 1, 1)], np.array([1, 0, 0, 0, 0, 1], np.uint8), l, [scenes.material(1e6)],
                      collide=True, zeta_collision=0.0, zeta_bond=0.0)
    o = Oracle(sc)
    s = o.state()
    pos = s["pos"].copy()
    pos[1, 0] = pos[0, 0] + 1.9 * l      # inside the 2-voxel horizon, not touching
    o.set_state(pos=pos, vel=np.array([[0.5, 0, 0], [-0.5, 0, 0]]))
    o.reset_candidates()
    assert [tuple(p) for p in o.candidate_pairs()] == [(0, 1)]
    e0 = o.energy()[0]
    o.step(4000)
    s = o.state()
    assert np.abs(s["vel"].sum(axis=0)).max() < 1e-15
    assert s["vel"][0, 0] < 0 < s["vel"][1, 0]            # bounced apart
    assert o.energy()[0] == pytest.approx(e0, rel=1e-2)   # elastic without damping


def test_forward_mode_matches_central_differences():
    """The dual-number rollout derivative equals central finite differences of
    the FP64 rollout (loss = mean x displacement of the body)."""
    sc = scenes.random_blob((4, 3, 3), seed=7, fill=0.9)
    sc.update(gravity_z=-9.81, floor=True, act_amplitude=20.0, act_period=40, zeta_bond=1.0)
    o = Oracle(sc)
    N = o.N
    rng = np.random.default_rng(8)
    logE = np.log(sc["palette"][0, 0]) + rng.uniform(-1, 1, N)
    base_phase = sc["phase"]
    dlog = rng.normal(size=N)
    dph = rng.normal(size=N)
    steps = 60

    def run(eps_l, eps_p):
        q = Oracle(sc)
        q.set_voxel_params(logE + eps_l * dlog, base_phase + eps_p * dph)
        dt0 = Oracle(sc)
        dt0.set_voxel_params(logE, base_phase)
        q.set_dt(dt0.dt())          # timestep frozen at the unperturbed value
        q.reset(sc["v0"])
        return q.rollout_jvp(steps)[0]

    o.set_voxel_params(logE, base_phase)
    o.reset(sc["v0"])
    L, dL = o.rollout_jvp(steps, dlog, dph)
    h = 1e-6
    fd = (run(h, h) - run(-h, -h)) / (2 * h)
    assert L == pytest.approx(run(0, 0), rel=1e-12)
    assert dL == pytest.approx(fd, rel=1e-5, abs=1e-12 * abs(L))


# ---------------------------------------------------------------------------
# dynamics: modal frequencies of the thin cantilever (validation section)
# ---------------------------------------------------------------------------

def thin_cantilever_scene(zeta=0.0):
    sc = scenes._base([[20, 1, 1]], np.ones(20, np.uint8), 1e-3, [scenes.material(1e6, 0.35, 1000.0)],
                      zeta_bond=zeta)
    sc["fixed"] = (np.arange(20) == 0).astype(np.uint8)
    return sc


def bending_frequencies(o, sc):
    """Frequencies [Hz] of the linearised lattice M u'' = -K u (printed [K],
    lumped m and I) whose mode moves the tip voxel in z."""
    import scipy.linalg as sla
    K, m = o.stiffness()
    free = np.repeat(sc["fixed"] == 0, 6)
    w2, phi = sla.eigh(K[np.ix_(free, free)], np.diag(m[free]))
    f = np.sqrt(np.maximum(w2, 0.0)) / (2 * np.pi)
    tip_z = 6 * 18 + 2                      # voxel 19 is the 19th free voxel
    return np.array([f[k] for k in range(len(f)) if abs(phi[tip_z, k]) > 1e-6 * np.abs(phi[tip_z]).max()])


def spectrum_peaks(z, dt, guesses):
    """Peak frequencies of z(t) near each guess (Hann window, parabolic
    interpolation of the log magnitude around the largest bin)."""
    z = np.asarray(z) - np.mean(z)
    spec = np.abs(np.fft.rfft(z * np.hanning(len(z))))
    freqs = np.fft.rfftfreq(len(z), dt)
    out = []
    for g in guesses:
        lo, hi = np.searchsorted(freqs, 0.85 * g), np.searchsorted(freqs, 1.15 * g)
        k = lo + int(np.argmax(spec[lo:hi]))
        a, b, c = np.log(spec[k - 1:k + 2])
        out.append(freqs[k] + 0.5 * (a - c) / (a - 2 * b + c) * (freqs[1] - freqs[0]))
    return np.array(out)


def test_cantilever_modes_match_beam_theory():
    """The linearised lattice of a 20x1x1, 1 mm, 1 MPa cantilever (voxel 0
    fixed) has the Euler-Bernoulli bending frequencies
    K_n / (2 pi) sqrt(E I / (m L^4)), K_n = 3.516, 22.03, 61.70 (Volterra's
    constants), for the free length L = 19.5 mm from the clamped voxel's
    centre to the tip face: the discretisation error grows with the mode."""
    sc = thin_cantilever_scene()
    o = Oracle(sc)
    f = np.unique(np.round(bending_frequencies(o, sc), 6))[:3]
    EI = 1e6 * (1e-3) ** 4 / 12.0
    mbar = 1000.0 * (1e-3) ** 2
    L = 19.5e-3
    beam = np.array([Kn / (2 * np.pi) * np.sqrt(EI / (mbar * L ** 4)) for Kn in (3.516, 22.03, 61.70)])
    assert np.all(np.abs(f / beam - 1.0) <= [0.002, 0.01, 0.02]), (f, beam)


def test_cantilever_impulse_response_rings_at_the_lattice_frequencies():
    """An impulse at the tip (no damping) rings at the linearised lattice's
    bending frequencies: the explicit step reproduces M u'' = -K u."""
    sc = thin_cantilever_scene()
    o = Oracle(sc)
    f_lin = np.unique(np.round(bending_frequencies(o, sc), 6))[:3]
    vel = np.zeros((20, 3))
    vel[19, 2] = 1e-3
    o.set_state(vel=vel)
    dt = o.dt()
    every, n = 10, 32768
    z = np.empty(n)
    for i in range(n):
        o.step(every)
        z[i] = o.state()["pos"][19, 2]
    peaks = spectrum_peaks(z, every * dt, f_lin)
    assert np.all(np.abs(peaks / f_lin - 1.0) <= 2e-3), (peaks, f_lin)


# ---------------------------------------------------------------------------
# shared world (several bodies colliding with each other)
# ---------------------------------------------------------------------------

def two_cubes(gap_voxels=3, v=0.2, n=3):
    """Two n^3 cubes of 1 mm voxels on the x axis, `gap_voxels` empty voxels
    apart, approaching head-on at +-v; one shared world (collide = 2)."""
    l = 1e-3
    sc = scenes._base([(n, n, n), (n, n, n)], np.ones(2 * n ** 3, np.uint8), l, [scenes.material(1e6)],
                      collide=2, zeta_collision=0.0, zeta_bond=1.0)
    sc["origin"] = scenes.f32([[0.0, 0.0, 0.0], [(n + gap_voxels) * l, 0.0, 0.0]])
    return sc, v


def test_shared_world_bodies_collide_and_bounce():
    """Voxels of different bodies are candidates only in the shared world,
    the contact pairs are exactly antisymmetric (total momentum constant to
    rounding), the bodies bounce apart, and both bodies run on the smaller
    timestep."""
    sc, v = two_cubes()
    o = Oracle(sc)
    assert o.dt(0) == o.dt(1)
    N = o.N
    vel = np.zeros((N, 3))
    vel[: N // 2, 0] = v
    vel[N // 2:, 0] = -v
    o.set_state(vel=vel)
    o.reset_candidates()
    assert len(o.candidate_pairs()) == 0                 # 3 voxels apart: outside the horizon
    p0 = o.momentum()[:3]
    seen_cross = 0
    for _ in range(40):
        o.step(100)
        pairs = o.candidate_pairs()
        seen_cross += sum(1 for i, j in pairs if (i < N // 2) != (j < N // 2))
    s = o.state()
    assert seen_cross > 0
    assert np.abs(o.momentum()[:3] - p0).max() <= 1e-12 * v * o.N * 1e-6
    m = 1000.0 * 1e-9
    va = s["vel"][: N // 2, 0].mean()
    vb = s["vel"][N // 2:, 0].mean()
    assert va < 0 < vb                                     # bounced apart


def test_separate_worlds_never_pair_bodies():
    sc, v = two_cubes(gap_voxels=0)                         # touching faces
    sc["collide"] = True                                    # self-collision only
    o = Oracle(sc)
    o.reset_candidates()
    N = o.N
    assert all((i < N // 2) == (j < N // 2) for i, j in o.candidate_pairs())
    sc["collide"] = 2
    o = Oracle(sc)
    o.reset_candidates()
    cross = [(i, j) for i, j in o.candidate_pairs() if (i < N // 2) != (j < N // 2)]
    # face-to-face neighbours across the two bodies (3 x 3 facing voxels, each
    # within 2 voxels of its facing partner and its in-plane neighbours)
    assert len(cross) > 0 and all(i < N // 2 <= j for i, j in cross)


def test_collision_schemes_give_the_same_trajectory():
    """The horizon rule is conservative and only overlapping candidates exert
    forces (summed in ascending partner order), so all-voxel / surface-voxel
    candidates and every-step / horizon rebuilds give the same trajectory
    bit for bit through the clapper's contact; the candidate sets differ
    only by pairs that are not overlapping."""
    sc = scenes.clapper()
    finals, npairs = [], []
    for all_voxels, every in ((False, False), (True, True), (False, True), (True, False)):
        o = Oracle(sc, apply_scene=False)
        o.set_collision_scheme(all_voxels, every)
        o.apply(sc)
        o.step(1200)
        finals.append(o.state())
        npairs.append(len(o.candidate_pairs()))
    for s in finals[1:]:
        for k in ("pos", "quat", "vel", "angvel"):
            assert np.array_equal(s[k], finals[0][k]), k
    assert npairs[0] > 0


# ---------------------------------------------------------------------------
# several temperature signals (Sec 2.3: separately controlled temperatures
# driving different materials)
# ---------------------------------------------------------------------------

def test_material_offsets_rest_length_closed_form():
    """Two materials held at their own offsets (no oscillation): the bond
    between them relaxes to l (1 + (a1 dT1 + a2 dT2) / 2), whatever the two
    stiffnesses (no force at the rest length)."""
    a1, a2, T1, T2 = 0.01, -0.004, 6.0, 9.0
    sc = two_voxel(0, mats=((1e6, 0.35, 1000.0, a1), (4e6, 0.3, 1500.0, a2)), grid=(1, 2), zeta_bond=1.0,
                   zeta_ground=0.02, act_offset=3.0)
    sc["mat_act_offset"] = scenes.f32([T1, T2])
    o = Oracle(sc)
    e = relax(o, lambda: o.state()["pos"][1, 0] - o.state()["pos"][0, 0], tol=1e-14)
    l = sc["voxel_size"]
    a1, a2 = sc["palette"][0, 3], sc["palette"][1, 3]
    T1, T2 = sc["mat_act_offset"]
    assert e == pytest.approx(l * (1 + 0.5 * (a1 * T1 + a2 * T2)), rel=1e-10)
    # the global offset alone would give a different length
    assert abs(e - l * (1 + 0.5 * (a1 + a2) * sc["act_offset"])) > 1e-3 * l * abs(a1 * T1)


def two_bodies_two_materials():
    pal = [scenes.material(1e6, 0.35, 1000.0, 0.01), scenes.material(3e6, 0.3, 1200.0, -0.02)]
    dims = [(4, 3, 2), (3, 3, 3)]
    grid = np.concatenate([np.full(24, 1, np.uint8), np.full(27, 2, np.uint8)])
    sc = scenes._base(dims, grid, 1e-3, pal, gravity_z=-9.81, floor=True, zeta_ground=0.05,
                      act_amplitude=5.0, act_period=300, act_offset=1.0)
    sc["origin"] = scenes.f32([[0.0, 0.0, 0.0], [0.01, 0.0, 0.0]])
    return sc


def test_material_signals_drive_each_material_independently():
    """Two bodies of one material each, every material on its own amplitude,
    offset and phase shift: each body follows, bit for bit, the same body
    simulated alone under the single global signal with those values (the
    phase shift carried by every voxel's own phase)."""
    sc = two_bodies_two_materials()
    amp, off, ph = scenes.f32([12.0, 4.0]), scenes.f32([-2.0, 3.0]), scenes.f32([0.0, 1.3])
    sc.update(mat_act_amplitude=amp, mat_act_offset=off, mat_act_phase=ph)
    o = Oracle(sc)
    o.step(900)
    both = o.state()
    n0 = 24
    for b, sl in ((0, slice(0, n0)), (1, slice(n0, None))):
        alone = scenes._base([sc["dims"][b]], sc["grid"][sl] * 0 + 1, 1e-3, [sc["palette"][b]],
                             gravity_z=-9.81, floor=True, zeta_ground=0.05, act_amplitude=float(amp[b]),
                             act_period=300, act_offset=float(off[b]))
        alone["origin"] = sc["origin"][b:b + 1]
        alone["phase"] = np.full(scenes.n_occupied(alone), ph[b], np.float32)
        oa = Oracle(alone)
        oa.step(900)
        s = oa.state()
        for k in ("pos", "quat", "vel", "angvel", "static"):
            assert np.array_equal(s[k], both[k][sl]), (b, k)
    # and the per-material signals matter: the global signal gives another motion
    g = Oracle(two_bodies_two_materials())
    g.step(900)
    assert not np.allclose(g.state()["pos"], both["pos"], rtol=0, atol=1e-9)


def test_material_signals_equal_to_global_change_nothing():
    """Per-material values equal to the global amplitude and offset, zero
    phase shifts: the same trajectory bit for bit; a phase shift of pi on a
    material equals flipping the sign of its expansion coefficient."""
    sc = two_bodies_two_materials()
    o = Oracle(sc)
    o.step(600)
    ref = o.state()
    sc2 = two_bodies_two_materials()
    sc2.update(mat_act_amplitude=scenes.f32([5.0, 5.0]), mat_act_offset=scenes.f32([1.0, 1.0]),
               mat_act_phase=scenes.f32([0.0, 0.0]))
    o2 = Oracle(sc2)
    o2.step(600)
    for k in ("pos", "quat", "vel", "angvel"):
        assert np.array_equal(o2.state()[k], ref[k]), k
    # sin(x + pi) = -sin(x): with zero offsets, a pi shift on material 1 and
    # its cte negated describe the same physics (equal up to sine rounding)
    sc3 = two_bodies_two_materials()
    sc3.update(act_offset=0.0, mat_act_phase=np.array([0.0, math.pi]))
    sc4 = two_bodies_two_materials()
    sc4.update(act_offset=0.0)
    sc4["palette"] = sc4["palette"].copy()
    sc4["palette"][1, 3] = -sc4["palette"][1, 3]
    o3, o4 = Oracle(sc3), Oracle(sc4)
    o3.step(600)
    o4.step(600)
    s3, s4 = o3.state(), o4.state()
    span = np.ptp(s4["pos"], axis=0).max()
    assert np.abs(s3["pos"] - s4["pos"]).max() <= 1e-9 * span
