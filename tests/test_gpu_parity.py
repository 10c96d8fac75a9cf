"""GPU (sm_103a kernels through the C ABI) against the FP64 oracle.

Every test builds the same seeded scene on both sides, steps both, and
compares element by element.  Tolerances (FP32 kernel vs FP64 oracle):
positions within 1e-5 of the body's bounding-box diagonal after 1,000 steps
without contact, 1e-3 with contact and friction; one-step force responses
within 1e-4 of the largest response; collision candidate sets bit-exact.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_1212_2845_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1212_2845_gb300 import build, vx as _vx
    build.build()
    return _vx


def f32_dt(ora):
    """The oracle's own timestep of every body, rounded to FP32 as the kernels step."""
    return np.array([np.float32(ora.dt(b)) for b in range(ora.n_bodies)], dtype=np.float64)


def pair(vx, sc):
    sim = vx.Sim(sc)
    ora = Oracle(sc)
    ora.set_dt(f32_dt(ora))
    return sim, ora


def body_diag(sc, pos):
    ijk = scenes.canonical_coords(sc)
    d = np.zeros(len(pos))
    for b in np.unique(ijk[:, 0]):
        m = ijk[:, 0] == b
        d[m] = np.linalg.norm(np.ptp(pos[m], axis=0)) if m.sum() > 1 else sc["voxel_size"]
    return d


def pos_error(sc, g, o):
    return np.max(np.linalg.norm(g["pos"] - o["pos"], axis=1) / body_diag(sc, o["pos"]))


def quat_error(g, o):
    d1 = np.abs(g["quat"] - o["quat"]).max(axis=1)
    d2 = np.abs(g["quat"] + o["quat"]).max(axis=1)
    return np.minimum(d1, d2).max()


# ---------------------------------------------------------------------------
# single step, every force term on, random perturbed state
# ---------------------------------------------------------------------------

def perturbed_scene(dims, seed, **kw):
    sc = scenes.random_blob(dims, seed=seed, fill=0.75)
    sc.update(gravity_z=-9.81, floor=True, zeta_bond=0.7, zeta_ground=0.05, zeta_collision=0.8,
              act_amplitude=15.0, act_period=37, act_offset=2.0)
    sc.update(kw)
    scenes.normalize(sc)
    rng = np.random.default_rng(seed)
    n = scenes.n_occupied(sc)
    sc["fixed"] = (rng.random(n) < 0.05).astype(np.uint8)
    sc["force"] = scenes.f32(rng.normal(size=(n, 3)) * 1e-4)
    return sc


def random_state(n, seed, l, amp=0.05):
    rng = np.random.default_rng(seed + 100)
    off = (rng.normal(size=(n, 3)) * amp * l).astype(np.float32)
    ax = rng.normal(size=(n, 3))
    ang = rng.normal(size=n) * 0.05
    ax /= np.linalg.norm(ax, axis=1, keepdims=True)
    q = np.concatenate([np.cos(ang / 2)[:, None], np.sin(ang / 2)[:, None] * ax], axis=1)
    q = (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)
    vel = (rng.normal(size=(n, 3)) * 0.01).astype(np.float32)
    w = (rng.normal(size=(n, 3)) * 5.0).astype(np.float32)
    return off, q, vel, w


def set_both(sim, ora, anchors, off, q, vel, w, flags=None):
    sim.write_state(offset=off, quat=q, vel=vel, angvel=w, flags=flags)
    st = None if flags is None else (flags >> 1) & 1
    ora.set_state(pos=anchors + off.astype(np.float64), quat=q.astype(np.float64), vel=vel.astype(np.float64),
                  angvel=w.astype(np.float64), static=st)


def with_material_signals(sc):
    """Three materials, each on its own temperature signal (Sec 2.3): own
    expansion coefficient sign, amplitude, offset and phase shift."""
    sc["palette"] = sc["palette"].copy()
    sc["palette"][:, 3] = scenes.f32([0.01, -0.015, 0.02])
    sc.update(mat_act_amplitude=scenes.f32([6.0, 3.0, -4.0]), mat_act_offset=scenes.f32([1.0, -1.0, 0.5]),
              mat_act_phase=scenes.f32([0.0, 2.1, -0.7]))
    return sc


@pytest.mark.parametrize("dims,seed,signals", [((7, 5, 4), 0, False), ((9, 6, 5), 1, False), ((33, 3, 2), 2, False),
                                               ((1, 1, 13), 3, False), ((9, 6, 5), 4, True), ((33, 3, 2), 5, True)])
def test_one_step_force_response(vx, dims, seed, signals):
    sc = perturbed_scene(dims, seed)
    if signals:
        sc = with_material_signals(sc)
    sim, ora = pair(vx, sc)
    anchors = ora.anchors(sc)
    assert np.allclose(sim.anchors(), anchors, rtol=0, atol=1e-15)
    off, q, vel, w = random_state(sim.N, seed, sc["voxel_size"])
    off[:, 2] -= 0.01 * sc["voxel_size"]  # some voxels pressed into the floor
    free = sc["fixed"] == 0
    vel[~free] = 0
    w[~free] = 0
    for n0 in (0, 11):  # two actuation phases
        sim.set_step(n0)
        ora.set_step_counter(n0)
        set_both(sim, ora, anchors, off, q, vel, w)
        sim.step(1)
        ora.step(1)
        g, o = sim.state(), ora.state()
        dv_g, dv_o = g["vel"] - vel, o["vel"] - vel
        dw_g, dw_o = g["angvel"] - w, o["angvel"] - w
        assert np.abs(dv_g - dv_o).max() <= 1e-4 * np.abs(dv_o).max() + 1e-9
        assert np.abs(dw_g - dw_o).max() <= 1e-4 * np.abs(dw_o).max() + 1e-6
        assert np.array_equal(g["static"], o["static"])
        assert np.abs(g["pos"] - o["pos"]).max() < 1e-10
        assert quat_error(g, o) < 1e-6


# ---------------------------------------------------------------------------
# rollouts
# ---------------------------------------------------------------------------

def test_cantilever_1000_steps(vx):
    """Config 1: 10x10x10 cantilever under gravity, 1,000 steps, 1e-5 of the diagonal."""
    sc = scenes.cantilever()
    sim, ora = pair(vx, sc)
    sim.step(1000)
    ora.step(1000)
    g, o = sim.state(), ora.state()
    err = pos_error(sc, g, o)
    disp = np.abs(o["pos"] - ora.anchors(sc)).max()
    rel_disp = np.abs(g["pos"] - o["pos"]).max() / disp
    print(f"cantilever: pos err/diag {err:.2e}, err/max displacement {rel_disp:.2e}")
    assert err < 1e-5
    assert rel_disp < 1e-3
    assert quat_error(g, o) < 1e-5


def test_hetero_block_reduced(vx):
    """Config 2 mix (soft/stiff, actuation, floor + friction) on a 16x16x8 block, 2,000 steps."""
    sc = scenes.hetero_block(dims=(16, 16, 8), seed=2)
    sim, ora = pair(vx, sc)
    sim.step(2000)
    ora.step(2000)
    g, o = sim.state(), ora.state()
    err = pos_error(sc, g, o)
    flips = int(np.sum(g["static"] != o["static"]))
    print(f"hetero block: pos err/diag {err:.2e}, static flag mismatches {flips}/{sim.N}")
    assert err < 1e-3


def test_material_signals_rollout_with_collisions(vx):
    """Per-material temperature signals through 1,500 steps with floor,
    friction and self-collision on (the collision sizes use each voxel's own
    signal too); the same scene under one global signal moves differently."""
    sc = with_material_signals(scenes.random_blob((10, 8, 6), seed=7, fill=0.8))
    sc.update(gravity_z=-9.81, floor=True, collide=True, zeta_ground=0.05, act_period=400)
    scenes.normalize(sc)
    sim, ora = pair(vx, sc)
    sim.step(1500)
    ora.step(1500)
    g, o = sim.state(), ora.state()
    assert pos_error(sc, g, o) < 1e-3
    sim.set_material_actuation(None, None, None)
    sim.reset()
    sim.step(1500)
    assert pos_error(sc, sim.state(), o) > 5e-3
    sim.close()


def test_population_reduced(vx):
    """Config 4 mix on 12 bodies of uneven size (per-body timestep), 600 steps."""
    sc = scenes.population(n_bodies=12, seed=4, lo=2, hi=9)
    sim, ora = pair(vx, sc)
    assert np.allclose(sim.dt(), [ora.dt(b) for b in range(12)], rtol=1e-7)
    sim.step(600)
    ora.step(600)
    g, o = sim.state(), ora.state()
    assert pos_error(sc, g, o) < 1e-3


def test_design_population_reduced(vx):
    """Config 5 inputs (per-voxel log-stiffness and phase) on 3 bodies of 6^3, 400 steps."""
    sc = scenes.design_population(n_bodies=3, n=6, seed=5)
    sim, ora = pair(vx, sc)
    sim.step(400)
    ora.step(400)
    assert pos_error(sc, sim.state(), ora.state()) < 1e-3


def test_appendix_a_program(vx):
    """App. A: 5x10x5 beam of 10 MPa voxels, -Y face fixed, force on the +Y face,
    slow damping 0.013, 400 steps.  The printed 1 kN (40 MPa on a 5 mm x 5 mm
    section, strain ~4) is far outside the small-angle beam model and diverges
    on both sides; 1 N keeps the same program in the elastic range."""
    sc = scenes._base([(5, 10, 5)], np.ones(250, np.uint8), 1e-3, [scenes.material(1e7, 0.3)],
                      zeta_ground=0.013)
    sim = vx.Sim(sc)
    ora = Oracle(sc)
    assert sim.add_fixed_region(0, (0, 0, 0), (1, 0.01, 1)) == 25      # the y = 0 layer, 5 x 5
    assert sim.add_forced_region(0, (0, 0.99, 0), (1, 0.01, 1), (0, 0, -1.0)) == 25
    fixed = ora.region_mask(0, (0, 0, 0), (1, 0.01, 1))
    ora.set_fixed(fixed)
    m = ora.region_mask(0, scenes.f32((0, 0.99, 0)), scenes.f32((1, 0.01, 1)))
    F = np.zeros((ora.N, 3))
    F[m.astype(bool), 2] = float(np.float32(-1.0 / 25))
    ora.set_force(F)
    ora.reset()
    ora.set_dt(f32_dt(ora))
    sim.step(400)
    ora.step(400)
    g, o = sim.state(), ora.state()
    assert np.array_equal(g["flags"] & 1, fixed)
    assert pos_error(sc, g, o) < 1e-5


def test_deterministic_bitwise(vx):
    sc = scenes.hetero_block(dims=(12, 9, 7), seed=6)
    outs = []
    for _ in range(2):
        sim = vx.Sim(sc)
        sim.step(300)
        s = sim.read_state()
        outs.append(np.concatenate([s["offset"].ravel(), s["quat"].ravel(), s["vel"].ravel(), s["angvel"].ravel()]))
        sim.close()
    assert np.array_equal(outs[0].view(np.uint32), outs[1].view(np.uint32))


def test_state_roundtrip_and_reset(vx):
    sc = scenes.random_blob((5, 4, 3), seed=9)
    sim = vx.Sim(sc)
    off, q, vel, w = random_state(sim.N, 9, sc["voxel_size"])
    flags = np.zeros(sim.N, np.uint8)
    sim.write_state(offset=off, quat=q, vel=vel, angvel=w, flags=flags)
    s = sim.read_state()
    for k, a in (("offset", off), ("quat", q), ("vel", vel), ("angvel", w)):
        assert np.array_equal(s[k], a)
    sim.reset()
    s = sim.read_state()
    assert not s["offset"].any() and not s["vel"].any()
    assert np.array_equal(s["quat"], np.tile([1, 0, 0, 0], (sim.N, 1)).astype(np.float32))
    assert sim.step_count == 0
    # the asynchronous upload from pinned host buffers, then a read on the
    # same stream into pinned buffers
    torch = pytest.importorskip("torch")
    fl2 = (np.arange(sim.N) % 3 == 0).astype(np.uint8) * 2
    pin = {k: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
           for k, a in (("offset", off), ("quat", q), ("vel", vel), ("angvel", w), ("flags", fl2))}
    stream = torch.cuda.Stream()
    sim.write_state_from(**pin, stream=stream, on_device=False, wait=False)
    out = {k: torch.empty_like(t).pin_memory() for k, t in pin.items()}
    sim.read_state_into(**out, stream=stream, on_device=False)
    for k in pin:
        assert torch.equal(out[k], pin[k]), k
    s = sim.read_state()  # pageable buffers: the staging copies
    for k in pin:
        assert np.array_equal(s[k], pin[k].numpy()), k
    # a view mixing pinned and pageable buffers
    off2 = off + np.float32(1e-6)
    sim.write_state_from(offset=torch.from_numpy(off2).pin_memory(), quat=np.ascontiguousarray(q[::-1]),
                         stream=stream, on_device=False)
    s = sim.read_state()
    assert np.array_equal(s["offset"], off2) and np.array_equal(s["quat"], q[::-1])
    part = {"vel": torch.empty_like(pin["vel"]).pin_memory()}
    sim.read_state_into(**part, stream=stream, on_device=False)  # one field, pinned
    assert torch.equal(part["vel"], pin["vel"])


def test_initial_velocity(vx):
    """vx_set_initial_velocity moves every non-fixed voxel at v now and is the
    velocity of a later reset without one; fixed voxels stay at rest."""
    sc = scenes.random_blob((6, 5, 4), seed=3)
    sc["fixed"] = (np.arange(scenes.n_occupied(sc)) % 5 == 0).astype(np.uint8)
    sim = vx.Sim(sc)
    sim.step(20)
    before = sim.read_state()
    v = np.array([0.01, -0.02, 0.03], np.float32)
    sim.set_initial_velocity(v)
    after = sim.read_state()
    free = sc["fixed"] == 0
    assert np.array_equal(after["vel"][free], np.tile(v, (free.sum(), 1)))
    assert not after["vel"][~free].any()
    for k in ("offset", "quat", "angvel"):
        assert np.array_equal(after[k], before[k]), k
    sim.reset()
    s = sim.read_state()
    assert np.array_equal(s["vel"][free], np.tile(v, (free.sum(), 1))) and not s["offset"].any()
    with pytest.raises(vx.VxError):
        sim.set_initial_velocity([np.nan, 0.0, 0.0])
    sim.close()


def test_checkpoint_resume_is_bit_exact_with_collisions(vx):
    """Stop a run, copy out its state (offsets, quaternions, velocities,
    angular velocities, flags) and step counter, load them into a new
    simulator and continue: the continuation equals the uninterrupted run bit
    for bit, through the shell's impact with self-collision.  Writing a
    state counts as motion for the horizon (here far past its threshold, so
    the lists are rebuilt from it); only overlapping candidates act, so the
    horizon history does not matter."""
    sc = scenes.hollow_ball(R=12, t=3)
    a = vx.Sim(sc)
    a.step(300)
    ck = a.read_state()
    n = a.step_count
    b = vx.Sim(sc)
    b.step(17)                                            # some other history first
    b.write_state(offset=ck["offset"], quat=ck["quat"], vel=ck["vel"], angvel=ck["angvel"], flags=ck["flags"])
    b.set_step(n)
    a.step(700)
    b.step(700)
    sa, sb = a.read_state(), b.read_state()
    for k in ("offset", "quat", "vel", "angvel", "flags"):
        assert np.array_equal(sa[k].view(np.uint8), sb[k].view(np.uint8)), k
    a.close()
    b.close()


def test_unstable_is_reported_not_trapped(vx):
    sc = scenes.random_blob((4, 4, 4), seed=1)
    sc.update(zeta_bond=0.0)
    sim = vx.Sim(sc)
    off, q, vel, w = random_state(sim.N, 1, sc["voxel_size"])
    sim.write_state(offset=off, quat=q, vel=vel, angvel=w)
    sim.set_dt(sim.dt() * 40)
    with pytest.raises(vx.VxError) as e:
        sim.step(3000)
    assert e.value.code == -4
    st, bad_step, bad_voxel = sim.status()
    assert st == -4 and 0 <= bad_step < 3000 and 0 <= bad_voxel < sim.N
    sim.reset()
    sim.set_dt_factor(0.9)
    sim.step(10)


# ---------------------------------------------------------------------------
# collision candidates (bit-exact sets)
# ---------------------------------------------------------------------------

def scrambled_offsets(n, l, seed, amp=0.45):
    rng = np.random.default_rng(seed)
    return (rng.uniform(-amp, amp, size=(n, 3)) * l).astype(np.float32)


@pytest.mark.parametrize("seed", [0, 1])
def test_collision_set_bit_exact_small(vx, seed):
    sc = scenes.hollow_ball(R=10, t=3)
    sc["collide"] = True
    sim, ora = pair(vx, sc)
    off = scrambled_offsets(sim.N, sc["voxel_size"], seed)
    sim.write_state(offset=off)
    sim.rebuild_collisions()
    gp = {tuple(p) for p in sim.collision_pairs()}
    op = {tuple(p) for p in ora.pairs_from_offsets(off.astype(np.float64))}
    print(f"pairs: gpu {len(gp)}, oracle {len(op)}")
    assert len(op) > 100
    assert gp == op


def test_collision_threshold_exact(vx):
    """Pairs placed exactly on, one unit inside and one unit outside the
    quantised 2-voxel horizon."""
    l = float(scenes.f32(1e-3))
    K, Q = Oracle.quant_params(l)
    grid = np.zeros(9, np.uint8)
    grid[[0, 4, 8]] = 1
    sc = scenes._base([(9, 1, 1)], grid, l, [scenes.material(1e6)], collide=True)
    sim, ora = pair(vx, sc)
    for dq, expect in [(0, False), (1, True), (-1, False)]:
        off = np.zeros((3, 3), np.float32)
        off[1, 0] = np.float32((-2 * Q - dq) / 2.0 ** K)   # voxel 4 moved to 2 Q - dq from voxel 0
        off[2, 0] = np.float32(10 * l)                       # voxel 8 far away
        sim.write_state(offset=off)
        sim.rebuild_collisions()
        gp = {tuple(p) for p in sim.collision_pairs()}
        op = {tuple(p) for p in ora.pairs_from_offsets(off.astype(np.float64))}
        assert gp == op
        assert ((0, 1) in gp) == expect


@pytest.mark.parametrize("R", [60, 100])
def test_collision_sets_complete_on_the_thread_query_path(vx, R):
    """Shells with more than 8 surface voxels per warp of the rebuild grid
    (R60 t8: 65,792 surface voxels, the smallest such shell; R100 t8: the
    full ball, 192,848), where the query searches one voxel per thread: the
    complete candidate set of a scrambled state against the oracle's search
    on the same FP32 offsets."""
    sc = scenes.hollow_ball(R=R, t=8)
    sim = vx.Sim(sc, apply_scene=False)
    sim.set_environment(0.0, False, True)
    ora = Oracle(sc, apply_scene=False)
    assert sim.n_surface > 65536
    off = scrambled_offsets(sim.N, sc["voxel_size"], 5, amp=0.4)
    sim.write_state(offset=off)
    sim.rebuild_collisions()
    gp = sim.collision_pairs()
    op = ora.pairs_from_offsets(off.astype(np.float64))
    gp = gp[np.lexsort((gp[:, 1], gp[:, 0]))]
    print(f"R{R}: {sim.n_surface} surface voxels, {len(op)} pairs")
    assert len(op) > 5000
    assert np.array_equal(gp, op)
    sim.close()


def test_ball_drop_with_self_collision(vx):
    """Config 3 physics on a scaled shell (R=12, t=3): floor impact, horizon
    rebuilds and voxel contacts, 900 steps."""
    sc = scenes.hollow_ball(R=12, t=3)
    sim, ora = pair(vx, sc)
    sim.step(900)
    ora.step(900)
    g, o = sim.state(), ora.state()
    err = pos_error(sc, g, o)
    nr_g, _ = sim.collision_stats()
    nr_o = ora.n_rebuilds()
    print(f"ball: pos err/diag {err:.2e}, rebuilds gpu {nr_g} oracle {nr_o}")
    assert err < 1e-3
    assert abs(nr_g - nr_o) <= max(2, nr_o // 10)


# ---------------------------------------------------------------------------
# step forms and tile sizes
# ---------------------------------------------------------------------------

def run_form(vx, sc, steps, form, tile_max=0):
    sim = vx.Sim(sc)
    sim.set_step_form(form, tile_max)
    sim.step(steps)
    s = sim.read_state()
    sim.close()
    return s


@pytest.mark.parametrize("which", ["hetero", "ball", "population"])
def test_fused_tile_sizes_bitwise_and_two_pass_close(vx, which):
    """Every operation of the step is an explicitly rounded intrinsic, so the
    fused kernel gives the same bits for every tile size and the two-pass form
    gives the same bits as the fused one, as does the pipelined form."""
    if which == "hetero":
        sc, steps = scenes.hetero_block(dims=(20, 17, 9), seed=3), 300
    elif which == "ball":
        sc, steps = scenes.hollow_ball(R=10, t=3), 500
    else:
        sc, steps = scenes.population(n_bodies=9, seed=7, lo=2, hi=11), 300
    ref = run_form(vx, sc, steps, vx.FORM_FUSED, 256)
    for tm in (128, 512):
        out = run_form(vx, sc, steps, vx.FORM_FUSED, tm)
        for k in ("offset", "quat", "vel", "angvel", "flags"):
            assert np.array_equal(out[k].view(np.uint8), ref[k].view(np.uint8)), (tm, k)
    for form, tm in ((vx.FORM_TWO_PASS, 0), (vx.FORM_PIPELINED, 256), (vx.FORM_PIPELINED, 128)):
        other = run_form(vx, sc, steps, form, tm)
        for k in ("offset", "quat", "vel", "angvel", "flags"):
            assert np.array_equal(other[k].view(np.uint8), ref[k].view(np.uint8)), (form, tm, k)


def _lean_scene(mode):
    """A lattice of each lean step kernel's feature set: voxel contacts (bit
    0), several bodies (bit 1), actuation with per-voxel phases (bit 2); and
    two that take the generic kernel (actuation without phases, per-voxel
    moduli)."""
    if mode == "generic_act_no_phase":
        sc = scenes.cantilever(n=(8, 5, 4))
        sc.update(act_amplitude=10.0, act_period=300)
        sc["palette"][:, 3] = 0.01
        return sc
    if mode == "generic_log_E":
        return scenes.design_population(n_bodies=3, n=5, seed=2)
    bits = mode - 1
    if bits & 2:
        sc = scenes.population(n_bodies=6, seed=5, lo=3, hi=8)
    else:
        sc = scenes.hollow_ball(R=8, t=3, drop=1)
    sc["collide"] = bool(bits & 1)
    if not bits & 4:
        sc.update(act_amplitude=0.0, act_period=0)
        sc["phase"] = None
    elif sc.get("phase") is None:
        sc.update(act_amplitude=15.0, act_period=400)
        sc["palette"][:, 3] = 0.01
        rng = np.random.default_rng(mode)
        sc["phase"] = scenes.f32(rng.uniform(0.0, 6.28, scenes.n_occupied(sc)))
    return sc


@pytest.mark.parametrize("mode", [1, 2, 3, 4, 5, 6, 7, 8, "generic_act_no_phase", "generic_log_E"])
def test_lean_step_kernels_bitwise_equal_generic(vx, mode):
    """The 256-voxel pipelined step launches a lean instantiation with the
    lattice's absent features fixed at compile time; every one gives the
    bits of the generic kernel (the 128-voxel tiles always take it)."""
    sc = _lean_scene(mode)
    ref = run_form(vx, sc, 250, vx.FORM_PIPELINED, 128)
    out = run_form(vx, sc, 250, vx.FORM_PIPELINED, 256)
    assert np.abs(ref["vel"]).max() > 0
    for k in ("offset", "quat", "vel", "angvel", "flags"):
        assert np.array_equal(out[k].view(np.uint8), ref[k].view(np.uint8)), k


# ---------------------------------------------------------------------------
# batched form: many bodies, all steps in one launch
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("group", [64, 700, 5000])
def test_batched_form_bitwise_equals_per_step(vx, group):
    sc = scenes.population(n_bodies=23, seed=17, lo=2, hi=12)
    ref = run_form(vx, sc, 250, vx.FORM_PIPELINED, 256)
    sim = vx.Sim(sc)
    sim.set_batching(group)
    sim.step(250)
    out = sim.read_state()
    assert sim.step_count == 250
    for k in ("offset", "quat", "vel", "angvel", "flags"):
        assert np.array_equal(out[k].view(np.uint8), ref[k].view(np.uint8)), k
    sim.set_batching(0)
    sim.step(3)                      # back to per-step launches, still consistent
    assert sim.step_count == 253


def test_batched_design_population_vs_oracle(vx):
    """Config 5 inputs (per-voxel log stiffness, phases) through the batched form."""
    sc = scenes.design_population(n_bodies=4, n=6, seed=5)
    sim, ora = pair(vx, sc)
    sim.set_batching(300)
    sim.step(300)
    ora.step(300)
    assert pos_error(sc, sim.state(), ora.state()) < 1e-3


def test_graph_replays_continue_the_rollout(vx):
    """One captured batched launch of 7 steps replayed 3 times equals 21
    steps (odd step count: the state buffer alternates between replays;
    actuation: each replay continues the step counter)."""
    sc = scenes.population(n_bodies=23, seed=17, lo=2, hi=12)
    sc["act_period"] = 40
    ref = run_form(vx, sc, 21, vx.FORM_PIPELINED, 256)
    sim = vx.Sim(sc)
    sim.set_batching(700)
    sim.graph_capture(7)
    for _ in range(3):
        sim.graph_launch()
    assert sim.status()[0] == 0
    out = sim.read_state()
    assert sim.step_count == 21
    for k in ("offset", "quat", "vel", "angvel", "flags"):
        assert np.array_equal(out[k].view(np.uint8), ref[k].view(np.uint8)), k
    sim.set_damping(1.0, 0.0, 0.5)               # model changed: the graph is stale
    with pytest.raises(vx.VxError) as e:
        sim.graph_launch()
    assert e.value.code == -6
    sim.close()


def test_autotuner_restores_state_and_keeps_results(vx):
    sc = scenes.population(n_bodies=40, seed=3, lo=3, hi=14)
    ref = run_form(vx, sc, 60, vx.FORM_PIPELINED, 256)
    sim = vx.Sim(sc)
    sim.step(20)
    before = sim.read_state()
    tm, gv, rate = sim.autotune_batching(10)
    assert tm in (128, 256) and gv in (0, 1024, 4096, 16384, 65536, vx.GROUPS_RESIDENT) and rate > 0
    after = sim.read_state()
    assert sim.step_count == 20
    for k in before:
        assert np.array_equal(before[k], after[k]), k
    assert sim.tiling()["tile_max"] == tm
    sim.step(40)                                  # the tuned form continues bit for bit
    out = sim.read_state()
    for k in ("offset", "quat", "vel", "angvel", "flags"):
        assert np.array_equal(out[k].view(np.uint8), ref[k].view(np.uint8)), k
    assert sim.autotune_batching(10)[:2] == (tm, gv)   # cached for the size class
    sim.close()


@pytest.mark.parametrize("which", ["hetero_small", "population"])
def test_multistep_launch_bitwise_equals_per_step_launches(vx, which):
    """One cooperative launch of n steps (grid barrier between steps) gives the
    bits of n separate launches."""
    if which == "hetero_small":
        sc = scenes.hetero_block(dims=(20, 18, 12), seed=9)
    else:
        sc = scenes.population(n_bodies=30, seed=8, lo=3, hi=14)
    out = []
    for multi in (0, 1, 2):           # per-step launches, default (resident on small lattices), grid launch
        sim = vx.Sim(sc)
        sim.set_multistep(multi)
        sim.step(301)
        out.append(sim.read_state())
        assert sim.step_count == 301
        sim.close()
    for o in out[1:]:
        for k in ("offset", "quat", "vel", "angvel", "flags"):
            assert np.array_equal(out[0][k].view(np.uint8), o[k].view(np.uint8)), k


@pytest.mark.parametrize("which", ["clapper_horizon", "clapper_every_step", "ball_impact", "shared_world"])
def test_multistep_launch_with_collisions_bitwise_equals_per_step_launches(vx, which):
    """With collisions on, the cooperative multi-step launch keeps the horizon
    and runs the candidate rebuilds between its steps on its own grid; states,
    candidate sets and the rebuild count equal those of one launch per step
    (followed by the separate rebuild launch)."""
    every = False
    if which.startswith("clapper"):
        sc, steps = scenes.clapper(), 1500
        every = which == "clapper_every_step"
    elif which == "ball_impact":
        sc, steps = scenes.hollow_ball(R=12, t=3), 900
    else:
        l = 1e-3
        sc = scenes._base([(3, 3, 3), (3, 3, 3)], np.ones(54, np.uint8), l, [scenes.material(1e6)],
                          collide=2, zeta_collision=0.0, zeta_bond=1.0)
        sc["origin"] = scenes.f32([[0.0, 0.0, 0.0], [6 * l, 0.0, 0.0]])
        steps = 2500
    out = []
    for multi in (0, 1):
        sim = vx.Sim(sc, apply_scene=False)
        sim.set_collision_scheme(False, every)
        sim.apply(sc)
        if which == "shared_world":
            vel = np.zeros((sim.N, 3), np.float32)
            vel[:27, 0], vel[27:, 0] = 0.2, -0.2
            sim.write_state(vel=vel)
        sim.set_multistep(multi)
        sim.step(steps)
        assert sim.status()[0] == 0
        out.append((sim.read_state(), sim.collision_pairs(), sim.collision_stats()[0]))
        sim.close()
    (s0, p0, n0), (s1, p1, n1) = out
    for k in ("offset", "quat", "vel", "angvel", "flags"):
        assert np.array_equal(s0[k].view(np.uint8), s1[k].view(np.uint8)), k
    assert np.array_equal(p0, p1)
    assert n0 == n1 and n0 > 0


def test_simulators_of_different_sizes_coexist(vx):
    """Kernel launch limits set for one simulator never break another one in
    the same process (every form, stepped in turn)."""
    a = vx.Sim(scenes.hetero_block(dims=(20, 18, 12), seed=9))       # phase: larger staging
    b = vx.Sim(scenes.cantilever())
    for form in (vx.FORM_PIPELINED, vx.FORM_FUSED):
        a.set_step_form(form)
        b.set_step_form(form)
        a.step(3)
        b.step(3)
        a.step(3)
    a.set_step_form(vx.FORM_PIPELINED)
    a.set_batching(1000)
    b.set_batching(1000)
    a.step(4)
    b.step(4)
    a.step(4)
    assert a.status()[0] == 0 and b.status()[0] == 0
    a.close()
    b.close()


def test_cantilever_impulse_response_modes(vx):
    """The kernels ring at the linearised lattice's bending frequencies (the
    oracle's assembled [K] and lumped masses) after a tip impulse, and follow
    the oracle's trajectory sample by sample."""
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from test_oracle_pins import thin_cantilever_scene, bending_frequencies, spectrum_peaks
    sc = thin_cantilever_scene()
    ora = Oracle(sc)
    f_lin = np.unique(np.round(bending_frequencies(ora, sc), 6))[:3]
    sim = vx.Sim(sc)
    ora.set_dt(f32_dt(ora))
    vel = np.zeros((20, 3), np.float32)
    vel[19, 2] = 1e-3
    sim.write_state(vel=vel)
    ora.set_state(vel=vel.astype(np.float64))
    every, n = 10, 32768
    zg, zo = np.empty(n), np.empty(n)
    for i in range(n):
        sim.step(every)
        ora.step(every)
        zg[i] = sim.state()["pos"][19, 2]
        zo[i] = ora.state()["pos"][19, 2]
    peaks = spectrum_peaks(zg, every * ora.dt(), f_lin)
    assert np.all(np.abs(peaks / f_lin - 1.0) <= 2e-3), (peaks, f_lin)
    amp = np.abs(zo - zo.mean()).max()
    assert np.abs(zg - zo).max() <= 1e-3 * amp


def test_relaxation_to_static_matches_linear_solve(vx):
    """App. A's static use: the -Y face of the 5x10x5 beam fixed, a small load
    on the +Y face (1 N, elastic range), damped stepping until every voxel
    speed is below 1e-4 m/s (the loaded tip moves at ~0.5 m/s; FP32 rounding
    of the forces keeps speeds near 1e-7-1e-6 m/s even at rest).  The relaxed
    deflection equals the oracle's linear direct-stiffness solve of the
    printed [K] to geometric nonlinearity (< 1 %)."""
    sc = scenes._base([(5, 10, 5)], np.ones(250, np.uint8), 1e-3, [scenes.material(1e7, 0.3)],
                      zeta_bond=1.0, zeta_ground=0.2)
    sim = vx.Sim(sc)
    sim.add_fixed_region(0, (0, 0, 0), (1, 0.01, 1))
    sim.add_forced_region(0, (0, 0.99, 0), (1, 0.01, 1), (0, 0, -1.0))
    steps, vmax, ok = sim.relax(400000, 1e-4, check_every=500)
    assert ok and vmax <= 1e-4 and 0 < steps < 400000, (steps, vmax)
    ora = Oracle(sc)
    fixed = ora.region_mask(0, (0, 0, 0), (1, 0.01, 1))
    ora.set_fixed(fixed)
    m = ora.region_mask(0, scenes.f32((0, 0.99, 0)), scenes.f32((1, 0.01, 1))).astype(bool)
    f = np.zeros((ora.N, 6))
    f[m, 2] = -1.0 / m.sum()
    u = ora.linear_static(f)
    g = sim.state()
    dz = g["pos"][:, 2] - sim.anchors()[:, 2]
    tip = m
    assert dz[tip].mean() == pytest.approx(u[tip, 2].mean(), rel=1e-2)
    assert np.abs(dz - u[:, 2]).max() <= 2e-2 * np.abs(u[:, 2]).max()
    # already static: converges at the first check
    n2, v2, ok2 = sim.relax(10000, 1e-4, check_every=500)
    assert ok2 and n2 == 500
    sim.close()


def test_shared_world_collision_matches_oracle(vx):
    """Two cubes in one world approach head-on, collide and bounce: the
    kernels follow the oracle, and the candidate set of the final GPU
    snapshot (cross-body pairs included) equals the oracle's brute force on
    the same offsets bit for bit."""
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from test_oracle_pins import two_cubes
    sc, v = two_cubes()
    sim, ora = pair(vx, sc)
    assert sim.dt()[0] == sim.dt()[1]
    N = sim.N
    vel = np.zeros((N, 3), np.float32)
    vel[: N // 2, 0] = v
    vel[N // 2:, 0] = -v
    sim.write_state(vel=vel)
    sim.rebuild_collisions()
    ora.set_state(vel=vel.astype(np.float64))
    ora.reset_candidates()
    cross = 0
    for _ in range(40):
        sim.step(100)
        ora.step(100)
        cross += sum(1 for i, j in sim.collision_pairs() if (i < N // 2) != (j < N // 2))
    g, o = sim.state(), ora.state()
    assert cross > 0
    assert pos_error(sc, g, o) < 1e-3
    assert g["vel"][: N // 2, 0].mean() < 0 < g["vel"][N // 2:, 0].mean()
    off = sim.read_state()["offset"].astype(np.float64)
    sim.rebuild_collisions()
    got = {tuple(int(x) for x in p) for p in sim.collision_pairs()}
    ref = {tuple(int(x) for x in p) for p in ora.pairs_from_offsets(off)}
    assert got == ref
    sim.close()


def test_collision_schemes_on_the_clapper(vx):
    """All four collision schemes (all / surface voxels x every step /
    horizon) step the clapper through its contact to the same bits; the
    trajectory follows the oracle; at the contact the candidate set of each
    scheme equals the oracle's brute force on the same GPU offsets."""
    sc = scenes.clapper()
    ora = Oracle(sc)
    ora.set_dt(f32_dt(ora))
    ora.step(1200)
    finals = []
    for all_voxels, every in ((False, False), (True, True), (False, True), (True, False)):
        sim = vx.Sim(sc)
        sim.set_collision_scheme(all_voxels, every)
        sim.step(1200)
        g = sim.state()
        finals.append(g)
        off = sim.read_state()["offset"].astype(np.float64)
        sim.rebuild_collisions()
        got = {tuple(int(x) for x in p) for p in sim.collision_pairs()}
        ref_o = Oracle(sc)
        ref_o.set_collision_scheme(all_voxels, every)
        ref = {tuple(int(x) for x in p) for p in ref_o.pairs_from_offsets(off)}
        assert got == ref and len(got) > 0, (all_voxels, every)
        sim.close()
    for g in finals[1:]:
        for k in ("pos", "quat", "vel", "angvel"):
            assert np.array_equal(g[k], finals[0][k]), k
    assert pos_error(sc, finals[0], ora.state()) < 1e-3


# ---------------------------------------------------------------------------
# full-size population in the bench's batched launch configuration, sampled
# ---------------------------------------------------------------------------

def population_body(sc, b):
    """Body b of a population scene as a scene of its own (same origin)."""
    dims = sc["dims"]
    sites = np.prod(dims, axis=1)
    s0 = int(sites[:b].sum())
    occ = np.array([np.count_nonzero(sc["grid"][int(sites[:k].sum()):int(sites[:k + 1].sum())])
                    for k in range(b + 1)])
    o0 = int(occ[:b].sum())
    out = dict(sc)
    out["dims"] = dims[b:b + 1].copy()
    out["grid"] = sc["grid"][s0:s0 + int(sites[b])].copy()
    out["origin"] = sc["origin"][b:b + 1].copy()
    out["phase"] = sc["phase"][o0:o0 + int(occ[b])].copy()
    return out, o0, int(occ[b])


def _oracle_body_run(args):
    sc, steps = args
    o = Oracle(sc)
    o.set_dt(f32_dt(o))
    o.step(steps)
    return o.state()["pos"]


def test_full_population_batched_graph_sampled_bodies(vx):
    """The batched workload at full size (4,096 bodies of edges U{4..24}, 8.9M
    voxels), stepped as the bench times it (groups of whole bodies, one
    captured graph replay of 200 steps); eight sampled bodies against the
    oracle stepping each body alone (the bodies are separate worlds)."""
    import multiprocessing as mp
    sc = scenes.population(n_bodies=4096)
    steps = 200
    rng = np.random.default_rng(12)
    picks = sorted(rng.choice(4096, size=8, replace=False).tolist())
    jobs, spans = [], []
    for b in picks:
        sb, o0, n = population_body(sc, b)
        jobs.append((sb, steps))
        spans.append((sb, o0, n))
    with mp.get_context("spawn").Pool(8) as pool:
        pending = pool.map_async(_oracle_body_run, jobs)
        sim = vx.Sim(sc)
        sim.set_batching(4096)
        sim.graph_capture(steps)
        sim.graph_launch()
        g = sim.state()
        assert sim.status()[0] == 0
        sim.close()
        ora = pending.get()
    for (sb, o0, n), o in zip(spans, ora):
        gp = g["pos"][o0:o0 + n]
        diag = np.linalg.norm(np.ptp(o, axis=0)) if n > 1 else sb["voxel_size"]
        assert np.abs(gp - o).max() / diag < 1e-3, (o0, n)


# ---------------------------------------------------------------------------
# edge lattices: no bonds, the largest lattice coordinates, isolated voxels,
# bodies of one voxel next to large ones, everything fixed, zero steps
# ---------------------------------------------------------------------------

def edge_scene(case):
    pal = [scenes.material(1e6, cte=0.01), scenes.material(5e7, rho=1200.0)]
    kw = dict(gravity_z=-9.81, floor=True, zeta_ground=0.05, act_amplitude=10.0, act_period=300)
    if case == "single_voxel":
        sc = scenes._base([(1, 1, 1)], [1], 1e-3, pal, **kw)
        sc["v0"] = (0.02, -0.01, -0.05)
        return scenes.normalize(sc), 3000
    if case in ("line_x_2048", "line_y_2048", "column_z_1024"):
        d = {"line_x_2048": (2048, 1, 1), "line_y_2048": (1, 2048, 1), "column_z_1024": (1, 1, 1024)}[case]
        n = int(np.prod(d))
        grid = 1 + (np.arange(n) % 7 == 3).astype(np.uint8)        # every 7th voxel stiff
        sc = scenes._base([d], grid, 1e-3, pal, **kw)
        sc["phase"] = scenes.f32(np.linspace(0.0, 2.0 * np.pi, n))
        return scenes.normalize(sc), 200
    if case == "sparse_blob":                                       # many isolated voxels and small clusters
        sc = scenes.random_blob((12, 10, 8), seed=21, fill=0.3)
        sc.update(collide=True, **kw)
        return scenes.normalize(sc), 800
    if case == "ragged_bodies":                                     # bodies of 1 to 5^3 sites, one world each
        # without the population's 20 K step of actuation strain at the
        # start, whose transient leaves a few dangling voxels spinning
        # chaotically in such small bodies
        sc = scenes.population(n_bodies=40, seed=9, lo=1, hi=5)
        sc.update(act_amplitude=0.0, zeta_ground=0.05)
        sc["v0"] = (0.01, 0.0, -0.02)
        return scenes.normalize(sc), 600
    raise KeyError(case)


@pytest.mark.parametrize("case", ["single_voxel", "line_x_2048", "line_y_2048", "column_z_1024", "sparse_blob",
                                  "ragged_bodies"])
def test_edge_lattices_follow_the_oracle(vx, case):
    sc, steps = edge_scene(case)
    sim, ora = pair(vx, sc)
    assert np.allclose(sim.anchors(), ora.anchors(sc), rtol=0, atol=1e-15)
    sim.step(steps)
    ora.step(steps)
    g, o = sim.state(), ora.state()
    assert pos_error(sc, g, o) < 1e-3, case
    # the body diagonal of a 2 m line is a loose yardstick: also hold the
    # error to a few percent of the largest displacement
    disp = np.abs(o["pos"] - ora.anchors(sc)).max()
    assert np.abs(g["pos"] - o["pos"]).max() <= 5e-2 * disp, case
    assert quat_error(g, o) < 1e-3
    sim.close()


def test_all_fixed_and_zero_steps_leave_the_state_unchanged(vx):
    sc = scenes.random_blob((7, 6, 5), seed=4, fill=0.8)
    sc.update(gravity_z=-9.81, floor=True, act_amplitude=20.0, act_period=50)
    scenes.normalize(sc)
    sc["fixed"] = np.ones(scenes.n_occupied(sc), np.uint8)
    sim = vx.Sim(sc)
    s0 = sim.read_state()
    sim.step(0)
    sim.step(300)
    s1 = sim.read_state()
    for k in ("offset", "quat", "vel", "angvel", "flags"):
        assert np.array_equal(s0[k], s1[k]), k
    assert sim.step_count == 300
    sim.close()
