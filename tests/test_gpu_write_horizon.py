"""A state write with collisions on is motion for the collision horizon
(Sec 2.2.2): each body's accumulator grows by twice the largest displacement
the write gives a voxel, and the candidate lists are rebuilt only when it
reaches the threshold.  The lists kept across a small write hold every pair
that can touch before the next rebuild, so the trajectory equals the one with
a rebuild forced after the write, bit for bit; a large write rebuilds lists
equal to the oracle's search of the written offsets."""
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


def _same(a, b):
    for k in ("offset", "quat", "vel", "angvel", "flags"):
        assert np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)), k


def test_writing_back_the_read_state_keeps_the_lists(vx):
    sim = vx.Sim(scenes.hollow_ball(R=12, t=3))
    sim.step(300)
    n0, acc0 = sim.collision_stats()
    pairs0 = sim.collision_pairs()
    st = sim.read_state()
    for _ in range(3):
        sim.write_state(offset=st["offset"], quat=st["quat"], vel=st["vel"], angvel=st["angvel"], flags=st["flags"])
    n1, acc1 = sim.collision_stats()
    assert n1 == n0 and acc1 == acc0
    assert np.array_equal(sim.collision_pairs(), pairs0)
    sim.write_state(vel=np.zeros((sim.N, 3), np.float32))   # velocities alone move nothing
    assert sim.collision_stats()[0] == n0
    sim.close()


@pytest.mark.parametrize("scale", [1e-3, 0.2])
def test_small_write_keeps_the_lists_and_the_trajectory(vx, scale):
    """Shift every offset by scale * l along x (2 scale l of horizon), then
    step through the shell's impact: equal bit for bit to the run that
    rebuilds right after the same write."""
    sc = scenes.hollow_ball(R=12, t=3)
    runs = []
    for force in (False, True):
        sim = vx.Sim(sc)
        sim.step(250)
        st = sim.read_state()
        off = st["offset"].copy()
        off[:, 0] += np.float32(scale * sim.l)
        n0, acc0 = sim.collision_stats()
        sim.write_state(offset=off)
        n1, acc1 = sim.collision_stats()
        if not force:
            if acc0 + 2 * scale * sim.l < 0.9 * sim.l:  # far from the threshold: no rebuild
                assert n1 == n0 and acc1 > acc0
        else:
            sim.rebuild_collisions()
        sim.step(900)
        assert sim.status()[0] == 0
        runs.append(sim.read_state())
        sim.close()
    _same(*runs)


def test_large_write_rebuilds_from_the_written_offsets(vx):
    sc = scenes.hollow_ball(R=10, t=3)
    sc["collide"] = True
    sim = vx.Sim(sc)
    ora = Oracle(sc)
    n0, _ = sim.collision_stats()
    rng = np.random.default_rng(7)
    off = (rng.uniform(-0.45, 0.45, size=(sim.N, 3)) * sc["voxel_size"]).astype(np.float32)
    off[0, 0] = np.float32(0.9 * sc["voxel_size"])   # one voxel moved by most of a voxel: over the threshold
    sim.write_state(offset=off)
    n1, acc1 = sim.collision_stats()
    assert n1 == n0 + 1 and acc1 == 0.0
    gp = {tuple(p) for p in sim.collision_pairs()}
    op = {tuple(p) for p in ora.pairs_from_offsets(off.astype(np.float64))}
    assert len(op) > 100 and gp == op
    sim.close()


def test_population_write_rebuilds_only_the_moved_body(vx):
    """Per-body worlds: a write that moves one body far and leaves the others
    in place flags that body alone; its lists equal the oracle's."""
    sc = scenes.population(n_bodies=6, seed=13, lo=3, hi=8)
    sc["collide"] = True
    sim = vx.Sim(sc)
    ora = Oracle(sc)
    ijk = scenes.canonical_coords(sc)
    st = sim.read_state()
    off = st["offset"].copy()
    rng = np.random.default_rng(3)
    moved = ijk[:, 0] == 2
    off[moved] = (rng.uniform(-0.45, 0.45, size=(int(moved.sum()), 3)) * sc["voxel_size"]).astype(np.float32)
    n0, _ = sim.collision_stats()
    sim.write_state(offset=off)
    assert sim.collision_stats()[0] == n0 + 1
    gp = {tuple(p) for p in sim.collision_pairs()}
    op = {tuple(p) for p in ora.pairs_from_offsets(off.astype(np.float64))}
    assert gp == op
    sim.close()


def test_large_state_round_trip(vx):
    """A state of more than 2^18 voxels: the round trip is exact through
    pageable and through pinned buffers, and a write's largest displacement
    is found wherever it lies (the last voxel of the canonical order too)."""
    torch = pytest.importorskip("torch")
    sim = vx.Sim(scenes.hollow_ball(R=60, t=8))
    assert sim.N >= 1 << 18
    sim.step(5)
    st = sim.read_state()
    rng = np.random.default_rng(2)
    off = (st["offset"] + rng.normal(scale=1e-7, size=st["offset"].shape)).astype(np.float32)
    vel = rng.normal(size=(sim.N, 3)).astype(np.float32)
    w = rng.normal(size=(sim.N, 3)).astype(np.float32)
    n0, acc0 = sim.collision_stats()
    sim.write_state(offset=off, quat=st["quat"], vel=vel, angvel=w, flags=st["flags"])
    back = sim.read_state()
    for k, a in (("offset", off), ("quat", st["quat"]), ("vel", vel), ("angvel", w), ("flags", st["flags"])):
        assert np.array_equal(back[k], a), k
    n1, acc1 = sim.collision_stats()
    d = np.sqrt(np.max(np.sum((off - st["offset"]).astype(np.float32) ** 2, axis=1)))
    assert n1 == n0 and acc1 - acc0 == pytest.approx(2 * d, rel=1e-3)
    pin = {k: torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for k, a in back.items()}
    stream = torch.cuda.Stream()
    sim.write_state_from(**pin, stream=stream, on_device=False, wait=False)
    out = {k: torch.empty_like(t).pin_memory() for k, t in pin.items()}
    sim.read_state_into(**out, stream=stream, on_device=False)
    for k in pin:
        assert torch.equal(out[k], pin[k]), k
    assert sim.collision_stats()[0] == n1
    off2 = back["offset"].copy()
    off2[sim.N - 1, 2] += np.float32(0.9 * sim.l)  # the last voxel
    sim.write_state(offset=off2)
    assert sim.collision_stats()[0] == n1 + 1
    sim.close()
