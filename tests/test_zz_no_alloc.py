"""GPU test of vx_collision_candidates_static, the collision-candidate entry
point that allocates no device memory (for callers that cannot call
cudaMalloc where they need the candidates: a memory arena owning the device
heap, a plug-in given only pre-sized buffers, a loop that must not hit
cudaMalloc's implicit synchronisation).

Its candidate lists must equal those of a simulator's own collision rebuild
(vx_rebuild_collisions + vx_get_collision_pairs) and the FP64 oracle's brute
force for the same FP32 offsets, on two calls in a row (the fixed scratch
array keeps the previous call's contents), and the second call must leave
the device's free memory unchanged.  Inputs the entry point cannot serve
(too many candidates for a voxel, body ids out of range, sizes above its
limits) come back as error codes.  The file is named to be collected last.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_1212_2845_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1212_2845_gb300 import build, vx
    build.build()
    return torch, vx


def scrambled(n, l, seed, amp=0.45):
    rng = np.random.default_rng(seed)
    return (rng.uniform(-amp, amp, size=(n, 3)) * l).astype(np.float32)


def static_pairs(torch, vx, sc, off, bijk, surface):
    """Candidate pairs (canonical indices, i < j) from the allocation-free entry point."""
    idx = np.nonzero(surface)[0]
    S = len(idx)
    lat = (bijk[idx, 1].astype(np.uint32) | bijk[idx, 2].astype(np.uint32) << 11 |
           bijk[idx, 3].astype(np.uint32) << 22).view(np.int32)
    dev = torch.device("cuda")
    t_lat = torch.from_numpy(lat.copy()).to(dev)
    t_off = torch.from_numpy(np.ascontiguousarray(off[idx].T)).to(dev)      # [3, S] planes
    t_body = torch.from_numpy(bijk[idx, 0].astype(np.int32)).to(dev)
    cnt = torch.full((S,), -1, dtype=torch.int32, device=dev)
    cand = torch.full((S, vx.CAND_CAP), -1, dtype=torch.int32, device=dev)
    n_bodies = int(bijk[:, 0].max()) + 1
    stream = torch.cuda.current_stream()
    vx.collision_candidates_static(t_lat, t_off, t_body, S, n_bodies, sc["voxel_size"], cnt, cand, stream)
    cnt, cand = cnt.cpu().numpy(), cand.cpu().numpy()
    pairs = set()
    for s in range(S):
        lst = cand[s, :cnt[s]]
        assert np.all(np.diff(lst) > 0)            # ascending
        for t in lst:
            a, b = int(idx[s]), int(idx[t])
            pairs.add((min(a, b), max(a, b)))
    return pairs


@pytest.mark.parametrize("which", ["ball", "bodies"])
def test_static_candidates_equal_simulator_rebuild(env, which):
    torch, vx = env
    if which == "ball":
        sc = scenes.hollow_ball(R=10, t=3)
    else:
        sc = scenes.population(n_bodies=5, seed=13, lo=3, hi=9)
        sc["collide"] = True
    sim = vx.Sim(sc)
    sim.set_environment(0.0, False, True)
    bijk, _, surface = Oracle(sc, apply_scene=False).topology()
    ora = Oracle(sc)
    for seed in (21, 22):                           # two calls in a row
        off = scrambled(sim.N, sc["voxel_size"], seed)
        sim.write_state(offset=off)
        sim.rebuild_collisions()
        ref = {tuple(int(x) for x in p) for p in sim.collision_pairs()}
        got = static_pairs(torch, vx, sc, off, bijk, surface)
        brute = {tuple(int(x) for x in p) for p in ora.pairs_from_offsets(off.astype(np.float64))}
        assert len(ref) > 20
        assert got == ref == brute
    sim.close()


def test_static_candidates_allocate_nothing(env):
    """The second call on prepared buffers leaves the device's free memory
    exactly as it was (the first call may load the module's code and look up
    the scratch array)."""
    torch, vx = env
    sc = scenes.hollow_ball(R=10, t=3)
    bijk, _, surface = Oracle(sc, apply_scene=False).topology()
    idx = np.nonzero(surface)[0]
    S = len(idx)
    lat = (bijk[idx, 1].astype(np.uint32) | bijk[idx, 2].astype(np.uint32) << 11 |
           bijk[idx, 3].astype(np.uint32) << 22).view(np.int32)
    off = scrambled(len(bijk), sc["voxel_size"], 5)[idx]
    t_lat = torch.from_numpy(lat.copy()).cuda()
    t_off = torch.from_numpy(np.ascontiguousarray(off.T)).cuda()
    cnt = torch.zeros(S, dtype=torch.int32, device="cuda")
    cand = torch.zeros((S, vx.CAND_CAP), dtype=torch.int32, device="cuda")
    vx.collision_candidates_static(t_lat, t_off, None, S, 1, sc["voxel_size"], cnt, cand)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    vx.collision_candidates_static(t_lat, t_off, None, S, 1, sc["voxel_size"], cnt, cand)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert int(cnt.sum()) > 0


def test_static_candidates_report_overflow_and_bad_body_ids(env):
    """60 voxels of one body, lattice sites 4 apart (never excluded), all
    moved onto one point: each has 59 candidates, more than the 48 slots, and
    the call returns VX_ERR_CAPACITY.  A body id outside [0, n_bodies)
    returns VX_ERR_ARG before anything is searched."""
    torch, vx = env
    n, l = 60, 1e-3
    i = 4 * np.arange(n, dtype=np.uint32)
    lat = torch.from_numpy(i.view(np.int32).copy()).cuda()
    off = np.zeros((3, n), np.float32)
    off[0] = (-i.astype(np.float64) * l).astype(np.float32)
    t_off = torch.from_numpy(off).cuda()
    cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    cand = torch.zeros((n, vx.CAND_CAP), dtype=torch.int32, device="cuda")
    with pytest.raises(vx.VxError) as e:
        vx.collision_candidates_static(lat, t_off, None, n, 1, l, cnt, cand)
    assert e.value.code == -7
    body = torch.zeros(n, dtype=torch.int32, device="cuda")
    body[17] = 2
    with pytest.raises(vx.VxError) as e:
        vx.collision_candidates_static(lat, t_off, body, n, 2, l, cnt, cand)
    assert e.value.code == -1 and "surface voxel 17" in str(e.value)
    body[17] = 1                                   # in range: fine (two small groups, spread apart)
    off[0, 30:] += np.float32(0.5)
    vx.collision_candidates_static(lat, torch.from_numpy(off).cuda(), body, n, 2, l, cnt, cand)


def test_static_candidates_reject_oversized_input(env):
    torch, vx = env
    t = torch.zeros(4, dtype=torch.int32, device="cuda")
    planes = torch.zeros((3, 4), dtype=torch.float32, device="cuda")
    cand = torch.zeros((4, vx.CAND_CAP), dtype=torch.int32, device="cuda")
    with pytest.raises(vx.VxError) as e:
        vx.collision_candidates_static(t, planes, t, vx.STATIC_MAX_SURFACE + 1, 1, 1e-3, t, cand)
    assert e.value.code == -1 and "n_surface" in str(e.value)
    with pytest.raises(vx.VxError) as e:
        vx.collision_candidates_static(t, planes, t, 4, vx.STATIC_MAX_BODIES + 1, 1e-3, t, cand)
    assert e.value.code == -1 and "n_bodies" in str(e.value)
