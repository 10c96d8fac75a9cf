"""The shared-memory-resident form (vx_set_batching(VX_GROUPS_RESIDENT)):
groups of whole bodies kept in the shared memory of a CTA cluster for all
steps of a launch.  It computes the per-step kernels' arithmetic in their
order, so its states must equal theirs bit for bit: on a single small
lattice spread over a cluster of 8 CTAs (the cantilever), on a population
of uneven bodies (several groups per cluster), on design bodies with
per-voxel stiffness (one body across a cluster of two CTAs), on one large
body across a wider cluster, with external forces, through captured graph
replays, and on the FP64 oracle's trajectory within the stated tolerance, with the
bond phase split either way (a thread per bond or a thread per voxel)."""
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


def per_step(vx, sc, steps):
    sim = vx.Sim(sc)
    sim.set_multistep(0)
    sim.step(steps)
    out = sim.read_state()
    sim.close()
    return out


def forced_cantilever():
    sc = scenes.cantilever(n=(12, 6, 5))
    ijk = scenes.canonical_coords(sc)
    F = np.zeros((len(ijk), 3))
    F[ijk[:, 1] == 11, 2] = -2e-4                     # a downward load on the free end
    sc["force"] = scenes.f32(F)
    return sc


CASES = {
    "cantilever": (scenes.cantilever, 300),
    "population": (lambda: scenes.population(n_bodies=23, seed=17, lo=2, hi=12), 250),
    "design_bodies": (lambda: scenes.design_population(n_bodies=6, n=12, seed=5), 200),
    "large_body": (lambda: scenes.hetero_block(dims=(22, 20, 18), seed=4), 120),
    "forced": (forced_cantilever, 300),
}


@pytest.mark.parametrize("split", ["auto", "bond", "voxel"])
@pytest.mark.parametrize("which", list(CASES))
def test_resident_form_bitwise_equals_per_step_launches(vx, which, split):
    mk, steps = CASES[which]
    sc = mk()
    ref = per_step(vx, sc, steps)
    sim = vx.Sim(sc)
    sim.set_batching({"auto": vx.GROUPS_RESIDENT, "bond": vx.GROUPS_RESIDENT_BOND,
                      "voxel": vx.GROUPS_RESIDENT_VOXEL}[split])
    sim.step(steps // 3)                       # two launches (odd and even step counts)
    sim.step(steps - steps // 3)
    assert sim.status()[0] == 0
    assert sim.step_count == steps
    out = sim.read_state()
    for k in ("offset", "quat", "vel", "angvel", "flags"):
        assert np.array_equal(out[k].view(np.uint8), ref[k].view(np.uint8)), k
    sim.set_batching(0)
    sim.step(3)                                # back to per-step launches
    assert sim.step_count == steps + 3
    sim.close()


def test_resident_graph_replays_continue_the_rollout(vx):
    sc = scenes.population(n_bodies=23, seed=17, lo=2, hi=12)
    sc["act_period"] = 40
    ref = per_step(vx, sc, 21)
    sim = vx.Sim(sc)
    sim.set_batching(vx.GROUPS_RESIDENT)
    sim.graph_capture(7)
    for _ in range(3):
        sim.graph_launch()
    assert sim.status()[0] == 0 and sim.step_count == 21
    out = sim.read_state()
    for k in ("offset", "quat", "vel", "angvel", "flags"):
        assert np.array_equal(out[k].view(np.uint8), ref[k].view(np.uint8)), k
    sim.close()


def test_resident_cantilever_follows_the_oracle(vx):
    """The cantilever (configuration 1) for its 1,000 steps in one resident
    launch: positions within 1e-5 of the body diagonal of the FP64 oracle."""
    sc = scenes.cantilever()
    sim = vx.Sim(sc)
    ora = Oracle(sc)
    ora.set_dt(np.float32(ora.dt()))
    sim.set_batching(vx.GROUPS_RESIDENT)
    sim.step(1000)
    ora.step(1000)
    g, o = sim.state(), ora.state()
    diag = np.linalg.norm(np.ptp(o["pos"], axis=0))
    err = np.abs(g["pos"] - o["pos"]).max() / diag
    print(f"resident cantilever: 1000 steps, max position error / diagonal {err:.2e}")
    assert err < 1e-5
    sim.close()


def test_resident_form_refuses_bodies_beyond_16_ctas(vx):
    sc = scenes.cantilever(n=(40, 40, 20))               # 32,000 voxels in one body
    sim = vx.Sim(sc)
    with pytest.raises(vx.VxError) as e:
        sim.set_batching(vx.GROUPS_RESIDENT)
    assert e.value.code == -6
    sim.close()
