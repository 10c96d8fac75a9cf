"""Failure detection without GPU faults: every failure is made on the host
(a NaN written into the state, a device allocation cap, a grid barrier told
to wait for CTAs that do not exist with a small wait budget) and must come
back as an error code, with the context still usable afterwards."""
import os

import numpy as np
import pytest

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


def test_barrier_wait_runs_out_and_reports_timeout(vx):
    sc = scenes.hetero_block(dims=(20, 18, 12), seed=9)
    sim = vx.Sim(sc)
    assert sim.tiling()["n_tiles"] > 1                 # several CTAs meet at the barrier
    sim.set_multistep(2)                               # the cooperative grid launch (not the resident form)
    sim.set_barrier_limits(max_spins=2000, phantom_ctas=1)
    with pytest.raises(vx.VxError) as e:
        sim.step(5)
    assert e.value.code == -5
    assert sim.status()[0] == -5
    # the context is usable: back to normal limits, fresh state, steps succeed
    sim.set_barrier_limits(0, 0)
    sim.reset()
    sim.step(5)
    assert sim.status()[0] == 0
    sim.close()


def test_rebuild_barrier_wait_runs_out_and_reports_timeout(vx):
    """A forced candidate rebuild whose grid barriers wait for a CTA that
    does not exist gives up after the small budget and returns
    VX_ERR_TIMEOUT; after a reset with normal limits it rebuilds again."""
    sc = scenes.hollow_ball(R=12, t=3)
    sim = vx.Sim(sc)
    n_pairs = len(sim.collision_pairs())
    sim.set_barrier_limits(max_spins=2000, phantom_ctas=1)
    with pytest.raises(vx.VxError) as e:
        sim.rebuild_collisions()
    assert e.value.code == -5
    sim.set_barrier_limits(0, 0)
    sim.reset()
    sim.rebuild_collisions()
    assert len(sim.collision_pairs()) == n_pairs
    sim.close()


def test_nan_in_the_input_state_is_reported_as_unstable(vx):
    sc = scenes.random_blob((5, 4, 3), seed=4)
    sim = vx.Sim(sc)
    vel = np.zeros((sim.N, 3), np.float32)
    vel[7, 1] = np.nan
    sim.write_state(vel=vel)
    with pytest.raises(vx.VxError) as e:
        sim.step(3)
    assert e.value.code == -4
    st, bad_step, bad_voxel = sim.status()
    assert st == -4 and bad_step == 0
    sim.reset()
    sim.step(3)
    sim.close()


def test_device_allocation_cap_gives_out_of_memory(vx):
    sc = scenes.hetero_block(dims=(24, 24, 16), seed=3)
    os.environ["VX_DEVICE_ALLOC_CAP"] = "65536"
    try:
        with pytest.raises(vx.VxError) as e:
            vx.Sim(sc)
        assert e.value.code == -3
    finally:
        del os.environ["VX_DEVICE_ALLOC_CAP"]
    sim = vx.Sim(sc)                                   # no cap: fine
    sim.step(2)
    sim.close()
