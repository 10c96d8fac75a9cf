"""Writes tests/golden/long_parity.npz: FP64 oracle states after the long
runs for which the tolerances are stated, at 1,024 sampled voxels per run:

  hetero_block_64x64x32   10,000 steps (the full heterogeneous-block run)
  hollow_ball_R40_t4       2,000 steps (a shell drop through impact and bounce)
  hollow_ball_R20_t4      20,000 steps (a scaled shell for the whole drop)
  population_16           20,000 steps (16 bodies of the population)
  hollow_ball_R100_t8      1,000 steps (the full 926,584-voxel ball drop,
                          through the impact near step 370 and ~27 rebuilds
                          of the candidate lists)

Every value comes from the oracle alone (the same scene recipes the GPU
tests build, the oracle's own timestep rounded to FP32 as the kernels step
with it).  Each run is kept in its own file as it finishes, then all are
combined.  Run from the repository root, about 25 minutes on 5 cores:

    python tests/golden/make_long_parity.py              # every case
    python tests/golden/make_long_parity.py NAME ...     # these cases, merged into the stored file
"""
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import Oracle  # noqa: E402
from paper_1212_2845_gb300 import scenes  # noqa: E402

CASES = {
    "hetero_block_64x64x32": ("hetero_block", {}, 10000),
    "hollow_ball_R40_t4": ("hollow_ball", {"R": 40, "t": 4}, 2000),
    "hollow_ball_R20_t4": ("hollow_ball", {"R": 20, "t": 4}, 20000),
    "population_16": ("population", {"n_bodies": 16}, 20000),
    "hollow_ball_R100_t8": ("hollow_ball", {"R": 100, "t": 8}, 1000),
}
N_SAMPLE = 1024


def scene(name):
    fn, kw, steps = CASES[name]
    return getattr(scenes, fn)(**kw), steps


def body_diagonals(sc, pos):
    ijk = scenes.canonical_coords(sc)
    d = np.zeros(len(pos))
    for b in np.unique(ijk[:, 0]):
        m = ijk[:, 0] == b
        d[m] = np.linalg.norm(np.ptp(pos[m], axis=0)) if m.sum() > 1 else sc["voxel_size"]
    return d


def run(name):
    part = os.path.join(HERE, f".long_parity_{name}.npz")
    if os.path.exists(part):
        return part
    sc, steps = scene(name)
    o = Oracle(sc)
    o.set_dt(np.array([np.float32(o.dt(b)) for b in range(o.n_bodies)], dtype=np.float64))
    o.step(steps)
    s = o.state()
    rng = np.random.default_rng(2024)
    idx = np.sort(rng.choice(o.N, size=min(N_SAMPLE, o.N), replace=False))
    diag = body_diagonals(sc, s["pos"])
    np.savez(part, steps=steps, idx=idx, pos=s["pos"][idx], static=s["static"][idx].astype(np.uint8),
             diag=diag[idx], max_disp=float(np.abs(s["pos"] - o.anchors(sc)).max()),
             n_rebuilds=o.n_rebuilds())
    return part


def main(names):
    names = names or list(CASES)
    with mp.get_context("spawn").Pool(len(names)) as pool:
        parts = pool.map(run, names)
    out = os.path.join(HERE, "long_parity.npz")
    arrays = {}
    if os.path.exists(out):                         # keep the stored cases not rerun
        with np.load(out) as r:
            arrays = {k: r[k] for k in r.files if k.split("/")[0] not in names}
    for name, part in zip(names, parts):
        with np.load(part) as r:
            for k in r.files:
                arrays[f"{name}/{k}"] = r[k]
    np.savez_compressed(out, **arrays)
    for part in parts:
        os.remove(part)


if __name__ == "__main__":
    main(sys.argv[1:])
