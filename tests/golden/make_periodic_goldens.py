"""Write the stored oracle solutions of the periodic workloads (test fixtures).

    python tests/golden/make_periodic_goldens.py [wells512] [batch16384] [wells1024]

Each case runs the plain FP64 oracle (oracle/periodic.py: direct O(M^2) DFT
sums, Table 1 weights, Richardson start-up, phases evaluated directly) on the
seeded synthetic inputs of synth/ and stores the solution at a few steps on a
strided subgrid, with the inputs on the same subgrid and the scalar
parameters (so a test can check that the generator still produces them):

  periodic_2d_wells_512.npz    the 2D wells workload (512^2, dt = 1e-3, the
                               8th-order scheme), seed 2, all 2000 steps;
                               u at steps 10, 500, 1000, 2000 on every 4th point
  periodic_1d_16384.npz        an uneven-batch member with N = 16384 (4 cosine
                               modes, pulse), 20 steps; u at 10, 20, every 8th point
  periodic_2d_wells_1024.npz   the 2D wells workload at 1024^2, seed 12, 9 steps;
                               u at 9, every 8th point

`--refresh-inputs` rewrites only the stored inputs of existing files.
Nothing here runs the CUDA library.  The full 2000-step 512^2 run takes a few
minutes on 8 cores (two dense 512 x 512 complex products per transform).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle.periodic import oracle_for  # noqa: E402


def input_fingerprint(inst, stride):
    """The seeded inputs on the stored subgrid and the scalar parameters: a
    test compares them with tolerance (the generator's libm results differ in
    the last bits between machines)."""
    sl = tuple(slice(None, None, stride) for _ in inst.shape)
    p = inst.pulse
    return {"u0_sample": inst.u0[sl], "V0_sample": inst.V0[sl],
            "params": np.array([inst.dt, inst.nsteps, p.A0, p.omega, p.T_pulse, *p.direction], dtype=np.float64)}


def batch_member_with(M: int, seed: int = 4, nsteps: int = 20):
    for i in range(4096):
        inst = synth.periodic_1d_batch_member(i, seed=seed, nsteps=nsteps)
        if inst.shape[0] == M:
            return i, inst
    raise RuntimeError("no member of that size")


def run(inst, keep, stride, path, extra):
    t0 = time.time()
    u, kept = oracle_for(inst).solve(inst.u0, inst.nsteps, keep=set(keep))
    sl = tuple(slice(None, None, stride) for _ in inst.shape)
    arrays = {f"u_{n}": kept[n][sl] for n in keep}
    np.savez_compressed(path, key=np.array(inst.name), steps=np.array(sorted(keep)),
                        stride=np.array(stride), shape=np.array(inst.shape), **extra, **arrays,
                        **input_fingerprint(inst, stride))
    print(f"{os.path.basename(path)}: {inst.name}, {inst.nsteps} steps, {time.time() - t0:.0f} s")


def refresh_inputs(path, inst):
    """Rewrite only the key and the input fingerprint of an existing file (the
    stored oracle solutions are kept as they are)."""
    g = dict(np.load(path))
    g["key"] = np.array(inst.name)
    g.update(input_fingerprint(inst, int(g["stride"])))
    np.savez_compressed(path, **g)


def main(argv):
    if argv and argv[0] == "--refresh-inputs":
        refresh_inputs(os.path.join(HERE, "periodic_2d_wells_512.npz"),
                       synth.periodic_2d_wells(seed=2, M=512, dt=1e-3, nsteps=2000))
        refresh_inputs(os.path.join(HERE, "periodic_1d_16384.npz"), batch_member_with(16384)[1])
        refresh_inputs(os.path.join(HERE, "periodic_2d_wells_1024.npz"),
                       synth.periodic_2d_wells(seed=12, M=1024, dt=1e-3, nsteps=9))
        return
    which = argv or ["wells512", "batch16384", "wells1024"]
    if "wells512" in which:
        inst = synth.periodic_2d_wells(seed=2, M=512, dt=1e-3, nsteps=2000)
        run(inst, [10, 500, 1000, 2000], 4, os.path.join(HERE, "periodic_2d_wells_512.npz"), {"seed": np.array(2)})
    if "batch16384" in which:
        i, inst = batch_member_with(16384)
        run(inst, [10, 20], 8, os.path.join(HERE, "periodic_1d_16384.npz"), {"member": np.array(i), "seed": np.array(4)})
    if "wells1024" in which:
        inst = synth.periodic_2d_wells(seed=12, M=1024, dt=1e-3, nsteps=9)
        run(inst, [9], 8, os.path.join(HERE, "periodic_2d_wells_1024.npz"), {"seed": np.array(12)})


if __name__ == "__main__":
    main(sys.argv[1:])
