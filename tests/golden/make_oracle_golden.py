"""Write the oracle reference traces used by the GPU parity tests.

Calls only ``oracle/`` (and the seeded workload generator for the instance
parameters).  Usage:  python tests/golden/make_oracle_golden.py [single|voxel IX IY]

* single      -> single_instance_L10.npz : the 1-instance workload (25 kHz sin
                 drive, L = 10, 4 periods x 1000 samples), rtol 1e-12.
* voxel IX IY -> sysmat_L16_vIX_IY.npz   : one voxel of the 32 x 32 system-matrix
                 workload (Lissajous drive, L = 16, 1 warm-up + 1 period of 1632
                 samples), rtol 1e-10.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import physics, solve                       # noqa: E402
from paper_2106_08040_gb300 import workloads            # noqa: E402  (input generator only)


def to_oracle(dspec, rec):
    drive = physics.Drive(amp=dspec.amp, freq=dspec.freq, phase=dspec.phase, period=dspec.period)
    sched = solve.Schedule(dspec.samples_per_period, dspec.warmup_periods, dspec.output_periods)
    inst = solve.Instance(h_off=tuple(rec["h_off"]), theta=float(rec["theta"]), phi=float(rec["phi"]),
                          K=float(rec["K"]), d=float(rec["d"]), L=int(rec["L"]))
    return drive, sched, inst


def main(argv):
    mat = physics.Material()
    if argv[0] == "single":
        dspec, inst = workloads.single_instance_workload()
        drive, sched, oi = to_oracle(dspec, inst[0])
        r = solve.solve_instance(mat, drive, oi, sched, rtol=1e-12)
        np.savez(os.path.join(HERE, "single_instance_L10.npz"), m=r["m"], dmdt=r["dmdt"], t=r["t"],
                 steps=r["steps"], rtol=1e-12)
    elif argv[0] == "voxel":
        ix, iy = int(argv[1]), int(argv[2])
        dspec, inst = workloads.system_matrix_workload()
        drive, sched, oi = to_oracle(dspec, inst[iy * 32 + ix])
        r = solve.solve_instance(mat, drive, oi, sched, rtol=1e-10)
        np.savez(os.path.join(HERE, "sysmat_L16_v%d_%d.npz" % (ix, iy)), m=r["m"], dmdt=r["dmdt"], t=r["t"],
                 steps=r["steps"], rtol=1e-10, ix=ix, iy=iy)
    else:
        raise SystemExit(__doc__)


if __name__ == "__main__":
    main(sys.argv[1:])
