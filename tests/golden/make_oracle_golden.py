"""Write the oracle reference traces used by the GPU parity tests.

Calls only ``oracle/`` (and the seeded workload generator for the instance
parameters).  Usage:  python tests/golden/make_oracle_golden.py [single|voxel IX IY]

* single      -> single_instance_L10.npz : the 1-instance workload (25 kHz sin
                 drive, L = 10, 4 periods x 1000 samples).
* voxel IX IY -> sysmat_L16_vIX_IY.npz   : one voxel of the 32 x 32 system-matrix
                 workload (Lissajous drive, L = 16, 1 warm-up + 1 period of 1632
                 samples).
* highl L     -> highdeg_L{L}.npz        : the high-degree workload instance at
                 degree L (rtol 1e-11, self-convergence against 1e-10: the
                 oracle's dense stage solves of size 3 (L+1)^2 are slow there).

Each file holds the oracle solution at rtol 1e-12 (m, dmdt, the max norm of
the state c at every sample (cmax), phi_hat of the x and y channels over the
last period) and its self-convergence: the same solve at rtol 1e-11, stored as
the relative L2 differences (selfconv_m, selfconv_dmdt, selfconv_phihat) and
the largest state difference over all samples relative to max |c|
(selfconv_c).  The two solves run in two spawned processes.
"""
import multiprocessing as mp
import os
import sys

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")         # one BLAS thread per solve (set before numpy loads)
import numpy as np                          # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import physics, solve                       # noqa: E402
from paper_2106_08040_gb300 import workloads            # noqa: E402  (input generator only)

RTOL_GOLD = 1e-12
RTOL_CHECK = 1e-11
RTOL_HIGHL = (1e-11, 1e-10)
CHANNELS = [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]]


def to_oracle(dspec, rec):
    drive = physics.Drive(amp=dspec.amp, freq=dspec.freq, phase=dspec.phase, period=dspec.period)
    sched = solve.Schedule(dspec.samples_per_period, dspec.warmup_periods, dspec.output_periods)
    inst = solve.Instance(h_off=tuple(rec["h_off"]), theta=float(rec["theta"]), phi=float(rec["phi"]),
                          K=float(rec["K"]), d=float(rec["d"]), L=int(rec["L"]))
    return drive, sched, inst


def _job(args):
    kind, ix, iy, rtol = args
    if kind == "single":
        dspec, inst = workloads.single_instance_workload()
        rec = inst[0]
    elif kind == "highl":
        dspec, inst = workloads.high_degree_workload(ix)
        rec = inst[0]
    else:
        dspec, inst = workloads.system_matrix_workload()
        rec = inst[iy * 32 + ix]
    drive, sched, oi = to_oracle(dspec, rec)
    r = solve.solve_instance(physics.Material(), drive, oi, sched, rtol=rtol, return_state=True)
    r["phihat"] = solve.phi_hat(r["dmdt"], CHANNELS, dspec.samples_per_period, dspec.samples_per_period // 2)
    return r


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def main(argv):
    if not argv or argv[0] not in ("single", "voxel", "highl"):
        raise SystemExit(__doc__)
    kind = argv[0]
    ix, iy = (int(argv[1]), int(argv[2])) if kind == "voxel" else ((int(argv[1]), 0) if kind == "highl" else (0, 0))
    r_gold, r_check = RTOL_HIGHL if kind == "highl" else (RTOL_GOLD, RTOL_CHECK)
    ctx = mp.get_context("spawn")
    with ctx.Pool(2) as pool:
        gold, check = pool.map(_job, [(kind, ix, iy, r_gold), (kind, ix, iy, r_check)])
    cmax = np.abs(gold["c"]).max(axis=1)
    extra = dict(selfconv_m=rel(check["m"], gold["m"]), selfconv_dmdt=rel(check["dmdt"], gold["dmdt"]),
                 selfconv_phihat=rel(check["phihat"], gold["phihat"]),
                 selfconv_c=float(np.abs(check["c"] - gold["c"]).max() / cmax.max()), rtol_check=r_check)
    name = {"single": "single_instance_L10.npz", "voxel": "sysmat_L16_v%d_%d.npz" % (ix, iy),
            "highl": "highdeg_L%d.npz" % ix}[kind]
    np.savez(os.path.join(HERE, name), m=gold["m"], dmdt=gold["dmdt"], t=gold["t"], cmax=cmax,
             phihat=gold["phihat"], steps=gold["steps"], rtol=r_gold, ix=ix, iy=iy, **extra)
    print(name, extra, "steps", gold["steps"], check["steps"])


if __name__ == "__main__":
    main(sys.argv[1:])
