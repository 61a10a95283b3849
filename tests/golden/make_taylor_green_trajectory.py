"""Writes taylor_green_64x128_trajectory.npz: the FP64 oracle's trajectory of the Taylor-Green suspension
(64 vesicles x 128 points, 10% area fraction, dt = 1e-3; workloads.taylor_green, seed 2) over 500 plain
steps (Algorithm 1 with exact operators), sampled at steps 1, 2, 10, 50, 100, 200, 300, 400, 500 for every
eighth vesicle: positions (CSR blocks x then y per vesicle), tension, and the running count of
area/length corrections of the whole suspension.

Only oracle/ computes here (the workload module only draws the inputs). Each step is the oracle's
Suspension.step for the plain mode: u^n from Suspension.interaction_velocity, then oracle.step.
advance_vesicle for every vesicle given its u^n, the vesicles spread over a pool of spawned processes
(they are independent given u^n). About half an hour on 8 host cores.

    python tests/golden/make_taylor_green_trajectory.py [processes]
"""
import multiprocessing as mp
import os
import sys
import time

# one BLAS thread per process (the processes already fill the cores)
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

SNAPSHOTS = (1, 2, 10, 50, 100, 200, 300, 400, 500)
SAMPLE = tuple(range(0, 64, 8))
OUT = os.path.join(HERE, "taylor_green_64x128_trajectory.npz")


def _advance(job):
    from oracle.step import advance_vesicle
    x, y, ux, uy, A0, L0, p = job
    return advance_vesicle(x, y, ux, uy, A0, L0, p)


def main():
    from oracle.step import Params, Suspension
    from paper_2606_25569_b300.workloads import taylor_green
    procs = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count()
    wl = taylor_green()
    p = Params(kappa=wl.kappa, mu=wl.mu, dt=wl.dt, flow_kind=wl.flow_kind, flow_p=wl.flow_p, corr_tol=0.01)
    s = Suspension(wl.xs, wl.ys, p)
    xy, sig, corr = [], [], []
    t0 = time.time()
    with mp.get_context("spawn").Pool(procs) as pool:
        for n in range(1, max(SNAPSHOTS) + 1):
            u = s.interaction_velocity()
            jobs = [(x, y, u[v][0], u[v][1], s.A0[v], s.L0[v], p) for v, (x, y) in enumerate(zip(s.xs, s.ys))]
            res = pool.map(_advance, jobs)
            s.xs = [r[0] for r in res]
            s.ys = [r[1] for r in res]
            s.sig = [r[2] for r in res]
            s.corrections += sum(int(r[3]) for r in res)
            if n in SNAPSHOTS:
                xy.append(np.concatenate([np.concatenate([s.xs[v], s.ys[v]]) for v in SAMPLE]))
                sig.append(np.concatenate([s.sig[v] for v in SAMPLE]))
                corr.append(s.corrections)
                print("step %d: %.0f s, corrections %d" % (n, time.time() - t0, s.corrections), flush=True)
    np.savez_compressed(OUT, steps=np.array(SNAPSHOTS), vesicles=np.array(SAMPLE), xy=np.array(xy),
                        sigma=np.array(sig), corrections=np.array(corr))


if __name__ == "__main__":
    main()
