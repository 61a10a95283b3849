#!/usr/bin/env python
"""Benchmark of the plain boundary-integral vesicle step on one B300 (vesicle-steps/s).

Workload: the dense Poiseuille suspension of Sec. 5.5 -- 2000 vesicles x 64 points, 30% area
fraction, channel of width 1, reduced area 0.65, Ca = 2, Cn = 0.025 -- drawn synthetically by
paper_2606_25569_b300.workloads.poiseuille_dense (seed 5). One step = one pass of the whole
hot path through libvesb300.so (force, far field with the near-field mask, advection,
relaxation, redistribution, tension, correction).

Prints one JSON line. Run as `python bench.py --gpus 1 --steps K --warmup W`, or under
torch.distributed.run for N > 1 (independent replicas, weak scaling). `--impl reference`
times the FP64 CPU oracle on a bounded sample of the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

# the oracle baseline runs one BLAS thread per process: pin BLAS threads before numpy loads
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "vesicle-steps/s: hybrid vs plain BIE on one B300 at shape error <=1e-2"
UNIT = "vesicle-steps/s"
MUFU_PER_CLK_SM = 16      # special-function results per clock per SM (4 per sub-partition)
FP32_LANES_PER_CLK_SM = 128  # FP32 lane operations per clock per SM (4 sub-partitions x 32 lanes; single and
                             # paired float2 instructions alike)
N_SM = 148
# k_farfield_sym: FP32 lane operations per unordered pair of points, both reactions (r 2, |r|^2 2, row
# reaction 7, column reaction 7), besides lg2 and rcp on the special-function unit; the log argument's
# per-pair scale rides on the coordinates and costs none
FFS_FP32_PER_PAIR = 18
# DRAM bytes per point of one far-field launch: ncu dram__bytes of k_farfield_f32 on the 1200 x 64 dense
# Poiseuille suspension (2.82 MB for 76,800 points; sources, centres and outputs, every re-read hits L2)
FF_DRAM_BYTES_PER_POINT = 2.82e6 / 76800
# DRAM bytes of one k_farfield_sym launch at 2000 x 64 (ncu dram__bytes_read.sum + dram__bytes_write.sum,
# one-pass capture of the bench workload with chunks of 16 vesicles: 3.19 MB read, 195.51 MB written, mostly
# the per-chunk partial sums that do not stay in L2)
FFS_DRAM_READ, FFS_DRAM_WRITE = 3.19e6, 195.51e6
FFS_DRAM_SOURCE = "ncu dram__bytes_read.sum + dram__bytes_write.sum, one-pass capture at 2000 x 64"
# learned advection and tension: velocity modes expanded and column modes kept, training epochs
FLOW_KF, FLOW_KOUT, FLOW_EPOCHS = 8, 24, 60
# hybrid training data and schedule: snapshots (15 steps apart) of a differently seeded suspension, epochs of
# the relaxation network, exact steps every HYBRID_EVERY steps (learned relaxation only) or FLOW_EVERY (with
# the learned advection and tension)
HYBRID_SNAPSHOTS, HYBRID_EPOCHS, HYBRID_EVERY, FLOW_EVERY = 128, 100, 3, 2
# learned near field: every density mode below the Nyquist one (the membrane force's high modes carry most of
# the near-field correction: on the oracle, keeping modes <= 24 of a 64-point vesicle leaves 20% of it out)
NEAR_SNAPSHOTS, NEAR_EPOCHS = 16, 40
# IVNet relaxation map: C channels, n_b blocks (0.43 M parameters; the paper's relaxation network has 0.6 M)
IV_C, IV_NB, IV_EPOCHS = 64, 8, 40


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="vesb300", choices=["vesb300", "reference"])
    ap.add_argument("--M", type=int, default=2000)
    ap.add_argument("--N", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--farfield-multipole", action="store_true",
                    help="time the plain step with the vesicle-multipole far field (not the headline configuration)")
    ap.add_argument("--no-hybrid", action="store_true", help="skip the learned-relaxation (hybrid) arm")
    ap.add_argument("--no-farfield-alone", action="store_true", help="skip the far field alone on the 2000 x 128 box")
    ap.add_argument("--no-near-arm", action="store_true", help="skip the plain step with near pairs")
    ap.add_argument("--no-uneven-arm", action="store_true", help="skip the plain step with 32/64/128-point vesicles")
    ap.add_argument("--no-implicit-arm", action="store_true", help="skip the fully implicit (GMRES) step")
    ap.add_argument("--no-near-learned-arm", action="store_true", help="skip the learned near field")
    ap.add_argument("--no-ivnet-arm", action="store_true", help="skip the IVNet relaxation map")
    ap.add_argument("--hybrid-steps", type=int, default=1000, help="steps over which the hybrid shape error is taken")
    ap.add_argument("--burn-in", type=int, default=300, help="steps before the steady-state measurement (0: skip)")
    return ap.parse_args()


def workload(args):
    from paper_2606_25569_b300.workloads import poiseuille_dense
    return poiseuille_dense(M=args.M, N=args.N, seed=5)


def config_of(wl, args, extra=None):
    c = {"workload": "dense Poiseuille suspension, %d vesicles x %d points, 30%% area fraction, "
                     "channel width 1, reduced area 0.65, Ca 2, Cn 0.025" % (wl.M, args.N),
         "mode": "plain BIE step (value); the hybrid learned-relaxation step is reported under 'hybrid'",
         "near_field": "mask + five-layer RBF correction (exact layer velocities)",
         "dt": wl.dt, "farfield": "fp32 compensated", "l2": "working set > L2 (no flush needed)",
         "launch": "each step replayed from a captured CUDA graph"}
    if extra:
        c.update(extra)
    return c


# ------------------------------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------ roofline
def kernel_flops(name, N, M):
    """Algorithmic FP64 flops of one launch over M vesicles of N points (dense operator algebra)."""
    n3 = float(N) ** 3
    table = {
        "k_bgemm<OpT>": 8 * n3, "k_bgemm<OpL>": 4 * n3, "k_bgemm<OpD2>": 2 * n3, "k_bgemm<OpD4>": 2 * n3,
        "k_bgemm<OpB>": 4 * n3, "k_bgemm<OpPB>": 8 * n3, "k_bgemm<OpA>": 8 * n3,
        "k_lu<A>": 2.0 / 3.0 * (2 * N) ** 3, "k_lu<L>": 2.0 / 3.0 * n3, "k_lu_solve_cols": 4 * n3,
    }
    return table.get(name, 0.0) * M


def measured_fp64_tflops(torch):
    """cuBLAS DGEMM rate measured here: the FP64 roofline denominator (no FP64 figure is
    supplied with the machine's measured peaks)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e9
    for _ in range(3):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        torch.matmul(a, b)
        e.record()
        torch.cuda.synchronize()
        best = min(best, s.elapsed_time(e))
    del a, b
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


# ------------------------------------------------------------------------------------------ oracle
_ORACLE_SOURCES = None


def _oracle_init(xs, ys, fx, fy, mu):
    """Worker set-up: every source point of the suspension with its density (for the far-field sample)."""
    global _ORACLE_SOURCES
    _ORACLE_SOURCES = (xs, ys, fx, fy, mu)


def _oracle_vesicles(job):
    """One oracle plain step of a sub-suspension (its own vesicles' mutual far field included); seconds."""
    from oracle.step import Params, Suspension
    xs, ys, pv = job
    sub = Suspension(xs, ys, Params(**pv))
    t0 = time.perf_counter()
    sub.step()
    return time.perf_counter() - t0


def _oracle_targets(tg):
    """The oracle's far field at the targets tg against every source; seconds."""
    from oracle.farfield import far_field
    xs, ys, fx, fy, mu = _ORACLE_SOURCES
    t0 = time.perf_counter()
    far_field(xs, ys, fx, fy, mu, near_mask=True, targets=tg)
    return time.perf_counter() - t0


def oracle_pool(wl, procs):
    """A spawned pool of `procs` oracle processes holding the workload's sources and densities (the
    forces of zero tension), started and warmed up (imports done); None for procs = 1."""
    import multiprocessing as mp
    from oracle.spectral import force
    fx, fy = [], []
    for x, y in zip(wl.xs, wl.ys):
        a, b = force(x, y, np.zeros(len(x)), wl.kappa)
        fx.append(a)
        fy.append(b)
    _oracle_init(wl.xs, wl.ys, fx, fy, wl.mu)
    if procs == 1:
        return None
    pool = mp.get_context("spawn").Pool(procs, initializer=_oracle_init, initargs=(wl.xs, wl.ys, fx, fy, wl.mu))
    pool.map(_oracle_targets, [np.arange(2) for _ in range(procs)])
    return pool


def oracle_sample(wl, n_ves=24, n_targets=2048, procs=1, pool=None):
    """Time the FP64 oracle on a bounded sample of the workload and extrapolate one full step.

    Per-vesicle part: oracle steps of n_ves vesicles per process (each process a sub-suspension of
    consecutive vesicles; their mutual far field is included, negligible). Far field: n_targets sampled
    targets per process against all sources. With procs > 1 the processes (spawned, one BLAS thread each)
    run at once on the host cores, and a part's time is the slowest process's. Full step time =
    M * t_vesicle + P * t_target, t_vesicle and t_target the part's time over the units all processes
    handled.
    """
    P = int(sum(len(x) for x in wl.xs))
    pv = dict(kappa=wl.kappa, mu=wl.mu, dt=wl.dt, flow_kind=wl.flow_kind, flow_p=wl.flow_p, near_field=True)
    stride = max(1, wl.M // (n_ves * procs))
    jobs = []
    for k in range(procs):
        idx = [(k * n_ves + i) * stride % wl.M for i in range(n_ves)]
        jobs.append(([wl.xs[i] for i in idx], [wl.ys[i] for i in idx], pv))
    tg = np.linspace(0, P - 1, n_targets * procs).astype(np.int64)
    tgs = [tg[k::procs] for k in range(procs)]
    own = pool is None and procs > 1
    if own or (procs == 1 and _ORACLE_SOURCES is None):
        pool = oracle_pool(wl, procs)
    try:
        if procs == 1:
            t_v = _oracle_vesicles(jobs[0]) / n_ves
            t_t = _oracle_targets(tgs[0]) / n_targets
        else:
            t_v = max(pool.map(_oracle_vesicles, jobs)) / (n_ves * procs)
            t_t = max(pool.map(_oracle_targets, tgs)) / (n_targets * procs)
    finally:
        if own:
            pool.close()
            pool.join()
    full = wl.M * t_v + P * t_t
    return {"value": wl.M / full, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": "FP64 numpy oracle in %d process%s of one BLAS thread: plain steps of %d of the %d vesicles "
                      "+ far field at %d of %d targets against all sources; one full step extrapolated linearly "
                      "(%.1f s)" % (procs, "es" if procs > 1 else "", n_ves * procs, wl.M, n_targets * procs, P,
                                    full)}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------------------------------ main
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload(args)
    procs = host_cores()
    pool = oracle_pool(wl, procs)
    for _ in range(args.warmup):
        oracle_sample(wl, n_ves=1, n_targets=32, procs=procs, pool=pool)
    vals, times = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle_sample(wl, n_ves=2, n_targets=96, procs=procs, pool=pool)
        times.append(time.perf_counter() - t0)
        vals.append(r["value"])
    if pool is not None:
        pool.close()
        pool.join()
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wl.M / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(wl, args, {"impl": "FP64 CPU oracle (numpy), sampled", "mode": "plain BIE step",
                                           "farfield": "fp64 brute force (oracle)",
                                           "launch": "numpy on the host cores, one vesicle at a time"}),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": "per step: %d processes (one per host core, one BLAS thread each), each an "
                                       "oracle plain step of 2 vesicles + far field at 96 targets against all "
                                       "sources, extrapolated to the full step" % procs},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def farfield_alone(stream, reps=10):
    """The far-field sum alone on the 2000 x 128 box (256,000 sources and targets, all pairs of different
    vesicles, no near mask) through vs_farfield_eval: the symmetric kernel (precision 0) and the per-target
    kernel (precision 3), CUDA events over `reps` evaluations after 3 warm-up ones."""
    import torch
    from paper_2606_25569_b300 import binding
    from paper_2606_25569_b300.workloads import farfield_box
    wl, fx, fy = farfield_box()
    off = wl.offsets
    xy = torch.as_tensor(wl.flat_xy(), device="cuda")
    f = torch.as_tensor(np.concatenate([np.concatenate([a, b]) for a, b in zip(fx, fy)]), device="cuda")
    u = torch.empty(2 * int(off[-1]), dtype=torch.float64, device="cuda")
    pairs = float(off[-1]) ** 2 - float(np.sum(wl.counts.astype(np.float64) ** 2))
    out = {"workload": "far field alone: 2000 vesicles x 128 points in a 20 x 20 box, densities N(0,1)",
           "ordered_pairs": pairs, "unit": "pairs/s"}
    P = int(off[-1])
    for name, prec in (("symmetric", 0), ("per_target", 3), ("symmetric_phased", 0)):
        if name == "symmetric_phased":  # partial sums bounded to 32 chunk slots a point (groups of 32 chunks)
            os.environ["VS_FFS_SLOT_BYTES"] = str(32 * P * 16)
        plan = binding.FarFieldPlan(off, mu=1.0, near_mask=False, precision=prec, stream=stream)
        os.environ.pop("VS_FFS_SLOT_BYTES", None)
        for _ in range(3):
            plan.eval(xy, f, u)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            plan.eval(xy, f, u)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        plan.close()
        out[name] = {"ms": ms, "value": pairs / (ms * 1e-3)}
    out["symmetric_phased"]["slots"] = "32 chunk slots a point (16 B each) instead of 125: 4 groups, 10 phases"
    out["multipole_scaling"] = multipole_scaling(stream)
    return out


def multipole_scaling(stream, reps=5):
    """The multipole far field alone at growing vesicle counts (64-point vesicles in a box of the 2000 x 128
    box's vesicle density): vesicle by vesicle (precision 2: every vesicle pair tested and translated, O(M^2))
    against the cluster tree (precision 4: O(M log M) translations), ms per evaluation and the two results'
    relative difference."""
    import torch
    from paper_2606_25569_b300 import binding
    from paper_2606_25569_b300.workloads import farfield_box
    res = {}
    for M in (2000, 8000, 16000):
        wl, fx, fy = farfield_box(M=M, N=64, seed=13, box=20.0 * np.sqrt(M / 2000.0))
        xy = torch.as_tensor(wl.flat_xy(), device="cuda")
        f = torch.as_tensor(np.concatenate([np.concatenate([a, b]) for a, b in zip(fx, fy)]), device="cuda")
        row, got = {}, {}
        for name, prec in (("vesicle_pairs", 2), ("tree", 4)):
            plan = binding.FarFieldPlan(wl.offsets, mu=1.0, near_mask=False, precision=prec, stream=stream)
            u = torch.empty_like(xy)
            for _ in range(3):
                plan.eval(xy, f, u)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                plan.eval(xy, f, u)
            e1.record(stream)
            torch.cuda.synchronize()
            row[name + "_ms"] = round(e0.elapsed_time(e1) / reps, 4)
            got[name] = u.cpu().numpy()
            plan.close()
        row["relative_difference"] = float(np.linalg.norm(got["tree"] - got["vesicle_pairs"]) /
                                           np.linalg.norm(got["vesicle_pairs"]))
        res["%dx64" % M] = row
    return res


def _profile_steps(sus, n):
    """Per-kernel CUDA-event times over n steps: {kernel: (ms, launches)}."""
    sus.profile(True)
    sus.step(n)
    prof = sus.profile_read()
    sus.profile(False)
    return prof


def near_field_arm(args, stream):
    """The plain step on the dense Poiseuille suspension with every tenth vesicle moved to 0.7 spacings h
    from its neighbour (workloads.poiseuille_dense, close_fraction 0.1): near pairs from the first step, so
    the five-layer RBF correction (k_near_*) does work. Pairs that close are not resolved by the explicit
    inter-vesicle coupling at the headline time step (their gaps jitter and the area/length correction
    stops converging within about 15 steps), so this arm takes a time step ten times smaller. Reports the
    near pairs of the first and the last step and the near-field kernels' time beside the step's."""
    from paper_2606_25569_b300 import binding
    from paper_2606_25569_b300.workloads import poiseuille_dense
    wl = poiseuille_dense(args.M, args.N, seed=5, close_fraction=0.1, close_gap=0.7)
    dt = wl.dt / 10
    sus = binding.Suspension(wl.flat_xy(), wl.offsets, kappa=wl.kappa, mu=wl.mu, dt=dt, corr_tol=0.01,
                             flow_kind=wl.flow_kind, flow_p=wl.flow_p, near_field=True, stream=stream, use_graph=True)
    sus.step(1)
    sus.sync()
    first = sus.counters()["near_pairs"]
    sus.step(2)
    sus.sync()
    n = max(4, args.steps)
    ms = _time_steps(sus, n, stream)
    c = sus.counters()
    prof = _profile_steps(sus, n)
    c2 = sus.counters()
    sus.close()
    near_ms = {k: round(v[0] / n, 4) for k, v in prof.items() if k.startswith("k_near")}
    out = {"workload": wl.name + ", dt = headline dt / 10", "value": wl.M / (ms * 1e-3), "unit": UNIT,
           "ms_per_step": ms, "steps_timed": n, "near_pairs_first_step": first,
           "near_pairs_last_step": c2["near_pairs"], "corrections_total": c2["corrections"], "err": c2["err"],
           "near_field_ms_per_step": round(sum(near_ms.values()), 4), "near_kernels_ms_per_step": near_ms}
    # the same suspension with the Ying-Zorin near field (Sec. 2.2.2), and the two schemes' interaction
    # velocities from the same initial state
    yz = binding.Suspension(wl.flat_xy(), wl.offsets, kappa=wl.kappa, mu=wl.mu, dt=dt, corr_tol=0.01,
                            flow_kind=wl.flow_kind, flow_p=wl.flow_p, near_field=True, stream=stream, use_graph=True,
                            near_yz=True)
    rbf = binding.Suspension(wl.flat_xy(), wl.offsets, kappa=wl.kappa, mu=wl.mu, dt=dt, corr_tol=0.01,
                             flow_kind=wl.flow_kind, flow_p=wl.flow_p, near_field=True, stream=stream)
    yz.step(1)
    rbf.step(1)
    uy_, ur_ = yz.velocity(), rbf.velocity()
    rbf.close()
    yz.step(2)
    yz.sync()
    ms_yz = _time_steps(yz, n, stream)
    prof = _profile_steps(yz, n)
    yz.close()
    out["ying_zorin"] = {"value": wl.M / (ms_yz * 1e-3), "ms_per_step": ms_yz,
                         "near_kernels_ms_per_step": {k: round(v[0] / n, 4) for k, v in prof.items()
                                                      if k.startswith("k_near")},
                         "rbf_against_ying_zorin_first_step": {
                             "relative_l2": float(np.linalg.norm(ur_ - uy_) / np.linalg.norm(uy_)),
                             "max_over_max": float(np.max(np.abs(ur_ - uy_)) / np.max(np.abs(uy_)))}}
    return out


def uneven_arm(args, stream):
    """The plain step on the dense Poiseuille lattice with vesicles of 32, 64 and 128 points in turn
    (2000 vesicles, 149,333 points): the symmetric far field (vesicles in classes of 1, 2, 4 segments) against
    the per-target kernel."""
    from paper_2606_25569_b300 import binding
    from paper_2606_25569_b300.workloads import poiseuille_dense
    wl = poiseuille_dense(args.M, (32, 64, 128), seed=5)
    out = {"workload": wl.name, "points": int(wl.offsets[-1]), "unit": UNIT}
    for name, extra in (("symmetric", {}), ("per_target", {"farfield_per_target": True})):
        sus = binding.Suspension(wl.flat_xy(), wl.offsets, kappa=wl.kappa, mu=wl.mu, dt=wl.dt, corr_tol=0.01,
                                 flow_kind=wl.flow_kind, flow_p=wl.flow_p, near_field=True, stream=stream,
                                 use_graph=True, **extra)
        sus.step(3)
        sus.sync()
        n = max(4, args.steps)
        ms = _time_steps(sus, n, stream)
        prof = _profile_steps(sus, n)
        sus.close()
        ff = sum(v[0] for k, v in prof.items() if k.startswith("k_farfield")) / n
        out[name] = {"value": wl.M / (ms * 1e-3), "ms_per_step": ms, "far_field_ms_per_step": round(ff, 4)}
        if name == "symmetric":
            kms = {k: round(v[0] / n, 4) for k, v in prof.items()}
            out[name]["kernel_ms_per_step"] = dict(sorted(kms.items(), key=lambda kv: -kv[1]))
    return out


def implicit_arm(args, stream, tol=1e-8, multipole=False):
    """The paper's ground-truth scheme on the headline suspension: the fully implicit step (Sec. 2.2.3,
    Eq. time_step_sc1) solved by restarted flexible GMRES (30 vectors) with the per-vesicle FP32
    preconditioner, every product through the symmetric far field (or the vesicle-multipole far field) and
    the Ying-Zorin near field (the ground truth's near-singular scheme, Sec. 2.2.2). Reports the GMRES iterations per step and the kernels' shares beside the step time."""
    from paper_2606_25569_b300 import binding
    wl = workload(args)
    sus = binding.Suspension(wl.flat_xy(), wl.offsets, kappa=wl.kappa, mu=wl.mu, dt=wl.dt, corr_tol=0.01,
                             flow_kind=wl.flow_kind, flow_p=wl.flow_p, near_field=True, stream=stream, mode=2,
                             farfield_multipole=multipole, near_yz=True)
    sus.set_gmres(tol=tol, restart=30, max_iter=600)
    sus.step(1)
    sus.sync()
    n = max(3, min(args.steps, 5))
    _, _, it0 = sus.gmres_stats()
    l0 = sus.counters()["launches"]
    ms = _time_steps(sus, n, stream)
    last, res, it1 = sus.gmres_stats()
    launches = sus.counters()["launches"] - l0
    prof = _profile_steps(sus, 1)
    _, _, it2 = sus.gmres_stats()
    c = sus.counters()
    sus.close()
    tot = sum(v[0] for v in prof.values())
    groups = {"far_field": "k_farfield", "near_field": "k_near", "gmres_vectors": "k_gm_", "products": "k_imp_"}
    shares = {g: round(sum(v[0] for k, v in prof.items() if k.startswith(pfx)) / tot, 4) for g, pfx in groups.items()}
    return {"workload": wl.name, "value": wl.M / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps_timed": n,
            "gmres": {"tol": tol, "restart": 30, "iterations_per_step": (it1 - it0) / n,
                      "last_residual_estimate": res, "iterations_profiled_step": it2 - it1},
            "gpu_launches_per_step": launches / n, "kernel_time_shares": shares, "corrections": c["corrections"],
            "near_pairs_last_product": c["near_pairs"],
            "far_field": ("fp32 vesicle multipole and local expansions for separated vesicles, point sums inside"
                          if multipole else "fp32 symmetric pair kernel (as the plain step)")}


def ivnet_arm(args, stream):
    """IVNet (Sec. 3.4.2, Fig. fig:net: the paper's architecture) against the MLP as the relaxation map: both
    trained on the GPU on the same 128 k exact relaxation pairs (64 snapshots of a differently seeded dense
    suspension), IVNet on point rows, the MLP on Fourier features; the held-out relative error of the
    displacement compared in point space, and the forward time at the suspension's batch."""
    import torch
    from paper_2606_25569_b300 import train
    from paper_2606_25569_b300.workloads import poiseuille_dense
    N, kmax, M = args.N, 16, args.M
    t0 = time.time()
    X, Y = train.relaxation_samples(poiseuille_dense(M=M, N=N, seed=105), 64, 15, stream, kmax)
    Xp, Yp = train.to_points(X, N, kmax), train.to_points(Y, N, kmax)
    t_data = time.time() - t0
    rm = train.train_relaxation(X, Y, hidden=(1024, 1024, 1024), epochs=40, batch=1024, lr=1e-3, lr_min=1e-5,
                                stream=stream, serve_batch=M)
    ri = train.train_ivnet(Xp, Yp, N, C=IV_C, nb=IV_NB, epochs=IV_EPOCHS, batch=1024, lr=1e-3, lr_min=1e-5,
                           stream=stream, serve_batch=M)
    n = X.shape[0]
    ntr = n - int(round(0.1 * n))
    # the MLP's held-out predictions in point space
    pred = torch.empty_like(Y[ntr:])
    for a in range(0, n - ntr, 1024):
        b = min(a + 1024, n - ntr)
        rm["net"].forward(X[ntr + a:ntr + b], pred[a:b], b - a)
    rm["net"].sync()
    pp, yp = train.to_points(pred, N, kmax), Yp[ntr:]
    mlp_pts = (torch.linalg.norm(pp - yp, dim=1) / torch.linalg.norm(yp, dim=1)).cpu().numpy()

    def fwd_ms(net, x, width):
        y = torch.empty(M, width, dtype=torch.float32, device="cuda")
        net.forward(x[:M], y, M)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(20):
            net.forward(x[:M], y, M)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 20

    out = {"samples": n, "data_seconds": round(t_data, 1),
           "mlp": {"dims": rm["dims"], "params": int(sum(a * b + b for a, b in zip(rm["dims"][:-1], rm["dims"][1:]))),
                   "holdout_rel_err_mean": float(np.mean(mlp_pts)),
                   "holdout_rel_err_features": float(np.mean(rm["holdout_err"])),
                   "train_seconds": round(rm["train_seconds"], 1), "forward_ms_batch_M": fwd_ms(rm["net"], X, X.shape[1])},
           "ivnet": {"channels": IV_C, "blocks": IV_NB, "levels": 2, "params": int(ri["params"]),
                     "holdout_rel_err_mean": float(np.mean(ri["holdout_err"])), "train_steps": ri["steps"],
                     "train_seconds": round(ri["train_seconds"], 1), "forward_ms_batch_M": fwd_ms(ri["net"], Xp, 2 * N)},
           "epochs": 40, "batch": 1024,
           "note": "held-out relative error of the relaxation displacement at the N points (the MLP's feature "
                   "output converted to points); the MLP's own feature-space error beside it"}
    rm["net"].close()
    ri["net"].close()
    return out


def near_learned_arm(args, stream):
    """The learned near field (Sec. 3.3, Eq. NearFieldMap) on the near-field arm's suspension: five layer
    networks (one per layer, density modes and columns up to N/2 - 1) trained on the GPU on exact layer columns
    (vs_near_maps) of 16 snapshots of a differently seeded dense suspension, then a hybrid suspension whose
    relaxation stays exact every step (exact_every = 1: only the near field is learned) against the plain step
    from the same state. Reports the interaction velocity's difference after the first step, throughput, and
    the shape error after 10 .. 300 steps (at the arm's time step, a tenth of the headline's)."""
    import torch
    from paper_2606_25569_b300 import binding, train
    from paper_2606_25569_b300.workloads import poiseuille_dense
    N, kmax = args.N, 16
    K = N // 2 - 1
    t0 = time.time()
    X, rows = train.near_samples(poiseuille_dense(M=args.M, N=N, seed=105), NEAR_SNAPSHOTS, 15, stream, kmax, K, K)
    t_data = time.time() - t0
    res = [train.train_relaxation(X, rows[d], hidden=(1024, 1024, 1024), epochs=NEAR_EPOCHS, batch=1024, lr=1e-3,
                                  lr_min=1e-5, beta=0.0, stream=stream, serve_batch=args.M) for d in range(5)]
    t_train = time.time() - t0 - t_data
    del X, rows
    W = binding.feature_width(N, kmax)
    rel = binding.Mlp([W, W], max_batch=args.M, stream=stream)  # input width only: the relaxation stays exact
    rel.set_params(np.zeros(W * W + W))
    wl = poiseuille_dense(args.M, N, seed=5, close_fraction=0.1, close_gap=0.7)
    kw = dict(kappa=wl.kappa, mu=wl.mu, dt=wl.dt / 10, corr_tol=0.01, flow_kind=wl.flow_kind, flow_p=wl.flow_p,
              near_field=True, stream=stream, use_graph=True)
    plain = binding.Suspension(wl.flat_xy(), wl.offsets, **kw)
    learned = binding.Suspension(wl.flat_xy(), wl.offsets, mode=1, exact_every=1, **kw)
    learned.set_network(rel, 1.0, kmax)
    learned.set_near_networks([r["net"] for r in res], K, K)
    plain.step(1)
    learned.step(1)
    up, ul = plain.velocity(), learned.velocity()
    near_pairs = plain.counters()["near_pairs"]
    du = {"relative_l2": float(np.linalg.norm(ul - up) / np.linalg.norm(up)),
          "max_over_max": float(np.max(np.abs(ul - up)) / np.max(np.abs(up)))}
    out = {"workload": wl.name + ", dt = headline dt / 10", "unit": UNIT, "near_pairs_first_step": near_pairs,
           "nets": {"dims": res[0]["dims"], "density_modes_Kf": K, "column_modes_Kout": K,
                    "holdout_rel_err_mean_by_layer": [float(np.mean(r["holdout_err"])) for r in res],
                    "train_samples": int(res[0]["train_err"].shape[0] + res[0]["holdout_err"].shape[0]),
                    "data_seconds": round(t_data, 1), "train_seconds": round(t_train, 1)},
           "interaction_velocity_difference_first_step": du}
    errs, done = {}, 1
    for S in (10, 100, 300):
        plain.step(S - done)
        learned.step(S - done)
        plain.sync()
        learned.sync()
        e, _ = train.centred_shape_error(learned.positions(), plain.positions(), wl.counts)
        errs[str(S)] = float(np.mean(e))
        done = S
    out["shape_error_mean_by_step"] = errs
    n = max(4, args.steps)
    for name, sus in (("plain", plain), ("learned", learned)):
        ms = _time_steps(sus, n, stream)
        prof = _profile_steps(sus, n)
        out[name] = {"value": wl.M / (ms * 1e-3), "ms_per_step": ms,
                     "near_kernels_ms_per_step": round(sum(v[0] for k, v in prof.items() if k.startswith("k_near"))
                                                       / n, 4)}
        sus.close()
    out["note"] = ("near_kernels_ms_per_step: the library's k_near_* launches (layers, RBF, apply); the learned "
                   "run's five network forwards run on the networks' handles and count in ms_per_step only")
    for r in res:
        r["net"].close()
    rel.close()
    return out


def _time_steps(sus, n, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sus.step(n)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def _window_len(key):
    a, b = key.split("-")
    return int(b) - int(a)


def long_run_arms(wl, args, stream):
    """Variants of the step against the plain step (all-pairs point sums) from the same state:
    * hybrid: learned relaxation, exact relaxation on every HYBRID_EVERY-th step and for vesicles in near
      pairs or within four spacings of another vesicle; the network trained on the GPU on exact relaxation
      pairs of a differently seeded suspension (HYBRID_SNAPSHOTS snapshots 15 steps apart);
    * farfield_multipole: the plain step with the vesicle-multipole far field;
    * hybrid_multipole: both;
    * hybrid_flow (and hybrid_flow_multipole): the hybrid step with the advection and the tension of every step
      from two more networks (Sec. 3.2, Eqs. advectionMap and advTenMap), trained on exact columns of the
      same snapshots.
    Each reports the mean over vesicles of the centred relative shape error (App. B) against the plain step
    after 10 .. args.hybrid_steps steps, and its throughput over that whole run (CUDA events per window; value
    and vs_plain against the plain run of the same steps), with the first steps' throughput beside it."""
    from paper_2606_25569_b300 import binding, train
    from paper_2606_25569_b300.workloads import poiseuille_dense
    kmax, width, Kf, Kout = 16, 1024, FLOW_KF, FLOW_KOUT
    t0 = time.time()
    X, Y, A, T = train.hybrid_samples(poiseuille_dense(M=wl.M, N=args.N, seed=105), HYBRID_SNAPSHOTS, 15, stream,
                                      kmax, Kf, Kout)
    t_data = time.time() - t0
    hid = (width, width, width)
    r = train.train_relaxation(X, Y, hidden=hid, epochs=HYBRID_EPOCHS, batch=1024, lr=1e-3, lr_min=1e-5,
                               stream=stream, serve_batch=wl.M)
    t_train = time.time() - t0 - t_data
    ra = train.train_relaxation(X, A, hidden=hid, epochs=FLOW_EPOCHS, batch=1024, lr=1e-3, lr_min=1e-5, beta=0.0,
                                stream=stream, serve_batch=wl.M)
    rt = train.train_relaxation(X, T, hidden=hid, epochs=FLOW_EPOCHS, batch=1024, lr=1e-3, lr_min=1e-5, beta=0.0,
                                stream=stream, serve_batch=wl.M)
    t_flow = time.time() - t0 - t_data - t_train
    del X, Y, A, T
    net = {"dims": r["dims"], "train_samples": int(r["train_err"].shape[0] + r["holdout_err"].shape[0]),
           "train_steps": r["steps"], "holdout_rel_err_mean": float(np.mean(r["holdout_err"])),
           "data_seconds": round(t_data, 1), "train_seconds": round(t_train, 1), "input_filter_kmax": kmax,
           "features": "Fourier, normalised"}
    flow_nets = {"advection": {"dims": ra["dims"], "holdout_rel_err_mean": float(np.mean(ra["holdout_err"])),
                               "train_steps": ra["steps"]},
                 "tension": {"dims": rt["dims"], "holdout_rel_err_mean": float(np.mean(rt["holdout_err"])),
                             "train_steps": rt["steps"]},
                 "velocity_modes_Kf": Kf, "column_modes_Kout": Kout, "train_seconds": round(t_flow, 1),
                 "maps": "advection (I - M) psi_k and tension L^-1 P psi_k, L^-1 P B X in the standard frame "
                         "(Eqs. advectionMap, advTenMap, S_sigma), learned in every step"}
    kw = dict(kappa=wl.kappa, mu=wl.mu, dt=wl.dt, corr_tol=0.01, flow_kind=wl.flow_kind, flow_p=wl.flow_p,
              near_field=True, stream=stream, use_graph=True)
    variants = {"hybrid": dict(mode=1, exact_every=HYBRID_EVERY),
                "farfield_multipole": dict(farfield_multipole=True),
                "hybrid_multipole": dict(mode=1, exact_every=HYBRID_EVERY, farfield_multipole=True),
                "hybrid_flow": dict(mode=1, exact_every=FLOW_EVERY, flow=True),
                "hybrid_flow_multipole": dict(mode=1, exact_every=FLOW_EVERY, farfield_multipole=True, flow=True)}

    def make(cfg):
        cfg = dict(cfg)
        flow = cfg.pop("flow", False)
        sus = binding.Suspension(wl.flat_xy(), wl.offsets, **cfg, **kw)
        if cfg.get("mode", 0) == 1:
            sus.set_network(r["net"], r["scale"], kmax)
        if flow:
            sus.set_flow_networks(ra["net"], rt["net"], Kf, Kout)
        return sus

    out = {}
    for name, cfg in variants.items():
        sus = make(cfg)
        sus.step(4)
        sus.sync()
        per = cfg.get("exact_every", 1)  # whole cycles of learned and exact relaxation
        n = per * max(2, args.steps // per)
        ms = _time_steps(sus, n, stream)
        prof = {}
        if "multipole" in name:
            sus.profile(True)
            sus.step(2)
            prof = sus.profile_read()
            sus.profile(False)
        sus.close()
        out[name] = {"unit": UNIT, "early": {"value": wl.M / (ms * 1e-3), "ms_per_step": ms,
                                             "steps_timed": "%d after 4" % n}}
        if prof:
            out[name]["far_field_ms_per_step"] = sum(v[0] for k, v in prof.items()
                                                     if k in ("k_ff_moments", "k_ff_local", "k_farfield_loc")) / 2
        if cfg.get("flow"):
            out[name]["flow_networks"] = flow_nets
        if cfg.get("mode", 0) == 1:
            out[name]["net"] = net
            out[name]["exact_every"] = cfg["exact_every"]
            out[name]["fallback"] = ("exact relaxation on every %d-th step and for vesicles within 4 spacings h of "
                                     "another vesicle" % cfg["exact_every"])
        if cfg.get("farfield_multipole"):
            out[name]["far_field"] = ("order-12 vesicle expansions translated to local expansions about each target "
                                      "vesicle's centre for vesicle pairs farther apart than twice the sum of "
                                      "their reach radii; for the other pairs the expansion per target point beyond "
                                      "three reach radii, point sums (with the near test) inside: an approximation of "
                                      "the all-pairs sum")
    # shape error against the plain step from the same initial state
    plain = binding.Suspension(wl.flat_xy(), wl.offsets, **kw)
    runs = {name: make(cfg) for name, cfg in variants.items()}
    errs = {name: {} for name in variants}
    windows = {name: {} for name in variants}
    plain_windows = {}
    failed = {}
    done = 0
    import torch
    for S in sorted({min(k, args.hybrid_steps) for k in (10, 100, 300, 500, 800, 1000, args.hybrid_steps)}):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plain.step(S - done)
        e1.record(stream)
        plain.sync()
        plain_windows["%d-%d" % (done, S)] = {"ms_per_step": e0.elapsed_time(e1) / (S - done)}
        ref = plain.positions()
        for name, sus in runs.items():
            if name in failed:
                continue
            try:
                c0 = sus.hybrid_counters()
                e0.record(stream)
                sus.step(S - done)
                e1.record(stream)
                sus.sync()
            except Exception as ex:  # a non-finite state ends that comparison
                failed[name] = "step %d..%d: %s" % (done, S, ex)
                continue
            c1 = sus.hybrid_counters()
            tests = c1["fallback_steps"] - c0["fallback_steps"]
            windows[name]["%d-%d" % (done, S)] = {
                "ms_per_step": e0.elapsed_time(e1) / (S - done),
                "exact_fraction": ((c1["exact_vesicles"] - c0["exact_vesicles"]) / (tests * wl.M)) if tests else None}
            e, _ = train.centred_shape_error(sus.positions(), ref, wl.counts)
            errs[name][str(S)] = float(np.mean(e))
        done = S
    plain.close()
    for name, sus in runs.items():
        sus.close()
        last = errs[name].get(str(args.hybrid_steps))
        out[name].update({"shape_error_mean_by_step": errs[name], "after_steps": args.hybrid_steps,
                          "meets_shape_error_1e-2": bool(last is not None and last <= 1e-2),
                          "windows": windows[name], "plain_windows": plain_windows})
        # throughput over the whole run and over its last window (the plain run timed on the same steps)
        if windows[name] and name not in failed:
            tot = sum(w["ms_per_step"] * _window_len(k) for k, w in windows[name].items())
            ptot = sum(plain_windows[k]["ms_per_step"] * _window_len(k) for k in windows[name])
            nst = sum(_window_len(k) for k in windows[name])
            out[name].update({"value": wl.M * nst / (tot * 1e-3), "ms_per_step": tot / nst, "vs_plain": ptot / tot,
                              "steps_timed": "0-%d" % nst, "plain_ms_per_step": ptot / nst})
        if windows[name]:
            key = list(windows[name])[-1]
            w = windows[name][key]
            out[name]["late_window"] = {"steps": key, "value": wl.M / (w["ms_per_step"] * 1e-3), "unit": UNIT,
                                        "ms_per_step": w["ms_per_step"], "exact_fraction": w["exact_fraction"],
                                        "vs_plain": plain_windows[key]["ms_per_step"] / w["ms_per_step"]}
        if name in failed:
            out[name]["failed"] = failed[name]
    r["net"].close()
    ra["net"].close()
    rt["net"].close()
    return out


def run_gpu(args):
    import torch
    from paper_2606_25569_b300 import build as _build
    _build.build()
    from paper_2606_25569_b300 import binding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = workload(args)
    stream = torch.cuda.current_stream()
    s = binding.Suspension(wl.flat_xy(), wl.offsets, kappa=wl.kappa, mu=wl.mu, dt=wl.dt, corr_tol=0.01,
                           flow_kind=wl.flow_kind, flow_p=wl.flow_p, near_field=True, stream=stream, use_graph=True,
                           farfield_multipole=args.farfield_multipole)
    fv = s.farfield_variant()
    for _ in range(max(args.warmup, 3)):
        s.step(1)
    s.sync()
    launches0 = s.counters()["launches"]
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    s.step(args.steps)
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if dist:
        dist.barrier()
    ms = t0.elapsed_time(t1)
    s.sync()
    c = s.counters()
    launches = c["launches"] - launches0
    # whole job: every rank's vesicle-steps over the slowest rank's time (replicas: weak scaling)
    from paper_2606_25569_b300.shard import job_throughput
    value, ms = job_throughput(wl.M * args.steps, ms)

    # per-kernel CUDA-event breakdown over the same number of steps
    s.profile(True)
    s.step(args.steps)
    prof = s.profile_read()
    s.profile(False)
    total_prof = sum(v[0] for v in prof.values())
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_n) = dom
    peaks, peak_src = load_peaks()
    fp64_peak = measured_fp64_tflops(torch)
    avg_ms = dom_ms / dom_n
    flops = kernel_flops(dom_name, args.N, wl.M)
    if flops > 0:
        achieved = flops / (avg_ms * 1e-3) / 1e12
        roof = {"kernel": dom_name, "bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "traffic": None,
                "peak_source": "FP64: cuBLAS DGEMM 4096^3 measured in this run (of measured)",
                "share_of_step": dom_ms / total_prof}
    elif dom_name.startswith("k_farfield_f32"):
        pairs = float(wl.offsets[-1]) ** 2 - float(np.sum(wl.counts.astype(np.float64) ** 2))
        mhz = clocks.get("sm_mhz") or 1920.0
        peak_mufu = MUFU_PER_CLK_SM * N_SM * mhz * 1e6 / 1e12
        achieved = 2 * pairs / (avg_ms * 1e-3) / 1e12
        roof = {"kernel": dom_name, "bound": "alu", "achieved": achieved, "peak": peak_mufu, "unit": "Tmufu/s",
                "frac": achieved / peak_mufu, "traffic": FF_DRAM_BYTES_PER_POINT * float(wl.offsets[-1]),
                "traffic_source": "ncu dram__bytes at 1200 x 64, scaled by points",
                "peak_source": "16 MUFU/clk/SM x 148 SMs x median SM clock (derived)",
                "share_of_step": dom_ms / total_prof}
    elif dom_name.startswith("k_farfield_sym"):
        # FP32-pipe bound (paired float2 instructions; the special-function unit carries lg2 and rcp beside it)
        pairs = (float(wl.offsets[-1]) ** 2 - float(np.sum(wl.counts.astype(np.float64) ** 2))) / 2
        mhz = clocks.get("sm_mhz") or 1920.0
        peak_fp32 = FP32_LANES_PER_CLK_SM * N_SM * mhz * 1e6 / 1e12
        achieved = FFS_FP32_PER_PAIR * pairs / (avg_ms * 1e-3) / 1e12
        # the measured traffic is for chunks of 16 vesicles; its partial-sum writes scale with the chunk count
        V = fv[2] // args.N if fv[0] < 0 else 16
        traffic = FFS_DRAM_READ + FFS_DRAM_WRITE * 16.0 / V
        # measured beside the derived peak: paired FMA chains alone, and the pair loop's own instruction mix
        # (registers only), both through the library's probe on this GPU
        ffma2, _ = binding.fp32_rate(0, stream=torch.cuda.current_stream())
        mix, _ = binding.fp32_rate(1, stream=torch.cuda.current_stream())
        roof = {"kernel": dom_name, "bound": "alu", "achieved": achieved, "peak": peak_fp32,
                "unit": "T FP32 lane-ops/s", "frac": achieved / peak_fp32, "traffic": traffic,
                "traffic_source": FFS_DRAM_SOURCE + (", writes scaled from 16 to %d vesicles per chunk" % V
                                                     if V != 16 else ""),
                "peak_source": "FP32 pipe: 128 lanes per clock per SM x 148 SMs x median SM clock (derived); "
                               "achieved counts 18 FP32 lane operations per unordered pair of points",
                "measured": {"ffma2_chains": ffma2, "frac_of_ffma2_chains": achieved / ffma2,
                             "pair_mix_registers_only": mix, "frac_of_pair_mix": achieved / mix,
                             "source": "vs_fp32_rate probes, 2 CTAs of 256 threads per SM, CUDA events"},
                "share_of_step": dom_ms / total_prof}
    else:
        roof = {"kernel": dom_name, "bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None, "share_of_step": dom_ms / total_prof}
    breakdown = {k: round(v[0] / v[1], 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}
    per_step = {k: round(v[0] / args.steps, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}

    # end to end through the C ABI with host buffers: upload state, step, read positions (right after the
    # timed region, so at the same stage of the run as the device-timed value)
    e2e = None
    if not args.no_e2e:
        xy_h = torch.empty(2 * s.P, dtype=torch.float64).pin_memory()
        sg_h = torch.empty(s.P, dtype=torch.float64).pin_memory()
        xy_h.copy_(torch.from_numpy(s.positions()))
        sg_h.copy_(torch.from_numpy(s.tension()))
        L = binding.lib()
        n_e2e = max(3, args.steps // 3)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for _ in range(n_e2e):
            assert L.vs_set_state(s._h, xy_h.data_ptr(), sg_h.data_ptr()) == 0
            assert L.vs_step(s._h, 1) == 0
            assert L.vs_get_positions(s._h, xy_h.data_ptr(), 2 * s.P) == 0
            assert L.vs_get_tension(s._h, sg_h.data_ptr(), s.P) == 0
        w1 = time.perf_counter()
        e2e = {"value": world * wl.M * n_e2e / (w1 - w0), "unit": UNIT, "h2d_bytes_per_step": 24 * s.P,
               "d2h_bytes_per_step": 24 * s.P, "steps": n_e2e,
               "note": "per step: vs_set_state (positions + tension from pinned host), vs_step, "
                       "vs_get_positions + vs_get_tension to pinned host; wall clock"}

    # steady state: after a burn-in the area/length correction fires for a few vesicles every step
    steady = None
    if args.burn_in > 0:
        s.step(args.burn_in)
        s.sync()
        c0 = s.counters()["corrections"]
        t2, t3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t2.record(stream)
        s.step(args.steps)
        t3.record(stream)
        torch.cuda.synchronize()
        ms_ss = t2.elapsed_time(t3) / args.steps
        steady = {"after_steps": args.burn_in + max(args.warmup, 3) + args.steps, "steps": args.steps,
                  "ms_per_step": ms_ss, "value": world * wl.M / (ms_ss * 1e-3), "unit": UNIT,
                  "corrections_per_step": (s.counters()["corrections"] - c0) / args.steps}

    ff_alone = farfield_alone(stream) if rank == 0 and not args.no_farfield_alone else None
    near_arm = near_field_arm(args, stream) if rank == 0 and not args.no_near_arm else None
    uneven = uneven_arm(args, stream) if rank == 0 and not args.no_uneven_arm else None
    near_learned = near_learned_arm(args, stream) if rank == 0 and not args.no_near_learned_arm else None
    ivnet = ivnet_arm(args, stream) if rank == 0 and not args.no_ivnet_arm else None
    implicit = implicit_arm(args, stream) if rank == 0 and not args.no_implicit_arm else None
    if implicit:
        implicit["plain_vs_implicit"] = (value / world) / implicit["value"]
        implicit["multipole"] = implicit_arm(args, stream, multipole=True)
    arms = {}
    if rank == 0 and not args.no_hybrid:
        arms = long_run_arms(wl, args, stream)
        for v in arms.values():
            if "vs_plain" not in v:  # a run that failed: its first steps against the headline
                v["vs_plain"] = v["early"]["value"] / (value / world)
            if "value" not in v:
                v["value"] = v["early"]["value"]
            if implicit:
                v["vs_implicit"] = v["value"] / implicit["value"]
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        procs = host_cores()
        cpu = oracle_sample(wl, procs=procs)
        one = oracle_sample(wl, n_ves=8, n_targets=512)
        cpu["single_core"] = {"value": one["value"], "cores": 1, "sample": one["sample"]}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config_of(wl, args, {"parallelism": "replicas" if world > 1 else "single GPU",
                                               "farfield_launch": ("symmetric pair kernel: %d threads per CTA, "
                                                                   "column chunks of %d points, persistent CTAs"
                                                                   % (fv[1], fv[2])) if fv[0] < 0 else
                                                                  ("per-target kernel: %d threads x %d staged source "
                                                                   "points per CTA (autotuned at create)"
                                                                   % (fv[1], fv[2]))}
                                    if not args.farfield_multipole else
                                    {"parallelism": "replicas" if world > 1 else "single GPU",
                                     "farfield": "fp32 vesicle multipole and local expansions for separated "
                                                 "vesicles, point sums inside (not the headline configuration)"}),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "kernel_ms_per_launch": breakdown, "kernel_ms_per_step": per_step,
                "steady_state": steady, "hybrid": arms.get("hybrid"),
                "farfield_multipole": arms.get("farfield_multipole"), "hybrid_multipole": arms.get("hybrid_multipole"),
                "hybrid_flow": arms.get("hybrid_flow"), "hybrid_flow_multipole": arms.get("hybrid_flow_multipole"),
                "farfield_2000x128": ff_alone, "near_field": near_arm, "uneven": uneven, "implicit": implicit,
                "near_field_learned": near_learned, "ivnet_relaxation": ivnet,
                "corrections": c["corrections"], "near_pairs_last_step": c["near_pairs"]}
        print(json.dumps(line))
    s.close()
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
