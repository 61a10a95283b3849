"""Sharding over ranks on the host (gloo, CPU processes): the partition, the source exchange and the
whole-job throughput of paper_2606_25569_b300.shard, with the FP64 oracle as the compute. A two-rank
sharded step (each rank its own vesicles, all sources exchanged, the far field for its own targets) must
give the single-process oracle's result; a rank that dies is detected by the other's next collective."""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2606_25569_b300.shard import allgather_rows, job_throughput, partition  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_covers_and_balances():
    rng = np.random.default_rng(0)
    for _ in range(50):
        M = int(rng.integers(1, 40))
        world = int(rng.integers(1, 9))
        counts = rng.choice([16, 32, 64, 128], size=M)
        parts = partition(counts, world)
        assert len(parts) == world and parts[0][0] == 0 and parts[-1][1] == M
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        assert all(v0 <= v1 for v0, v1 in parts)
        if M >= world:
            assert all(v1 > v0 for v0, v1 in parts)
        w = counts.astype(float) ** 2
        loads = [w[v0:v1].sum() for v0, v1 in parts]
        # contiguous ranges: each within one (largest) item of the even share, when every rank has one
        if M >= world:
            assert max(loads) <= w.sum() / world + 2 * w.max()


def _suspension(seed=4):
    from paper_2606_25569_b300.workloads import vesicle_outline
    rng = np.random.default_rng(seed)
    xs, ys = [], []
    for v in range(5):
        x, y = vesicle_outline(16, 0.7, 1.0, 1e-2, rng, rng.uniform(0, 2 * np.pi))
        xs.append(x + 2.6 * (v % 3))
        ys.append(y + 2.6 * (v // 3))
    return xs, ys


def _params():
    from oracle.step import Params
    return Params(kappa=1.0, mu=1.0, dt=1e-3, flow_kind=1, flow_p=(0.5, 0, 0, 0), near_field=True)


def _sharded_steps(rank, world, port, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle.farfield import far_field
    from oracle.flows import background
    from oracle.nearfield import near_correction
    from oracle.spectral import force
    from oracle.step import Suspension, advance_vesicle
    p = _params()
    xs, ys = _suspension()
    o = Suspension(xs, ys, p)  # the shared initial state (redistributed points, sigma^0, A_0, L_0)
    v0, v1 = partition([len(x) for x in o.xs], world)[rank]
    lx, ly, ls = o.xs[v0:v1], o.ys[v0:v1], o.sig[v0:v1]
    for _ in range(steps):
        # the exchange: every rank's points and forces, in rank order
        rows, cnt = [], []
        for x, y, s in zip(lx, ly, ls):
            fx, fy = force(x, y, s, p.kappa)
            rows.append(np.stack([x, y, fx, fy], axis=1))
            cnt.append(len(x))
        allr = allgather_rows(torch.as_tensor(np.concatenate(rows))).numpy()
        allc = allgather_rows(torch.as_tensor(np.array(cnt, dtype=np.int64)[:, None])).numpy()[:, 0]
        off = np.concatenate([[0], np.cumsum(allc)])
        gx = [allr[off[v]:off[v + 1], 0] for v in range(len(allc))]
        gy = [allr[off[v]:off[v + 1], 1] for v in range(len(allc))]
        gfx = [allr[off[v]:off[v + 1], 2] for v in range(len(allc))]
        gfy = [allr[off[v]:off[v + 1], 3] for v in range(len(allc))]
        mine = np.arange(off[v0], off[v1])
        ux, uy, near = far_field(gx, gy, gfx, gfy, p.mu, near_mask=True, targets=mine)
        if near:
            cx, cy = near_correction(gx, gy, gfx, gfy, p.mu, near)
            ux, uy = ux + cx[mine], uy + cy[mine]
        nx, ny, ns = [], [], []
        for k, v in enumerate(range(v0, v1)):
            a, b = off[v] - off[v0], off[v + 1] - off[v0]
            bx, by = background(p.flow_kind, p.flow_p, gx[v], gy[v])
            x1, y1, s1, _ = advance_vesicle(gx[v], gy[v], ux[a:b] + bx, uy[a:b] + by, o.A0[v], o.L0[v], p)
            nx.append(x1)
            ny.append(y1)
            ns.append(s1)
        lx, ly, ls = nx, ny, ns
    final = allgather_rows(torch.as_tensor(np.concatenate([np.concatenate([x, y]) for x, y in zip(lx, ly)])[:, None]))
    if rank == 0:
        np.save(out, final.numpy()[:, 0])
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_steps_match_single_process():
    from oracle.step import Suspension
    steps = 2
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "final.npy")
        mp.spawn(_sharded_steps, args=(2, _free_port(), steps, out), nprocs=2, join=True)
        got = np.load(out)
    xs, ys = _suspension()
    o = Suspension(xs, ys, _params())
    for _ in range(steps):
        o.step()
    ref = np.concatenate([np.concatenate([x, y]) for x, y in zip(o.xs, o.ys)])
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def _throughput(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    v, ms = job_throughput(100.0 * (rank + 1), 10.0 + rank)
    if rank == 0:
        np.save(out, np.array([v, ms]))
    dist.destroy_process_group()


def test_job_throughput_is_all_units_over_the_slowest_rank():
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "t.npy")
        mp.spawn(_throughput, args=(2, _free_port(), out), nprocs=2, join=True)
        v, ms = np.load(out)
    assert ms == 11.0 and abs(v - 300.0 / 11e-3) <= 1e-9 * v


def _dies(rank, world, port, out):
    import datetime
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    dist.barrier()
    if rank == 1:
        os._exit(0)  # leaves between steps, with no collective in flight
    try:
        allgather_rows(torch.zeros(3, 4))
        detected = "no"
    except Exception as ex:  # the peer's socket closed or the timeout ran out
        detected = "yes: " + type(ex).__name__
    with open(out, "w") as f:
        f.write(detected)
    os._exit(0)


def test_dead_rank_is_detected_by_the_next_collective():
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "r.txt")
        ctx = mp.start_processes(_dies, args=(2, _free_port(), out), nprocs=2, join=False, start_method="spawn")
        for proc in ctx.processes:
            proc.join(60)
        with open(out) as f:
            assert f.read().startswith("yes")
