"""Learned relaxation map: data generation on the GPU, training with the library's tensor-core MLP,
and the shape-error comparison of the hybrid step against the plain step (Sec. 3.2-3.4, App. B).

Data: a plain suspension is stepped with libvesb300; every `every` steps each vesicle's current
(equal-arclength) shape is taken as an input and the library's exact relaxation map gives the
target (vs_training_pairs: network input = filtered standardised shape, target = relaxation
displacement in the standard frame). Training: relative L2 loss with the derivative term and
AdamW at learning rate 1e-3 (Sec. 3.4.2), all in libvesb300 (vs_mlp_*). This module only
arranges calls, draws the initial weights and copies data.
"""
import time

import numpy as np

from . import binding


def he_uniform(dims, rng):
    """Initial flat parameters: He-uniform weights, zero biases (layout of vs_mlp)."""
    ws, bs = [], []
    for a, b in zip(dims[:-1], dims[1:]):
        lim = np.sqrt(6.0 / a)
        ws.append(rng.uniform(-lim, lim, size=(b, a)).ravel())
        bs.append(np.zeros(b))
    return np.concatenate(ws + bs).astype(np.float32)


def relaxation_samples(wl, snapshots, every, stream, kmax, near_field=None, skip=0):
    """(X, Y): FP32 device tensors (snapshots * M, W) of network inputs and raw targets (Fourier
    features up to mode kmax, W = binding.feature_width), taken every `every` steps after `skip`
    initial steps."""
    import torch
    nf = wl.near_field if near_field is None else near_field
    s = binding.Suspension(wl.flat_xy(), wl.offsets, kappa=wl.kappa, mu=wl.mu, dt=wl.dt, corr_tol=0.01,
                           flow_kind=wl.flow_kind, flow_p=wl.flow_p, near_field=nf, stream=stream)
    M, W = wl.M, binding.feature_width(len(wl.xs[0]), kmax)
    if skip:
        s.step(skip)
    X = torch.empty(snapshots * M, W, dtype=torch.float32, device="cuda")
    Y = torch.empty_like(X)
    for k in range(snapshots):
        xy = torch.as_tensor(s.positions(), device="cuda")
        s.training_pairs(xy, X[k * M:(k + 1) * M], Y[k * M:(k + 1) * M], 1.0, kmax)
        s.sync()
        if k + 1 < snapshots:
            s.step(every)
    s.sync()
    s.close()
    return X, Y


def hybrid_samples(wl, snapshots, every, stream, kmax, Kf, Kout, near_field=None, skip=0):
    """Training data of the hybrid step's three networks from one plain run: every `every` steps, each
    vesicle's current shape gives the network input X (Fourier features up to kmax of the standardised shape),
    the relaxation target R (vs_training_pairs), and the exact advection and tension columns A, T
    (vs_flow_maps, modes <= Kf of the velocity, columns up to Kout). FP32 device tensors, snapshots * M
    rows."""
    import torch
    nf = wl.near_field if near_field is None else near_field
    s = binding.Suspension(wl.flat_xy(), wl.offsets, kappa=wl.kappa, mu=wl.mu, dt=wl.dt, corr_tol=0.01,
                           flow_kind=wl.flow_kind, flow_p=wl.flow_p, near_field=nf, stream=stream)
    M, W = wl.M, binding.feature_width(len(wl.xs[0]), kmax)
    la, lt = binding.flow_widths(Kf, Kout)
    if skip:
        s.step(skip)
    X = torch.empty(snapshots * M, W, dtype=torch.float32, device="cuda")
    R = torch.empty_like(X)
    A = torch.empty(snapshots * M, la, dtype=torch.float32, device="cuda")
    T = torch.empty(snapshots * M, lt, dtype=torch.float32, device="cuda")
    X2 = torch.empty(M, W, dtype=torch.float32, device="cuda")
    for k in range(snapshots):
        rows = slice(k * M, (k + 1) * M)
        xy = torch.as_tensor(s.positions(), device="cuda")
        s.training_pairs(xy, X[rows], R[rows], 1.0, kmax)
        s.flow_maps(Kf, Kout, kmax, X2, A[rows], T[rows])
        s.sync()
        if k + 1 < snapshots:
            s.step(every)
    s.sync()
    s.close()
    return X, R, A, T


def near_samples(wl, snapshots, every, stream, kmax, Kf, Kout, skip=0):
    """Training data of the five near-field layer networks from one plain run: every `every` steps, each
    vesicle's current shape gives the network input X (as for the relaxation network) and the exact layer
    columns of the basis densities (vs_near_maps, density modes <= Kf, columns up to Kout). FP32 device
    tensors: X (snapshots * M rows) and a list of five (snapshots * M) x width tensors, layer order -h .. h."""
    import torch
    s = binding.Suspension(wl.flat_xy(), wl.offsets, kappa=wl.kappa, mu=wl.mu, dt=wl.dt, corr_tol=0.01,
                           flow_kind=wl.flow_kind, flow_p=wl.flow_p, near_field=True, stream=stream)
    M, W = wl.M, binding.feature_width(len(wl.xs[0]), kmax)
    width = binding.flow_widths(Kf, Kout)[0]
    if skip:
        s.step(skip)
    X = torch.empty(snapshots * M, W, dtype=torch.float32, device="cuda")
    rows = [torch.empty(snapshots * M, width, dtype=torch.float32, device="cuda") for _ in range(5)]
    buf = torch.empty(5, M, width, dtype=torch.float32, device="cuda")
    for k in range(snapshots):
        sl = slice(k * M, (k + 1) * M)
        s.near_maps(Kf, Kout, kmax, X[sl], buf)
        for d in range(5):
            rows[d][sl].copy_(buf[d])
        s.sync()
        if k + 1 < snapshots:
            s.step(every)
    s.sync()
    s.close()
    return X, rows


def relative_errors(net, X, Y, batch):
    """Per-sample ||Yhat - Y|| / ||Y|| of the network on (X, Y) (device tensors)."""
    import torch
    out = torch.empty_like(Y)
    for a in range(0, X.shape[0], batch):
        b = min(a + batch, X.shape[0])
        net.forward(X[a:b], out[a:b], b - a)
    net.sync()
    return (torch.linalg.norm(out - Y, dim=1) / torch.linalg.norm(Y, dim=1)).cpu().numpy()


def train_relaxation(X, Y, hidden=(512, 512, 512), epochs=100, batch=4096, lr=1e-3, lr_min=1e-5, beta=0.1,
                     holdout=0.1, seed=0, stream=None, ncomp=2, serve_batch=0, normalise=True, rel_floor=1e-3):
    """Train on (X, Y); the last `holdout` fraction is held out. AdamW starts at lr (Sec. 3.4.2:
    1e-3) and decays on a cosine to lr_min over the epochs. The network can afterwards run batches of
    up to max(batch, serve_batch) rows (a suspension needs at least its vesicle count).

    normalise: every input and output feature is mapped to zero mean and unit deviation over the
    training rows (vs_mlp_fit_affine; the maps are part of the network, so the output scale is 1),
    deviations below rel_floor times the largest one raised to it.
    This matters here: the standardised shapes differ from each other by ~1e-2 of their size, below
    what a bfloat16 input resolves next to the shape itself. Otherwise the targets are divided by
    their RMS (the returned scale). Returns a dict with the network, its output scale, the loss
    history, held-out errors and timings."""
    import torch
    n = X.shape[0]
    nh = int(round(holdout * n))
    ntr = n - nh
    dims = [X.shape[1]] + list(hidden) + [Y.shape[1]]
    net = binding.Mlp(dims, max_batch=max(batch, serve_batch), ncomp=ncomp, beta=beta, stream=stream)
    net.set_params(he_uniform(dims, np.random.default_rng(seed)))
    if normalise:
        scale = 1.0
        Yn = Y
        net.fit_affine(X[:ntr].contiguous(), Y[:ntr].contiguous(), ntr, rel_floor)
    else:
        scale = float(torch.sqrt(torch.mean(Y[:ntr].double() ** 2)).item())
        Yn = (Y / scale).contiguous()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    hist = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps = 0
    for ep in range(epochs):
        lr_ep = lr_min + 0.5 * (lr - lr_min) * (1.0 + np.cos(np.pi * ep / max(1, epochs)))
        perm = torch.randperm(ntr, device="cuda", generator=gen)
        Xs, Ys = X[perm].contiguous(), Yn[perm].contiguous()
        for a in range(0, ntr - batch + 1, batch):
            want = (a == 0)
            lo = net.train_step(Xs[a:a + batch], Ys[a:a + batch], batch, lr=lr_ep, want_loss=want)
            steps += 1
            if want:
                hist.append(lo)
    net.sync()
    t_train = time.perf_counter() - t0
    err_tr = relative_errors(net, X[:ntr], Yn[:ntr], batch)
    err_ho = relative_errors(net, X[ntr:], Yn[ntr:], batch) if nh else np.array([])
    return {"net": net, "scale": scale, "dims": dims, "history": hist, "train_err": err_tr,
            "holdout_err": err_ho, "train_seconds": t_train, "steps": steps}


def centred_shape_error(xy_a, xy_b, counts):
    """Per-vesicle ||(X_a - c_a) - (X_b - c_b)|| / ||X_b - c_b|| (App. B error on centred shapes),
    with c the mean of the points, and the centre distance over the vesicle's radius of gyration."""
    out, cen = [], []
    o = 0
    for n in counts:
        xa, ya = xy_a[2 * o:2 * o + n], xy_a[2 * o + n:2 * o + 2 * n]
        xb, yb = xy_b[2 * o:2 * o + n], xy_b[2 * o + n:2 * o + 2 * n]
        ca, cb = np.array([xa.mean(), ya.mean()]), np.array([xb.mean(), yb.mean()])
        da = np.concatenate([xa - ca[0], ya - ca[1]])
        db = np.concatenate([xb - cb[0], yb - cb[1]])
        out.append(np.linalg.norm(da - db) / np.linalg.norm(db))
        cen.append(np.linalg.norm(ca - cb) / (np.linalg.norm(db) / np.sqrt(n)))
        o += n
    return np.array(out), np.array(cen)
