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


def ivnet_convs(C, nb, cin=2):
    """(C_in, C_out, k) of IVNet's convolutions in vs_ivnet's parameter order."""
    h = C // 2
    out = [(cin, C, 3)]
    for _ in range(nb):
        out += [(C, h, 3)] * 4 + [(C, C, 3), (C, C, 3), (C, C, 1)]
    return out + [(C, 2, 1)]


def ivnet_he_uniform(C, nb, rng, cin=2):
    """Initial flat parameters of vs_ivnet: He-uniform weights (fan-in C_in k), zero biases, and zero weights
    in the mixing convolutions, so that every block starts as the identity on its residual stream (without
    it the residual sums grow block by block: the first loss of an 8-block network was 197 against 1.4)."""
    out = []
    convs = ivnet_convs(C, nb, cin)
    for j, (ci, co, k) in enumerate(convs):
        lim = np.sqrt(6.0 / (ci * k))
        mixing = 0 < j < len(convs) - 1 and (j - 1) % 7 == 6
        out += [np.zeros(co * ci * k) if mixing else rng.uniform(-lim, lim, co * ci * k), np.zeros(co)]
    return np.concatenate(out).astype(np.float32)


def to_points(F, N, kmax):
    """Fourier feature rows (modes <= min(kmax, N/2 - 1), vs_training_pairs' layout) -> point rows
    [x(N), y(N)] (vs_feature_points)."""
    import torch
    K = min(kmax, N // 2 - 1)
    out = torch.empty(F.shape[0], 2 * N, dtype=torch.float32, device="cuda")
    binding.feature_points(F.contiguous(), F.shape[0], F.shape[1], N, K, out)
    return out


def split_points(F, N, kmax, k_split):
    """Fourier feature rows -> point rows of four signals [x_low(N), y_low(N), x_high(N), y_high(N)]: the modes
    <= k_split and the modes above it (to kmax) as separate signals, each normalised on its own by the network's
    input map (the high modes are ~1e-2 of the shape, below a bfloat16 input's resolution next to it)."""
    import torch
    K = min(kmax, N // 2 - 1)
    per = 2 * K + 1
    r = np.arange(per)
    mode = np.where(r <= K, r, r - K)
    low = np.zeros(F.shape[1], dtype=np.float32)
    for c in range(2):
        low[c * per:(c + 1) * per] = (mode <= k_split)
    low_t = torch.as_tensor(low, device="cuda")
    lo = to_points(F * low_t, N, kmax)
    hi = to_points(F * (1.0 - low_t) * (torch.arange(F.shape[1], device="cuda") < 2 * per), N, kmax)
    return torch.cat([lo, hi], dim=1).contiguous()


def train_ivnet(X, Y, N, C=64, nb=4, epochs=40, batch=1024, lr=1e-3, lr_min=1e-5, beta=0.1, holdout=0.1, seed=0,
                stream=None, serve_batch=0, rel_floor=1e-3, cin=2):
    """IVNet (Sec. 3.4.2) on point rows (X, Y) [x(N), y(N)]: normalised features (vs_ivnet_fit_affine), AdamW
    from lr decaying on a cosine to lr_min, the last `holdout` fraction held out (as train_relaxation)."""
    import torch
    n = X.shape[0]
    nh = int(round(holdout * n))
    ntr = n - nh
    net = binding.Ivnet(N, C, nb, max_batch=max(batch, serve_batch), beta=beta, stream=stream, in_channels=cin)
    net.set_params(ivnet_he_uniform(C, nb, np.random.default_rng(seed), cin))
    net.fit_affine(X[:ntr].contiguous(), Y[:ntr].contiguous(), ntr, rel_floor)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    hist = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps = 0
    for ep in range(epochs):
        lr_ep = lr_min + 0.5 * (lr - lr_min) * (1.0 + np.cos(np.pi * ep / max(1, epochs)))
        perm = torch.randperm(ntr, device="cuda", generator=gen)
        Xs, Ys = X[perm].contiguous(), Y[perm].contiguous()
        for a in range(0, ntr - batch + 1, batch):
            want = (a == 0)
            lo = net.train_step(Xs[a:a + batch], Ys[a:a + batch], batch, lr=lr_ep, want_loss=want)
            steps += 1
            if want:
                hist.append(lo)
    net.sync()
    t_train = time.perf_counter() - t0
    err_tr = relative_errors(net, X[:ntr], Y[:ntr], batch)
    err_ho = relative_errors(net, X[ntr:], Y[ntr:], batch) if nh else np.array([])
    return {"net": net, "params": net.nparam, "history": hist, "train_err": err_tr, "holdout_err": err_ho,
            "train_seconds": t_train, "steps": steps}


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
