"""FP64 multilayer perceptron: forward, backward, loss and AdamW (Sec. 3.4.2). Test infrastructure only.

The paper's networks are IVNets; the learned part here is a fully connected network (ReLU on the
hidden layers, affine output) trained with the paper's loss and optimiser:
    loss = mean_b ( ||Yhat_b - Y_b|| / ||Y_b|| + beta ||D(Yhat_b - Y_b)|| / ||D Y_b|| )     (Sec. 3.4.2)
D = the periodic forward difference along the discretisation index inside each of the `ncomp`
equal blocks of an output vector (its "derivative with respect to discretization"), and AdamW
with the decoupled weight decay w <- w (1 - lr wd) - lr mhat / (sqrt(vhat) + eps).
Parameters of layer l: W_l (d_{l+1} x d_l, row-major) and b_l (d_{l+1}); the flat parameter
vector is every W_l then every b_l, in layer order.

Optional per-feature affine maps (feature normalisation of the data): affine = (in_shift, in_scale,
out_shift, out_scale); the first layer sees (x - in_shift) * in_scale and the output is
z * out_scale + out_shift for the last layer's value z; the loss compares z with the mapped targets
(y - out_shift) / out_scale. With bf16=True the two maps of the inputs and targets are taken in
float32 as the GPU does (subtract, then multiply by the float32 scale or float32 reciprocal).

bf16=True rounds the GEMM operands (inputs, hidden activations, weights) to bfloat16 (round to
nearest even) where the tensor-core path does, accumulating in FP64; gradients are then those of
the rounded forward pass (straight-through), as the GPU computes them.

Pins (tests/test_oracle_mlp.py): gradients against central finite differences (FP64, rel 1e-7),
AdamW's first step in closed form, the loss of a perfect prediction is zero, and the affine maps
against the same network with the maps folded into its first and last layers.
"""
import numpy as np


def bf16_round(a):
    """Round float64 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(dims, rng):
    """He-uniform weights, zero biases (flat vector)."""
    ws, bs = [], []
    for a, b in zip(dims[:-1], dims[1:]):
        lim = np.sqrt(6.0 / a)
        ws.append(rng.uniform(-lim, lim, size=(b, a)).ravel())
        bs.append(np.zeros(b))
    return np.concatenate(ws + bs)


def unpack(params, dims):
    ws, bs = [], []
    o = 0
    for a, b in zip(dims[:-1], dims[1:]):
        ws.append(params[o:o + a * b].reshape(b, a))
        o += a * b
    for b in dims[1:]:
        bs.append(params[o:o + b])
        o += b
    return ws, bs


def map_inputs(X, affine, bf16):
    """(X - in_shift) * in_scale (float32 arithmetic when bf16, else FP64)."""
    X = np.asarray(X, dtype=np.float64)
    if affine is None:
        return X
    sh, sc = affine[0], affine[1]
    if bf16:
        f32 = np.float32
        return ((X.astype(f32) - np.asarray(sh, f32)) * np.asarray(sc, f32)).astype(np.float64)
    return (X - np.asarray(sh, np.float64)) * np.asarray(sc, np.float64)


def map_targets(Y, affine, bf16):
    """(Y - out_shift) / out_scale, as (Y - out_shift) * float32(1/out_scale) in float32 when bf16."""
    Y = np.asarray(Y, dtype=np.float64)
    if affine is None:
        return Y
    sh, sc = affine[2], affine[3]
    if bf16:
        f32 = np.float32
        inv = (f32(1.0) / np.asarray(sc, f32)).astype(f32)
        return ((Y.astype(f32) - np.asarray(sh, f32)) * inv).astype(np.float64)
    return (Y - np.asarray(sh, np.float64)) / np.asarray(sc, np.float64)


def forward(params, dims, X, bf16=False, affine=None, out_map=True):
    """Returns (Y, cache). X: (batch, d0). With affine, out_map=False returns the last layer's value
    before the output map (the quantity the loss sees)."""
    ws, bs = unpack(params, dims)
    rd = bf16_round if bf16 else (lambda a: a)
    H = [rd(map_inputs(X, affine, bf16))]
    L = len(ws)
    for l in range(L):
        Z = H[-1] @ rd(ws[l]).T + bs[l]
        if l < L - 1:
            H.append(rd(np.maximum(Z, 0.0)))
        else:
            Y = Z
    if affine is not None and out_map:
        Y = Y * np.asarray(affine[3], np.float64) + np.asarray(affine[2], np.float64)
    return Y, H


def _diff(E, ncomp):
    B, d = E.shape
    n = d // ncomp
    Eb = E.reshape(B, ncomp, n)
    return (np.roll(Eb, -1, axis=2) - Eb).reshape(B, d)


def _diff_T(G, ncomp):
    B, d = G.shape
    n = d // ncomp
    Gb = G.reshape(B, ncomp, n)
    return (np.roll(Gb, 1, axis=2) - Gb).reshape(B, d)


def loss_and_grad_output(Yhat, Y, beta, ncomp):
    """Loss (Sec. 3.4.2) and its gradient with respect to Yhat."""
    B = Y.shape[0]
    E = Yhat - Y
    ne = np.linalg.norm(E, axis=1)
    ny = np.linalg.norm(Y, axis=1)
    DE, DY = _diff(E, ncomp), _diff(Y, ncomp)
    nde = np.linalg.norm(DE, axis=1)
    ndy = np.linalg.norm(DY, axis=1)
    loss = np.mean(ne / ny + beta * nde / ndy)
    with np.errstate(invalid="ignore", divide="ignore"):
        g1 = np.where(ne[:, None] > 0, E / (ne * ny)[:, None], 0.0)
        g2 = np.where(nde[:, None] > 0, _diff_T(DE, ncomp) / (nde * ndy)[:, None], 0.0)
    return loss, (g1 + beta * g2) / B


def backward(params, dims, cache, dY, bf16=False):
    """Gradient of sum(dY * Y) with respect to the flat parameters."""
    ws, bs = unpack(params, dims)
    rd = bf16_round if bf16 else (lambda a: a)
    L = len(ws)
    gws, gbs = [None] * L, [None] * L
    G = dY
    for l in range(L - 1, -1, -1):
        Gr = rd(G)
        gws[l] = Gr.T @ cache[l]
        gbs[l] = G.sum(axis=0)
        if l > 0:
            G = (Gr @ rd(ws[l])) * (cache[l] > 0)
    return np.concatenate([g.ravel() for g in gws] + gbs)


def loss_and_gradient(params, dims, X, Y, beta=1.0, ncomp=2, bf16=False, affine=None):
    Yhat, cache = forward(params, dims, X, bf16, affine, out_map=False)
    loss, dY = loss_and_grad_output(Yhat, map_targets(Y, affine, bf16), beta, ncomp)
    return loss, backward(params, dims, cache, dY, bf16)


class AdamW:
    """AdamW (Sec. 3.4.2: learning rate 1e-3) with the standard defaults."""

    def __init__(self, n, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.01):
        self.lr, self.b1, self.b2, self.eps, self.wd = lr, beta1, beta2, eps, weight_decay
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0

    def step(self, w, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return w * (1 - self.lr * self.wd) - self.lr * mh / (np.sqrt(vh) + self.eps)
