"""IVNet, the paper's network (Sec. 3.4.2, Fig. fig:net), for 1D periodic signals along a vesicle: forward,
backward and the loss of oracle.mlp. Test infrastructure only.

A sample is the N points of a standardised vesicle as cin signals (two: x, y; or more, e.g. the shape's
low and high Fourier modes as separate signals); the output is N points of two channels (the relaxation
displacement). Signals are laid out (batch, position, channel); every
convolution is circular (the curve is closed), with k taps centred on the output position:
    out[p, o] = b[o] + sum_c sum_t W[o, c, t] in[(s p + d (t - (k - 1) / 2)) mod n_in, c]
(stride s, dilation d). The network (Fig. fig:net, with L = 2 levels):
    h_0 = relu(conv_{k=3}(x; cin -> C))                                        (lift)
    block i (n_b blocks):  r1 = [relu(R_1^1 h) | relu(R_1^2 h)]       (two paths of C/2 channels, stride 2,
                                                                        dilations 1 and 2; length N/2)
                           r2 = [relu(R_2^1 r1) | relu(R_2^2 r1)]     (length N/4)
                           i1 = relu(conv_3(up(r2) + r1))             (length N/2)
                           i2 = relu(conv_3(up(i1) + h_i))            (length N)
                           h_{i+1} = h_i + conv_1(i2)                 (the mixing convolution C_m, residual)
    y = conv_1(h_{n_b}; C -> 2)                                              (projection)
up: periodic linear interpolation by 2 (out[2q] = in[q], out[2q+1] = (in[q] + in[q+1]) / 2).
Readings (the figure fixes the two restriction paths, their dilations, the concatenation, the two
interpolations, the mixing convolution and the residual; the paper gives no kernel sizes, activation,
channel counts at each level or lifting): kernel size 3 (1 for the mixing and the projection), ReLU after
every convolution but the mixing one and the projection, each restriction path C/2 channels so that the
concatenation has C, the interpolation added to the finer level's signal of the descent (a multigrid
V-cycle adds the prolongated coarse correction to the finer level; without it a block could only add
signals that passed through the coarsest level) and then a convolution (the figure's upsampling "via
direct convolutions"), a lifting convolution from the input signals to C channels and a projection back to
two.

Parameters: per convolution, in the order lift, (R_1^1, R_1^2, R_2^1, R_2^2, I_1, I_2, C_m) per block,
projection: W (C_out x C_in x k, row-major) then b (C_out). The per-feature affine maps, the loss and
AdamW are those of oracle.mlp, on rows [x(N), y(N)] (ncomp = 2).

bf16=True rounds the convolution operands (the gathered inputs and the weights) and the output gradient
to bfloat16 where the tensor-core path does, accumulating in FP64 (activations, sums and the residual
stream stay unrounded); gradients are those of the rounded forward pass.

Pins (tests/test_oracle_ivnet.py): a convolution against its definition by explicit loops, the
interpolation against its adjoint, gradients against central finite differences (FP64), equivariance
under cyclic shifts of the points by multiples of 4 (the two stride-2 levels), the parameter count.
"""
import numpy as np

from .mlp import bf16_round, loss_and_grad_output, map_inputs, map_targets


def convs(C, nb, cin=2):
    """(C_in, C_out, k, stride, dilation, relu) of every convolution, in parameter order (cin input
    signals)."""
    h = C // 2
    out = [(cin, C, 3, 1, 1, True)]
    for _ in range(nb):
        out += [(C, h, 3, 2, 1, True), (C, h, 3, 2, 2, True), (C, h, 3, 2, 1, True), (C, h, 3, 2, 2, True),
                (C, C, 3, 1, 1, True), (C, C, 3, 1, 1, True), (C, C, 1, 1, 1, False)]
    out.append((C, 2, 1, 1, 1, False))
    return out


def param_count(C, nb, cin=2):
    return sum(co * ci * k + co for ci, co, k, _, _, _ in convs(C, nb, cin))


def unpack(params, C, nb, cin=2):
    ws, bs, o = [], [], 0
    for ci, co, k, _, _, _ in convs(C, nb, cin):
        ws.append(params[o:o + co * ci * k].reshape(co, ci, k))
        o += co * ci * k
        bs.append(params[o:o + co])
        o += co
    return ws, bs


def init_params(C, nb, rng, cin=2):
    """He-uniform weights (fan-in C_in k), zero biases."""
    out = []
    for ci, co, k, _, _, _ in convs(C, nb, cin):
        lim = np.sqrt(6.0 / (ci * k))
        out += [rng.uniform(-lim, lim, co * ci * k), np.zeros(co)]
    return np.concatenate(out)


def gather(x, k, s, d):
    """The convolution's input columns: col[b, p, c k + t] = x[b, (s p + d (t - (k-1)/2)) mod n, c]."""
    B, n, c = x.shape
    no = n // s
    p = np.arange(no)[:, None]
    t = np.arange(k)[None, :]
    idx = (s * p + d * (t - (k - 1) // 2)) % n  # (no, k)
    g = x[:, idx, :]  # (B, no, k, c)
    return g.transpose(0, 1, 3, 2).reshape(B, no, c * k)


def scatter(dcol, n, c, k, s, d):
    """Adjoint of gather: the input gradient from the columns' gradient."""
    B, no, _ = dcol.shape
    p = np.arange(no)[:, None]
    t = np.arange(k)[None, :]
    idx = (s * p + d * (t - (k - 1) // 2)) % n
    g = dcol.reshape(B, no, c, k).transpose(0, 1, 3, 2)  # (B, no, k, c)
    out = np.zeros((B, n, c))
    for tt in range(k):
        np.add.at(out, (slice(None), idx[:, tt], slice(None)), g[:, :, tt, :])
    return out


def up(x):
    """Periodic linear interpolation by 2 along positions."""
    nx = np.roll(x, -1, axis=1)
    B, n, c = x.shape
    out = np.empty((B, 2 * n, c))
    out[:, 0::2] = x
    out[:, 1::2] = 0.5 * (x + nx)
    return out


def up_T(g):
    """Adjoint of up."""
    e, o = g[:, 0::2], g[:, 1::2]
    return e + 0.5 * o + 0.5 * np.roll(o, 1, axis=1)


def conv(x, W, b, k, s, d, rd):
    col = rd(gather(x, k, s, d))
    co = W.shape[0]
    return col @ rd(W.reshape(co, -1)).T + b, col


def to_points(rows, N):
    """rows [s_0(N), s_1(N), ...] -> (B, N, channels)."""
    B = rows.shape[0]
    return rows.reshape(B, -1, N).transpose(0, 2, 1)


def to_rows(x):
    B, N, _ = x.shape
    return x.transpose(0, 2, 1).reshape(B, 2 * N)


def forward(params, C, nb, X, bf16=False, affine=None, out_map=True, cin=2):
    """Y (batch, 2N) for inputs X (batch, cin N) = rows of cin signals of N points ([x(N), y(N)] for cin = 2);
    returns (Y, cache)."""
    ws, bs = unpack(params, C, nb, cin)
    spec = convs(C, nb, cin)
    rd = bf16_round if bf16 else (lambda a: a)
    N = X.shape[1] // cin
    x = to_points(map_inputs(X, affine, bf16), N)
    cache = []

    def apply(j, inp):
        ci, co, k, s, d, relu = spec[j]
        z, col = conv(inp, ws[j], bs[j], k, s, d, rd)
        out = np.maximum(z, 0.0) if relu else z
        cache.append((j, inp.shape, col, out))
        return out

    h = apply(0, x)
    j = 1
    for _ in range(nb):
        r1 = np.concatenate([apply(j, h), apply(j + 1, h)], axis=2)
        r2 = np.concatenate([apply(j + 2, r1), apply(j + 3, r1)], axis=2)
        i1 = apply(j + 4, up(r2) + r1)
        i2 = apply(j + 5, up(i1) + h)
        h = h + apply(j + 6, i2)
        j += 7
    y = to_rows(apply(j, h))
    if affine is not None and out_map:
        y = y * np.asarray(affine[3], np.float64) + np.asarray(affine[2], np.float64)
    return y, cache


def backward(params, C, nb, cache, dY, bf16=False, cin=2):
    """Gradient of sum(dY * Y) (Y before the output map) with respect to the flat parameters."""
    ws, _ = unpack(params, C, nb, cin)
    spec = convs(C, nb, cin)
    rd = bf16_round if bf16 else (lambda a: a)
    entries = {j: (shape, col, out) for j, shape, col, out in cache}
    gw, gb = [None] * len(spec), [None] * len(spec)

    def back(j, g):
        """g: gradient at conv j's output; returns the gradient at its input."""
        ci, co, k, s, d, relu = spec[j]
        shape, col, out = entries[j]
        if relu:
            g = g * (out > 0)
        B, no, _ = g.shape
        gr = rd(g).reshape(B * no, co)
        gw[j] = (gr.T @ col.reshape(B * no, -1)).reshape(co, ci, k)
        gb[j] = g.reshape(B * no, co).sum(axis=0)
        dcol = (gr @ rd(ws[j].reshape(co, -1))).reshape(B, no, ci * k)
        return scatter(dcol, shape[1], ci, k, s, d)

    N = dY.shape[1] // 2
    j = len(spec) - 1
    gh = back(j, to_points(dY, N))
    hC = C // 2
    for blk in range(nb - 1, -1, -1):
        j = 1 + 7 * blk
        gi2 = back(j + 6, gh)
        gu2 = back(j + 5, gi2)
        gu1 = back(j + 4, up_T(gu2))
        gr2 = up_T(gu1)
        gr1 = gu1 + back(j + 2, gr2[:, :, :hC]) + back(j + 3, gr2[:, :, hC:])
        gh = gh + gu2 + back(j, gr1[:, :, :hC]) + back(j + 1, gr1[:, :, hC:])
    back(0, gh)
    return np.concatenate([np.concatenate([w.ravel(), b]) for w, b in zip(gw, gb)])


def loss_and_gradient(params, C, nb, X, Y, beta=1.0, bf16=False, affine=None, cin=2):
    Yhat, cache = forward(params, C, nb, X, bf16, affine, out_map=False, cin=cin)
    loss, dY = loss_and_grad_output(Yhat, map_targets(Y, affine, bf16), beta, 2)
    return loss, backward(params, C, nb, cache, dY, bf16, cin)
