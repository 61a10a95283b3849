// Host side of IVNet (Sec. 3.4.2, Fig. fig:net; kernels in k_ivnet.cuh, GEMMs on k_gemm_bf16): the
// convolution list, forward, backward, the paper's loss and AdamW. Included by vesb300.cu after the MLP
// part, whose GEMM launcher, loss, column statistics and AdamW kernels it shares.
//
// Parameters on the device are kept padded for the GEMMs: convolution j has W_j (coutp x kp, K index
// c k + t, zero outside C_out x C_in k) then b_j (coutp); the C ABI takes and returns the unpadded layout of
// the oracle (per convolution W (C_out x C_in x k) then b).

struct vs_ivnet {
  int N = 0, C = 0, nb = 0, Bcap = 0, nch = 2;  // nch input signals of N points
  float beta = 1.f;
  std::vector<IvConv> cv;
  std::vector<int64_t> woff, boff;  // padded flat layout
  int64_t nparam = 0, npad = 0;
  cudaStream_t stream = nullptr;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  std::vector<__nv_bfloat16*> Wb, WbT, col, colT;
  float* x0 = nullptr;                                   // input signal (N x 2)
  std::vector<float*> hs;                                // residual stream h_0 .. h_nb (N x C)
  std::vector<float*> r1, r2, u1, i1, u2, i2, cm;        // per block
  float *y16 = nullptr, *yrows = nullptr;
  float *gh = nullptr, *gi2 = nullptr, *gu2 = nullptr, *gi1 = nullptr, *gu1 = nullptr, *gr2 = nullptr, *gr1 = nullptr;
  float *gm = nullptr, *dcol = nullptr, *dy16 = nullptr, *part = nullptr, *wpart = nullptr;
  __nv_bfloat16 *gb = nullptr, *gbT = nullptr;
  float *g32 = nullptr, *ynorm = nullptr, *loss_b = nullptr, *loss = nullptr;
  __nv_bfloat16 *lbf = nullptr, *lbfT = nullptr;
  float* aff = nullptr;   // [in_shift nch N | in_scale nch N | out_shift 2N | out_scale 2N | 1/out_scale 2N]
  double* stats = nullptr;
  bool has_in = false, has_out = false;
  unsigned* err = nullptr;
  int64_t t = 0;
  std::string msg;
};

namespace {

constexpr int IV_PARTS = 512;  // row chunks of the deterministic column sums
constexpr int IV_KCHUNK = 1024;  // rows per split of the weight-gradient GEMM (split K)

// column sums of a rows x cols FP32 matrix: per-chunk partial sums, then the chunks in order
__global__ void k_iv_colsum_part(const float* __restrict__ G, int64_t rows, int cols, float* __restrict__ part) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  const int64_t per = (rows + IV_PARTS - 1) / IV_PARTS;
  const int64_t r0 = (int64_t)blockIdx.y * per, r1 = min(rows, r0 + per);
  float s = 0.f;
  for (int64_t r = r0; r < r1; ++r) s += G[r * cols + c];
  part[(int64_t)blockIdx.y * cols + c] = s;
}
__global__ void k_iv_colsum_final(const float* __restrict__ part, int cols, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int p = 0; p < IV_PARTS; ++p) s += part[(int64_t)p * cols + c];
  out[c] = s;
}

inline unsigned iv_grid(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 148 * 64); }

void ivnet_free(vs_ivnet* h) {
  auto F = [](auto* p) { cudaFree(p); };
  F(h->w); F(h->g); F(h->m); F(h->v);
  for (auto* p : h->Wb) F(p);
  for (auto* p : h->WbT) F(p);
  for (auto* p : h->col) F(p);
  for (auto* p : h->colT) F(p);
  F(h->x0);
  for (auto* p : h->hs) F(p);
  for (auto* vec : {&h->r1, &h->r2, &h->u1, &h->i1, &h->u2, &h->i2, &h->cm})
    for (auto* p : *vec) F(p);
  F(h->y16); F(h->yrows); F(h->gh); F(h->gi2); F(h->gu2); F(h->gi1); F(h->gu1); F(h->gr2); F(h->gr1);
  F(h->gm); F(h->dcol); F(h->dy16); F(h->part); F(h->wpart); F(h->gb); F(h->gbT); F(h->g32); F(h->ynorm); F(h->loss_b);
  F(h->loss); F(h->lbf); F(h->lbfT); F(h->aff); F(h->stats); F(h->err);
}

vs_status iv_gemm(vs_ivnet* h, const GemmArgs& a, int splits = 1) {
  const dim3 grid((a.N + MM_BN - 1) / MM_BN, (a.M + MM_BM - 1) / MM_BM, splits);
  k_gemm_bf16<<<grid, MM_THREADS, MM_SMEM, h->stream>>>(a);
  VS_CK(h, cudaGetLastError(), "ivnet gemm");
  return VS_OK;
}

vs_status iv_refresh_bf16(vs_ivnet* h) {
  for (size_t j = 0; j < h->cv.size(); ++j) {
    const IvConv& c = h->cv[j];
    const int64_t n = (int64_t)c.coutp * c.kp;
    k_weights_bf16<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(h->w + h->woff[j], c.coutp, c.kp, h->Wb[j],
                                                                        h->WbT[j]);
  }
  VS_CK(h, cudaGetLastError(), "ivnet weights");
  return VS_OK;
}

// convolution j of the signal src (n_in positions, leading dimension ldx) into dst + col_off (leading
// dimension ld_dst), bias and ReLU in the GEMM's epilogue; train keeps the transposed columns
vs_status iv_conv(vs_ivnet* h, int j, const float* src, int64_t ldx, int n_in, float* dst, int64_t ld_dst, int Bp,
                  bool train) {
  const IvConv& c = h->cv[j];
  const int64_t M = (int64_t)Bp * (n_in / c.s);
  k_iv_gather<<<iv_grid(M * c.kp), 256, 0, h->stream>>>(src, (int)ldx, Bp, n_in, c, h->col[j]);
  if (train) k_iv_gatherT<<<iv_grid(M * c.kp), 256, 0, h->stream>>>(src, (int)ldx, Bp, n_in, c, h->colT[j]);
  GemmArgs a = gemm_args(h->col[j], c.kp, h->Wb[j], c.kp, (int)M, c.coutp, c.kp, h->err);
  a.bias = h->w + h->boff[j];
  a.act = (j == 0 || (j < (int)h->cv.size() - 1 && (j - 1) % 7 != 6)) ? EPI_RELU : EPI_NONE;
  a.out_f32 = dst;
  a.ld_f32 = ld_dst;
  return iv_gemm(h, a);
}

vs_status iv_forward(vs_ivnet* h, const float* x, int batch, bool out_map, bool train) {
  const int Bp = round_up(batch, MM_BM), N = h->N, C = h->C, hc = C / 2;
  const int di = h->nch * N;
  k_iv_rows_in<<<iv_grid((int64_t)Bp * di), 256, 0, h->stream>>>(x, batch, Bp, N, h->nch, h->has_in ? h->aff : nullptr,
                                                                 h->aff + di, h->x0);
  vs_status st;
  if ((st = iv_conv(h, 0, h->x0, h->nch, N, h->hs[0], C, Bp, train)) != VS_OK) return st;
  for (int b = 0; b < h->nb; ++b) {
    const int j = 1 + 7 * b;
    if ((st = iv_conv(h, j, h->hs[b], C, N, h->r1[b], C, Bp, train)) != VS_OK) return st;
    if ((st = iv_conv(h, j + 1, h->hs[b], C, N, h->r1[b] + hc, C, Bp, train)) != VS_OK) return st;
    if ((st = iv_conv(h, j + 2, h->r1[b], C, N / 2, h->r2[b], C, Bp, train)) != VS_OK) return st;
    if ((st = iv_conv(h, j + 3, h->r1[b], C, N / 2, h->r2[b] + hc, C, Bp, train)) != VS_OK) return st;
    k_iv_up<<<iv_grid((int64_t)Bp * N / 2 * C), 256, 0, h->stream>>>(h->r2[b], h->r1[b], Bp, N / 4, C, h->u1[b]);
    if ((st = iv_conv(h, j + 4, h->u1[b], C, N / 2, h->i1[b], C, Bp, train)) != VS_OK) return st;
    k_iv_up<<<iv_grid((int64_t)Bp * N * C), 256, 0, h->stream>>>(h->i1[b], h->hs[b], Bp, N / 2, C, h->u2[b]);
    if ((st = iv_conv(h, j + 5, h->u2[b], C, N, h->i2[b], C, Bp, train)) != VS_OK) return st;
    if ((st = iv_conv(h, j + 6, h->i2[b], C, N, h->cm[b], C, Bp, train)) != VS_OK) return st;
    k_iv_add<<<iv_grid((int64_t)Bp * N * C), 256, 0, h->stream>>>(h->hs[b], h->cm[b], (int64_t)Bp * N * C, h->hs[b + 1]);
  }
  const int jl = (int)h->cv.size() - 1;
  if ((st = iv_conv(h, jl, h->hs[h->nb], C, N, h->y16, 16, Bp, train)) != VS_OK) return st;
  const bool om = out_map && h->has_out;
  k_iv_rows_out<<<iv_grid((int64_t)batch * 2 * N), 256, 0, h->stream>>>(h->y16, batch, N, om ? h->aff + 2 * di + 2 * N : nullptr,
                                                                          om ? h->aff + 2 * di : nullptr, h->yrows);
  VS_CK(h, cudaGetLastError(), "ivnet forward");
  return VS_OK;
}

// gradient g (channels [0, coutp) of a signal with leading dimension ldg; ReLU' from post when non-null)
// at convolution j's output: its weight and bias gradients, and when dsrc is non-null dsrc += the gradient
// at its input (n_in positions, leading dimension ld_src)
vs_status iv_back(vs_ivnet* h, int j, const float* g, int64_t ldg, const float* post, float* dsrc, int64_t ld_src,
                  int n_in, int Bp) {
  const IvConv& c = h->cv[j];
  const int64_t M = (int64_t)Bp * (n_in / c.s);
  k_iv_grad<<<iv_grid(M * c.coutp), 256, 0, h->stream>>>(g, ldg, post, M, c.coutp, h->gm, h->gb, h->gbT);
  // the weight gradient: K = M rows split into chunks of IV_KCHUNK, partial products summed in order
  const int S = (int)((M + IV_KCHUNK - 1) / IV_KCHUNK);
  GemmArgs a = gemm_args(h->gbT, M, h->colT[j], M, c.coutp, c.kp, (int)M, h->err);
  a.out_f32 = h->wpart;
  a.ld_f32 = c.kp;
  a.kchunk = IV_KCHUNK;
  a.split_ld = (int64_t)c.coutp * c.kp;
  vs_status st = iv_gemm(h, a, S);
  if (st != VS_OK) return st;
  k_iv_splitsum<<<iv_grid(a.split_ld), 256, 0, h->stream>>>(h->wpart, S, a.split_ld, h->g + h->woff[j]);
  k_iv_colsum_part<<<dim3((c.coutp + 127) / 128, IV_PARTS), 128, 0, h->stream>>>(h->gm, M, c.coutp, h->part);
  k_iv_colsum_final<<<(c.coutp + 127) / 128, 128, 0, h->stream>>>(h->part, c.coutp, h->g + h->boff[j]);
  if (dsrc) {
    GemmArgs b = gemm_args(h->gb, c.coutp, h->WbT[j], c.coutp, (int)M, c.kp, c.coutp, h->err);
    b.out_f32 = h->dcol;
    b.ld_f32 = c.kp;
    if ((st = iv_gemm(h, b)) != VS_OK) return st;
    k_iv_scatter<<<iv_grid((int64_t)Bp * n_in * c.cin), 256, 0, h->stream>>>(h->dcol, Bp, n_in, c, dsrc, ld_src);
  }
  VS_CK(h, cudaGetLastError(), "ivnet backward");
  return VS_OK;
}

vs_status iv_zero(vs_ivnet* h, float* p, int64_t n) {
  VS_CK(h, cudaMemsetAsync(p, 0, n * sizeof(float), h->stream), "ivnet zero");
  return VS_OK;
}

vs_status iv_backward(vs_ivnet* h, const float* y, int batch) {
  const int Bp = round_up(batch, MM_BM), N = h->N, C = h->C, hc = C / 2, d = 2 * N, di = h->nch * N;
  const float* ysh = h->has_out ? h->aff + 2 * di : nullptr;
  k_mlp_loss<<<Bp, 128, 0, h->stream>>>(h->yrows, y, ysh, h->aff + 2 * di + 4 * N, h->ynorm, batch, d, 2, h->beta, h->g32,
                                        h->lbf, h->lbfT, Bp, h->loss_b);
  k_mean<<<1, 32, 0, h->stream>>>(h->loss_b, batch, h->loss);
  k_iv_rows_grad<<<iv_grid((int64_t)Bp * N * 16), 256, 0, h->stream>>>(h->g32, Bp, N, h->dy16);
  VS_CK(h, cudaGetLastError(), "ivnet loss");
  const int64_t full = (int64_t)Bp * N * C, half = full / 2, quarter = full / 4;
  vs_status st;
  if ((st = iv_zero(h, h->gh, full)) != VS_OK) return st;
  const int jl = (int)h->cv.size() - 1;
  if ((st = iv_back(h, jl, h->dy16, 16, nullptr, h->gh, C, N, Bp)) != VS_OK) return st;
  for (int b = h->nb - 1; b >= 0; --b) {
    const int j = 1 + 7 * b;
    // gh: the gradient at h_{b+1}; the mixing convolution and the residual
    if ((st = iv_zero(h, h->gi2, full)) != VS_OK) return st;
    if ((st = iv_back(h, j + 6, h->gh, C, nullptr, h->gi2, C, N, Bp)) != VS_OK) return st;
    if ((st = iv_zero(h, h->gu2, full)) != VS_OK) return st;
    if ((st = iv_back(h, j + 5, h->gi2, C, h->i2[b], h->gu2, C, N, Bp)) != VS_OK) return st;
    // u2 = up(i1) + h_b: the skip's gradient goes to h_b
    k_iv_add<<<iv_grid(full), 256, 0, h->stream>>>(h->gh, h->gu2, full, h->gh);
    if ((st = iv_zero(h, h->gi1, half)) != VS_OK) return st;
    k_iv_up_T<<<iv_grid(half), 256, 0, h->stream>>>(h->gu2, Bp, N / 2, C, h->gi1);
    if ((st = iv_zero(h, h->gu1, half)) != VS_OK) return st;
    if ((st = iv_back(h, j + 4, h->gi1, C, h->i1[b], h->gu1, C, N / 2, Bp)) != VS_OK) return st;
    if ((st = iv_zero(h, h->gr2, quarter)) != VS_OK) return st;
    k_iv_up_T<<<iv_grid(quarter), 256, 0, h->stream>>>(h->gu1, Bp, N / 4, C, h->gr2);
    // u1 = up(r2) + r1: the skip's gradient starts r1's
    VS_CK(h, cudaMemcpyAsync(h->gr1, h->gu1, half * sizeof(float), cudaMemcpyDeviceToDevice, h->stream), "ivnet");
    if ((st = iv_back(h, j + 2, h->gr2, C, h->r2[b], h->gr1, C, N / 2, Bp)) != VS_OK) return st;
    if ((st = iv_back(h, j + 3, h->gr2 + hc, C, h->r2[b] + hc, h->gr1, C, N / 2, Bp)) != VS_OK) return st;
    if ((st = iv_back(h, j, h->gr1, C, h->r1[b], h->gh, C, N, Bp)) != VS_OK) return st;
    if ((st = iv_back(h, j + 1, h->gr1 + hc, C, h->r1[b] + hc, h->gh, C, N, Bp)) != VS_OK) return st;
  }
  return iv_back(h, 0, h->gh, C, h->hs[0], nullptr, 0, N, Bp);
}

vs_status iv_check_err(vs_ivnet* h) {
  unsigned e = 0;
  VS_CK(h, cudaStreamSynchronize(h->stream), "ivnet sync");
  VS_CK(h, cudaMemcpy(&e, h->err, sizeof e, cudaMemcpyDeviceToHost), "ivnet error word");
  if (e & ERR_MMA_TIMEOUT) { h->msg = "tensor-core GEMM wait timed out"; return VS_ERR_TIMEOUT; }
  return VS_OK;
}

// unpadded (oracle) <-> padded (device) parameter vectors
void iv_pad(const vs_ivnet* h, const float* p, std::vector<float>& out) {
  out.assign(h->npad, 0.f);
  int64_t o = 0;
  for (size_t j = 0; j < h->cv.size(); ++j) {
    const IvConv& c = h->cv[j];
    for (int r = 0; r < c.cout; ++r)
      for (int q = 0; q < c.cin * c.k; ++q) out[h->woff[j] + (int64_t)r * c.kp + q] = p[o + (int64_t)r * c.cin * c.k + q];
    o += (int64_t)c.cout * c.cin * c.k;
    for (int r = 0; r < c.cout; ++r) out[h->boff[j] + r] = p[o + r];
    o += c.cout;
  }
}
void iv_unpad(const vs_ivnet* h, const std::vector<float>& q, float* p) {
  int64_t o = 0;
  for (size_t j = 0; j < h->cv.size(); ++j) {
    const IvConv& c = h->cv[j];
    for (int r = 0; r < c.cout; ++r)
      for (int e = 0; e < c.cin * c.k; ++e) p[o + (int64_t)r * c.cin * c.k + e] = q[h->woff[j] + (int64_t)r * c.kp + e];
    o += (int64_t)c.cout * c.cin * c.k;
    for (int r = 0; r < c.cout; ++r) p[o + r] = q[h->boff[j] + r];
    o += c.cout;
  }
}

}  // namespace

extern "C" {

vs_status vs_ivnet_create(int32_t N, int32_t in_channels, int32_t C, int32_t nblocks, int32_t max_batch, float beta,
                          void* cuda_stream, vs_ivnet** out) {
  if (!out) return VS_ERR_INVALID_ARG;
  *out = nullptr;
  if (N < 8 || N > NMAX || N % 4 != 0 || C < 32 || C > 1024 || C % 32 != 0 || nblocks < 1 || max_batch < 1 ||
      in_channels < 1 || in_channels > 16 || !(beta >= 0.f)) {
    g_create_msg = "IVNet needs N a multiple of 4 in [8, 128], 1 to 16 input signals, C a multiple of 32 in "
                   "[32, 1024], nblocks >= 1";
    return VS_ERR_INVALID_ARG;
  }
  if ((int64_t)round_up(max_batch, MM_BM) * N * round_up(3 * C, 16) >= (1ll << 31)) {
    g_create_msg = "IVNet: max_batch x N x 3C must stay below 2^31 (32-bit column indices)";
    return VS_ERR_INVALID_ARG;
  }
  vs_ivnet* h = new (std::nothrow) vs_ivnet();
  if (!h) return VS_ERR_NOMEM;
  h->N = N; h->C = C; h->nb = nblocks; h->Bcap = round_up(max_batch, MM_BM); h->beta = beta;
  h->nch = in_channels;
  h->stream = (cudaStream_t)cuda_stream;
  const int hc = C / 2;
  auto add = [&](int ci, int co, int k, int s, int d) {
    IvConv c{ci, co, k, s, d, round_up(ci * k, 16), std::max(16, round_up(co, 16))};
    h->cv.push_back(c);
  };
  add(in_channels, C, 3, 1, 1);
  for (int b = 0; b < nblocks; ++b) {
    add(C, hc, 3, 2, 1); add(C, hc, 3, 2, 2); add(C, hc, 3, 2, 1); add(C, hc, 3, 2, 2);
    add(C, C, 3, 1, 1); add(C, C, 3, 1, 1); add(C, C, 1, 1, 1);
  }
  add(C, 2, 1, 1, 1);
  int64_t o = 0;
  for (const IvConv& c : h->cv) {
    h->woff.push_back(o); o += (int64_t)c.coutp * c.kp;
    h->boff.push_back(o); o += c.coutp;
    h->nparam += (int64_t)c.cout * c.cin * c.k + c.cout;
  }
  h->npad = o;
  cudaError_t e;
  auto fail = [&](cudaError_t ee) {
    cuda_fail(g_create_msg, ee, "vs_ivnet_create");
    ivnet_free(h);
    delete h;
    return ee == cudaErrorMemoryAllocation ? VS_ERR_NOMEM : VS_ERR_CUDA;
  };
#define VS_I(x) do { e = (x); if (e != cudaSuccess) return fail(e); } while (0)
  const int64_t B = h->Bcap, full = B * N * C;
  VS_I(dalloc(&h->w, h->npad)); VS_I(dalloc(&h->g, h->npad)); VS_I(dalloc(&h->m, h->npad)); VS_I(dalloc(&h->v, h->npad));
  int64_t mk = 0, mc = 0;  // largest columns (M kp) and gradient (M coutp) sizes
  int n_in = N;
  for (size_t j = 0; j < h->cv.size(); ++j) {
    const IvConv& c = h->cv[j];
    // input length of convolution j: N for the lift, the block's h and i2/u2 and the projection, N/2 for
    // the second restriction level and i1 (on u1)
    const int r = j == 0 ? 0 : (j == h->cv.size() - 1 ? 6 : (int)((j - 1) % 7));
    n_in = (r == 2 || r == 3 || r == 4) ? N / 2 : N;
    const int64_t M = B * (n_in / c.s);
    __nv_bfloat16 *wb, *wbt, *cl, *clt;
    VS_I(dalloc(&wb, (int64_t)c.coutp * c.kp)); h->Wb.push_back(wb);
    VS_I(dalloc(&wbt, (int64_t)c.coutp * c.kp)); h->WbT.push_back(wbt);
    VS_I(dalloc(&cl, M * c.kp)); h->col.push_back(cl);
    VS_I(dalloc(&clt, M * c.kp)); h->colT.push_back(clt);
    mk = std::max(mk, M * c.kp);
    mc = std::max(mc, M * c.coutp);
  }
  VS_I(dalloc(&h->x0, B * N * in_channels));
  for (int b = 0; b <= nblocks; ++b) { float* p; VS_I(dalloc(&p, full)); h->hs.push_back(p); }
  for (int b = 0; b < nblocks; ++b) {
    float* p;
    VS_I(dalloc(&p, full / 2)); h->r1.push_back(p);
    VS_I(dalloc(&p, full / 4)); h->r2.push_back(p);
    VS_I(dalloc(&p, full / 2)); h->u1.push_back(p);
    VS_I(dalloc(&p, full / 2)); h->i1.push_back(p);
    VS_I(dalloc(&p, full)); h->u2.push_back(p);
    VS_I(dalloc(&p, full)); h->i2.push_back(p);
    VS_I(dalloc(&p, full)); h->cm.push_back(p);
  }
  VS_I(dalloc(&h->y16, B * N * 16)); VS_I(dalloc(&h->yrows, B * 2 * N));
  VS_I(dalloc(&h->gh, full)); VS_I(dalloc(&h->gi2, full)); VS_I(dalloc(&h->gu2, full)); VS_I(dalloc(&h->gi1, full / 2));
  VS_I(dalloc(&h->gu1, full / 2)); VS_I(dalloc(&h->gr2, full / 4)); VS_I(dalloc(&h->gr1, full / 2));
  VS_I(dalloc(&h->gm, mc)); VS_I(dalloc(&h->gb, mc)); VS_I(dalloc(&h->gbT, mc)); VS_I(dalloc(&h->dcol, mk));
  VS_I(dalloc(&h->dy16, B * N * 16)); VS_I(dalloc(&h->part, (int64_t)IV_PARTS * std::max(C, 16)));
  int64_t wmax = 0;
  for (const IvConv& c : h->cv) wmax = std::max(wmax, (int64_t)c.coutp * c.kp);
  VS_I(dalloc(&h->wpart, wmax * ((B * N + IV_KCHUNK - 1) / IV_KCHUNK)));
  VS_I(dalloc(&h->g32, B * 2 * N)); VS_I(dalloc(&h->ynorm, B * 2 * N)); VS_I(dalloc(&h->loss_b, B));
  VS_I(dalloc(&h->loss, 1)); VS_I(dalloc(&h->lbf, B * 2 * N)); VS_I(dalloc(&h->lbfT, B * 2 * N));
  const int64_t di = (int64_t)in_channels * N;
  VS_I(dalloc(&h->aff, 2 * di + 6 * (int64_t)N)); VS_I(dalloc(&h->stats, 2 * std::max(di, 2 * (int64_t)N)));
  VS_I(dalloc(&h->err, 1));
  VS_I(cudaMemset(h->err, 0, sizeof(unsigned)));
  VS_I(cudaMemset(h->w, 0, h->npad * sizeof(float)));
  VS_I(cudaMemset(h->m, 0, h->npad * sizeof(float)));
  VS_I(cudaMemset(h->v, 0, h->npad * sizeof(float)));
  VS_I(cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, MM_SMEM));
  {
    std::vector<float> a(2 * di + 6 * (size_t)N, 0.f);
    for (int i = 0; i < di; ++i) a[di + i] = 1.f;
    for (int i = 0; i < 2 * N; ++i) { a[2 * di + 2 * N + i] = 1.f; a[2 * di + 4 * N + i] = 1.f; }
    VS_I(cudaMemcpy(h->aff, a.data(), a.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
#undef VS_I
  if (iv_refresh_bf16(h) != VS_OK) return fail(cudaErrorUnknown);
  *out = h;
  return VS_OK;
}

vs_status vs_ivnet_num_params(const vs_ivnet* h, int64_t* n) {
  if (!h || !n) return VS_ERR_INVALID_ARG;
  *n = h->nparam;
  return VS_OK;
}

vs_status vs_ivnet_set_params(vs_ivnet* h, const float* p, int64_t n) {
  if (!h || !p || n != h->nparam) return VS_ERR_INVALID_ARG;
  std::vector<float> q;
  iv_pad(h, p, q);
  VS_CK(h, cudaMemcpyAsync(h->w, q.data(), h->npad * sizeof(float), cudaMemcpyHostToDevice, h->stream), "set params");
  VS_CK(h, cudaMemsetAsync(h->m, 0, h->npad * sizeof(float), h->stream), "set params");
  VS_CK(h, cudaMemsetAsync(h->v, 0, h->npad * sizeof(float), h->stream), "set params");
  h->t = 0;
  vs_status st = iv_refresh_bf16(h);
  if (st != VS_OK) return st;
  VS_CK(h, cudaStreamSynchronize(h->stream), "set params");
  return VS_OK;
}

vs_status vs_ivnet_get_params(vs_ivnet* h, float* p, int64_t n) {
  if (!h || !p || n != h->nparam) return VS_ERR_INVALID_ARG;
  std::vector<float> q(h->npad);
  VS_CK(h, cudaMemcpyAsync(q.data(), h->w, h->npad * sizeof(float), cudaMemcpyDeviceToHost, h->stream), "get params");
  VS_CK(h, cudaStreamSynchronize(h->stream), "get params");
  iv_unpad(h, q, p);
  return VS_OK;
}

vs_status vs_ivnet_set_affine(vs_ivnet* h, const float* in_shift, const float* in_scale, const float* out_shift,
                              const float* out_scale) {
  if (!h) return VS_ERR_INVALID_ARG;
  const int di = h->nch * h->N, d = 2 * h->N;
  std::vector<float> a(2 * (size_t)di + 3 * (size_t)d);
  for (int j = 0; j < di; ++j) {
    a[j] = in_shift ? in_shift[j] : 0.f;
    a[di + j] = in_scale ? in_scale[j] : 1.f;
  }
  for (int j = 0; j < d; ++j) {
    a[2 * di + j] = out_shift ? out_shift[j] : 0.f;
    const float t = out_scale ? out_scale[j] : 1.f;
    if (!(t != 0.f) || !std::isfinite(t)) return VS_ERR_INVALID_ARG;
    a[2 * di + d + j] = t;
    a[2 * di + 2 * d + j] = 1.f / t;
  }
  for (float x : a)
    if (!std::isfinite(x)) return VS_ERR_INVALID_ARG;
  VS_CK(h, cudaMemcpyAsync(h->aff, a.data(), a.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream), "set affine");
  VS_CK(h, cudaStreamSynchronize(h->stream), "set affine");
  h->has_in = in_shift || in_scale;
  h->has_out = out_shift || out_scale;
  return VS_OK;
}

vs_status vs_ivnet_fit_affine(vs_ivnet* h, const float* x, const float* y, int32_t rows, double rel_floor) {
  if (!h || !x || !y || rows < 1 || !(rel_floor >= 0.0)) return VS_ERR_INVALID_ARG;
  const int dims[2] = {h->nch * h->N, 2 * h->N};
  const int dmx = std::max(dims[0], dims[1]);
  std::vector<double> st(2 * (size_t)dmx);
  std::vector<float> sh[2], sc[2];
  for (int pass = 0; pass < 2; ++pass) {
    const int d = dims[pass];
    k_colstats<<<(d + 127) / 128, 128, 0, h->stream>>>(pass ? y : x, rows, d, h->stats, h->stats + dmx);
    VS_CK(h, cudaGetLastError(), "fit affine");
    VS_CK(h, cudaMemcpyAsync(st.data(), h->stats, 2 * dmx * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
          "fit affine");
    VS_CK(h, cudaStreamSynchronize(h->stream), "fit affine");
    double sdmax = 0.0;
    for (int j = 0; j < d; ++j)
      if (std::isfinite(st[dmx + j])) sdmax = std::max(sdmax, st[dmx + j]);
    sh[pass].resize(d);
    sc[pass].resize(d);
    for (int j = 0; j < d; ++j) {
      const double sd = std::max(st[dmx + j], rel_floor * sdmax);
      const bool flat = !(sd > 0.0) || !std::isfinite(sd);
      sh[pass][j] = (float)st[j];
      sc[pass][j] = flat ? 1.f : (float)(pass ? sd : 1.0 / sd);
    }
  }
  return vs_ivnet_set_affine(h, sh[0].data(), sc[0].data(), sh[1].data(), sc[1].data());
}

vs_status vs_ivnet_forward(vs_ivnet* h, const float* x, int32_t batch, float* y) {
  if (!h || !x || !y || batch < 1 || batch > h->Bcap) return VS_ERR_INVALID_ARG;
  vs_status st = iv_forward(h, x, batch, true, false);
  if (st != VS_OK) return st;
  VS_CK(h, cudaMemcpyAsync(y, h->yrows, (size_t)batch * 2 * h->N * sizeof(float), cudaMemcpyDeviceToDevice, h->stream),
        "ivnet forward out");
  return VS_OK;
}

vs_status vs_ivnet_loss_grad(vs_ivnet* h, const float* x, const float* y, int32_t batch, float* loss, float* grad,
                             int64_t n) {
  if (!h || !x || !y || !loss || batch < 1 || batch > h->Bcap) return VS_ERR_INVALID_ARG;
  if (grad && n != h->nparam) return VS_ERR_INVALID_ARG;
  vs_status st = iv_forward(h, x, batch, false, true);
  if (st == VS_OK) st = iv_backward(h, y, batch);
  if (st != VS_OK) return st;
  VS_CK(h, cudaMemcpyAsync(loss, h->loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream), "loss");
  if (grad) {
    std::vector<float> q(h->npad);
    VS_CK(h, cudaMemcpyAsync(q.data(), h->g, h->npad * sizeof(float), cudaMemcpyDeviceToHost, h->stream), "grad");
    if ((st = iv_check_err(h)) != VS_OK) return st;
    iv_unpad(h, q, grad);
    return VS_OK;
  }
  return iv_check_err(h);
}

vs_status vs_ivnet_train_step(vs_ivnet* h, const float* x, const float* y, int32_t batch, const vs_adamw* opt,
                              float* loss) {
  if (!h || !x || !y || !opt || batch < 1 || batch > h->Bcap) return VS_ERR_INVALID_ARG;
  vs_status st = iv_forward(h, x, batch, false, true);
  if (st == VS_OK) st = iv_backward(h, y, batch);
  if (st != VS_OK) return st;
  h->t += 1;
  const float c1 = 1.f - powf(opt->beta1, (float)h->t), c2 = 1.f - powf(opt->beta2, (float)h->t);
  k_adamw<<<(unsigned)((h->npad + 255) / 256), 256, 0, h->stream>>>(h->w, h->g, h->m, h->v, h->npad, opt->lr,
                                                                     opt->beta1, opt->beta2, opt->eps,
                                                                     opt->weight_decay, c1, c2);
  VS_CK(h, cudaGetLastError(), "ivnet adamw");
  if ((st = iv_refresh_bf16(h)) != VS_OK) return st;
  if (loss) {
    VS_CK(h, cudaMemcpyAsync(loss, h->loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream), "loss");
    return iv_check_err(h);
  }
  return VS_OK;
}

vs_status vs_ivnet_sync(vs_ivnet* h) {
  if (!h) return VS_ERR_INVALID_ARG;
  return iv_check_err(h);
}

const char* vs_ivnet_last_error(const vs_ivnet* h) { return h ? h->msg.c_str() : g_create_msg.c_str(); }

void vs_ivnet_destroy(vs_ivnet* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  ivnet_free(h);
  delete h;
}

vs_status vs_feature_points(const float* feat, int32_t rows, int64_t ld, int32_t N, int32_t K, float* out,
                            void* cuda_stream) {
  if (!feat || !out || rows < 1 || N < 8 || N > NMAX || K < 0 || K > N / 2 - 1 || ld < 4 * K + 2)
    return VS_ERR_INVALID_ARG;
  k_feature_points<<<iv_grid((int64_t)rows * 2 * N), 256, 0, (cudaStream_t)cuda_stream>>>(feat, rows, ld, N, K, out);
  return cudaGetLastError() == cudaSuccess ? VS_OK : VS_ERR_CUDA;
}

}  // extern "C"
