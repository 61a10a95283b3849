// Near-field correction: five layers + Gaussian RBF (Sec. 3.3, Algorithm 4, App. A).
//
// For every source vesicle v with at least one near target (recorded by the far-field kernel):
//  k_near_layers  the 5N layer points X + d h n, d in {-1, -1/2, 0, 1/2, 1}, and the exact
//                 single layer S[X, f] there: on the curve S f with the cached self matrix (FP64 sums),
//                 off the curve the trapezoid rule on the curve upsampled by rho = ceil(sqrt(N)), in FP32
//                 (the RBF that takes these values is FP32) with the far field's log scaling: each
//                 target's log arguments scaled by a power of two near 1 / (|x - c|^2 + reach^2) and the
//                 exponent times the density sum added once;
//                 With the learned near field (Sec. 3.3, Eq. NearFieldMap; k_near_layers<true>) the layer
//                 velocities come from the networks' rows instead: the density's Fourier features in the
//                 vesicle's standard frame combine the columns of each layer (the layer velocities of the
//                 basis densities at the unit-length standardised shape, mu = 1), and
//                 S[X, f_K] = L R^T shift(sum_i c_i Q_d,i) / mu - (L log L / (4 pi mu)) I_d for the density's
//                 modes <= Kf, f_K, I_d the integral of f_K over the unit-length curve by the layer's own
//                 quadrature (the N points on the curve, the upsampled curve off it);
//                 With the Ying-Zorin scheme (VS_FLAG_NEAR_YZ; k_near_layers<NEAR_YZ> + k_near_yz) the layers
//                 and the RBF are replaced by the evaluation of Sec. 2.2.2 at each near target (k_near_yz).
//  k_near_rbf     (Phi + lam I) w = u_layers, Phi_ab = exp(-|x_a - x_b|^2 / (c h)^2), c = 2,
//                 lam = 1e-3, by an FP32 Cholesky (the paper's precision): k_near_rbf_smem holds the
//                 lower triangle in shared memory (5N <= 320), k_near_rbf works in the vesicle's scratch;
//  k_near_apply   u(x_t) += sum_b phi(|x_t - x_b|) w_b for each near (target, vesicle) pair.
#pragma once
#include "common.cuh"
#include "k_dense.cuh"
#include "k_farfield.cuh"
#include "k_standardize.cuh"
#include "k_vesicle.cuh"

namespace vs {

constexpr double NEAR_RBF_C = 2.0;
constexpr double NEAR_RBF_NUGGET = 1e-3;
constexpr int NEAR_LAYERS = 5;
__device__ __constant__ double c_layer_d[NEAR_LAYERS] = {-1.0, -0.5, 0.0, 0.5, 1.0};

__device__ __forceinline__ int near_rho(int N) { return (int)ceil(sqrt((double)N)); }

// Mark source vesicles that have near targets.
__global__ void k_near_mark(int64_t P, const int* __restrict__ near_cnt, const int* __restrict__ near_v,
                            int* __restrict__ has_near) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P) return;
  const int c = near_cnt[t];
  for (int k = 0; k < c; ++k) has_near[near_v[t * MAX_NEAR + k]] = 1;
}

// involved[v] = 1 for every vesicle in a near pair: the owner of a target with near vesicles and each
// of those vesicles.
__global__ void k_near_involved(int64_t P, const int32_t* __restrict__ owner, const int* __restrict__ near_cnt,
                                const int* __restrict__ near_v, int* __restrict__ involved) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P) return;
  const int c = near_cnt[t];
  if (c > 0) involved[owner[t]] = 1;
  for (int k = 0; k < c; ++k) involved[near_v[t * MAX_NEAR + k]] = 1;
}

// involved[a] = 1 when a point of vesicle a lies within gap_h times the larger spacing h = L/N of the two
// vesicles from a point of another vesicle b. One CTA per vesicle a: the threads screen the other vesicles
// by their bounding circles (centre, reach = largest distance to the centre plus h) and collect the
// candidates, which are then compared point by point. More than PROX_CAND candidates counts as a hit.
constexpr int PROX_CAND = 64;
__global__ void __launch_bounds__(128) k_proximity(VesIndex vi, const double* __restrict__ xy,
                                                   const double2* __restrict__ centre, const float2* __restrict__ h2,
                                                   int M, double gap_h, int* __restrict__ involved) {
  __shared__ float px[NMAX], py[NMAX];
  __shared__ int cand[PROX_CAND];
  __shared__ int nc, hit;
  const int a = vi.vid(blockIdx.x);
  const int Na = vi.N[a];
  const int64_t oa = vi.off[a];
  const double2 ca = centre[a];
  const float2 ha = h2[a];
  for (int i = threadIdx.x; i < Na; i += blockDim.x) {
    px[i] = (float)(xy[2 * oa + i] - ca.x);
    py[i] = (float)(xy[2 * oa + Na + i] - ca.y);
  }
  if (threadIdx.x == 0) { nc = 0; hit = 0; }
  __syncthreads();
  const float ra = sqrtf(ha.y), hA = sqrtf(ha.x);
  for (int b = threadIdx.x; b < M; b += blockDim.x) {
    if (b == a) continue;
    const float2 hb = h2[b];
    const double2 cb = centre[b];
    const float dx = (float)(cb.x - ca.x), dy = (float)(cb.y - ca.y);
    const float lim = ra + sqrtf(hb.y) + (float)gap_h * fmaxf(hA, sqrtf(hb.x));
    if (dx * dx + dy * dy <= lim * lim) {
      const int k = atomicAdd(&nc, 1);
      if (k < PROX_CAND) cand[k] = b;
    }
  }
  __syncthreads();
  const int n = min(nc, PROX_CAND);
  if (nc > PROX_CAND && threadIdx.x == 0) hit = 1;
  __syncthreads();
  for (int c = 0; c < n && !hit; ++c) {  // hit is read after a barrier: uniform
    const int b = cand[c];
    const int Nb = vi.N[b];
    const int64_t ob = vi.off[b];
    const float gap = (float)gap_h * fmaxf(hA, sqrtf(h2[b].x));
    float mn = 3.0e38f;
    for (int j = threadIdx.x; j < Nb; j += blockDim.x) {
      const float qx = (float)(xy[2 * ob + j] - ca.x), qy = (float)(xy[2 * ob + Nb + j] - ca.y);
      for (int i = 0; i < Na; ++i) {
        const float rx = qx - px[i], ry = qy - py[i];
        mn = fminf(mn, rx * rx + ry * ry);
      }
    }
    if (mn <= gap * gap) hit = 1;  // every writer stores 1
    __syncthreads();
  }
  if (threadIdx.x == 0 && hit) involved[a] = 1;
}

// Hybrid fallback statistics (one CTA): acc[0] += number of vesicles flagged for the exact step, acc[1] += 1.
__global__ void __launch_bounds__(256) k_count_flags(int M, const int* __restrict__ flag,
                                                      unsigned long long* __restrict__ acc) {
  __shared__ int part[8];
  int c = 0;
  for (int v = threadIdx.x; v < M; v += blockDim.x) c += flag[v] != 0;
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    acc[0] += (unsigned long long)t;
    acc[1] += 1ull;
  }
}

struct NearBufs {
  double* layer;   // per vesicle at 30 off[v]: LX, LY, UX, UY, WX, WY (5N each)
  float* phi;      // per vesicle at moff[v]: (5N)^2 floats
};

// The learned near field's inputs: one network output row per vesicle and layer (row v of layer d at
// rows[d] + v ld: the nb = 4 Kf + 2 columns of velocity features up to Kout, 2 (2 Kout + 1) floats each) and
// the standardisation frames of the same step.
struct NearNets {
  const float* rows[NEAR_LAYERS];
  int64_t ld;
  int Kf, Kout;
  const StdFrame* frames;
};

// Learned layer velocities of vesicle v (all threads of the CTA; module header), written to UX, UY (5N each,
// layer-major, the vesicle's own point labels): those of f_K, the density's modes <= Kf. gs = the upsampled
// quadrature's density sums sum_q f_K,u |X'_u| (2 pi / Nu) / (4 pi mu), the off-curve layers' integral of f_K
// times L / (4 pi mu).
__device__ void near_learned_layers(const NearNets& nn, int v, int N, int64_t o, const double* T,
                                    const double* __restrict__ f, PointGeom g, double L, double mu,
                                    const double* gs, double* UX, double* UY) {
  __shared__ double w[2][NMAX];
  __shared__ double c[4 * (NMAX / 2) + 2];
  __shared__ double gd[NEAR_LAYERS][2 * NMAX];
  __shared__ double ic[2], red[8];
  const int t = threadIdx.x;
  const StdFrame fr = nn.frames[v];
  // f in the frame: rotated and relabelled
  for (int k = t; k < N; k += blockDim.x) {
    const int i = (k + fr.j0) % N;
    const double fx = f[2 * o + i], fy = f[2 * o + N + i];
    w[0][k] = fr.ct * fx - fr.st * fy;
    w[1][k] = fr.st * fx + fr.ct * fy;
  }
  __syncthreads();
  // its features (modes <= Kf)
  const int pf = 2 * nn.Kf + 1, nbasis = 2 * pf;
  for (int e = t; e < nbasis; e += blockDim.x) {
    const int cc = e / pf, r = e - cc * pf;
    const int q = r <= nn.Kf ? r : r - nn.Kf;
    const int off = r <= nn.Kf ? 15 * N : 16 * N;
    double acc = 0.0;
    int m = 0;
    for (int j = 0; j < N; ++j) {
      acc = fma(w[cc][j], T[off + m], acc);
      m += q;
      if (m >= N) m -= N;
    }
    c[e] = (r <= nn.Kf ? acc : -acc) / N;
  }
  __syncthreads();
  // the integral of f_K (the density's modes <= Kf, synthesised from c and turned back to the vesicle's
  // axes) over the curve by the N-point trapezoid rule, the on-curve layer's quadrature
  double ax = 0.0, ay = 0.0;
  for (int k = t; k < N; k += blockDim.x) {
    double a = c[0], b = c[pf];
    int m = 0;
    for (int q = 1; q <= nn.Kf; ++q) {
      m += k;
      if (m >= N) m -= N;
      const double cs = T[15 * N + m], sn = T[16 * N + m];
      a += 2.0 * (c[q] * cs - c[nn.Kf + q] * sn);
      b += 2.0 * (c[pf + q] * cs - c[pf + nn.Kf + q] * sn);
    }
    const double sa = g.sa[o + (k + fr.j0) % N];
    ax += (fr.ct * a + fr.st * b) * sa;
    ay += (-fr.st * a + fr.ct * b) * sa;
  }
  ax = block_sum(ax, red);
  ay = block_sum(ay, red);
  if (t == 0) { ic[0] = ax * (2.0 * VS_PI / N); ic[1] = ay * (2.0 * VS_PI / N); }
  // each layer's velocity features: the columns combined
  const int po = 2 * nn.Kout + 1, cw = 2 * po;
  for (int e = t; e < NEAR_LAYERS * cw; e += blockDim.x) {
    const int d = e / cw, k = e - d * cw;
    const float* row = nn.rows[d] + (int64_t)v * nn.ld;
    double acc = 0.0;
    for (int i = 0; i < nbasis; ++i) acc = fma(c[i], (double)row[i * cw + k], acc);
    gd[d][k] = acc;
  }
  __syncthreads();
  // synthesis at frame label k, back to the vesicle's label and axes, scaled
  const double sc = L / mu, k0 = -L * log(L) / (4.0 * VS_PI * mu);
  const double iux = 4.0 * VS_PI * mu * gs[0] / L, iuy = 4.0 * VS_PI * mu * gs[1] / L;  // off-curve integrals
  const double icx = ic[0] / L, icy = ic[1] / L;                                     // on-curve integrals
  for (int e = t; e < NEAR_LAYERS * N; e += blockDim.x) {
    const int d = e / N, k = e - d * N;
    const double* G = gd[d];
    double a = G[0], b = G[po];
    int m = 0;
    for (int q = 1; q <= nn.Kout; ++q) {
      m += k;
      if (m >= N) m -= N;
      const double cs = T[15 * N + m], sn = T[16 * N + m];
      a += 2.0 * (G[q] * cs - G[nn.Kout + q] * sn);
      b += 2.0 * (G[po + q] * cs - G[po + nn.Kout + q] * sn);
    }
    const int i = (k + fr.j0) % N;
    const bool on = d == NEAR_LAYERS / 2;
    UX[d * N + i] = sc * (fr.ct * a + fr.st * b) + k0 * (on ? icx : iux);
    UY[d * N + i] = sc * (-fr.st * a + fr.ct * b) + k0 * (on ? icy : iuy);
  }
}

// Layer points and exact layer velocities. Dynamic shared memory: near_layers_smem(N) bytes.
inline size_t near_layers_smem(int N) {
  const int Nu = (int)std::ceil(std::sqrt((double)N)) * N;
  return (size_t)Nu * sizeof(float4) + 2 * (size_t)Nu * sizeof(float);
}

// What k_near_layers computes for each near source vesicle: the exact layer velocities, the learned ones, or
// (NEAR_YZ) the per-vesicle data of the Ying-Zorin evaluation (k_near_yz).
enum : int { NEAR_EXACT = 0, NEAR_LEARNED = 1, NEAR_YZ = 2 };

// Ying-Zorin data of a source vesicle at 30 off[v] in nb.layer (doubles): the FP64 Fourier coefficients
// (re, im; k = 0..N/2) of x, y and of the on-curve single layer u0 = S f (x and y components), then gsum_x,
// gsum_y, the mean point (cx, cy) and reach^2, then the upsampled sources as float4 (x - cx, y - cy, g_x, g_y).
struct YzLayout {
  int N;
  __host__ __device__ int cx() const { return 0; }
  __host__ __device__ int cy() const { return N + 2; }
  __host__ __device__ int ux() const { return 2 * N + 4; }
  __host__ __device__ int uy() const { return 3 * N + 6; }
  __host__ __device__ int misc() const { return 4 * N + 8; }
  __host__ __device__ int src() const { return 4 * N + 16; }  // doubles; 16-byte aligned
};

template <int MODE>
__global__ void __launch_bounds__(256) k_near_layers(VesIndex vi, const int* __restrict__ has_near,
                                                     const double* __restrict__ xy, const double* __restrict__ f,
                                                     PointGeom g, const double* __restrict__ length,
                                                     const double* __restrict__ tab,
                                                     const double* __restrict__ scratch,
                                                     const float* __restrict__ scratch32, int s, double mu,
                                                     NearBufs nb, NearNets nn) {
  extern __shared__ float4 smf[];
  const int v = vi.vid(blockIdx.x);
  if (!has_near[v]) return;
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int rho = near_rho(N), Nu = rho * N;
  const int tid = threadIdx.x;
  float4* src = smf;                  // upsampled points relative to the mean point, and g (Nu)
  float* cs = (float*)(smf + Nu);     // cos(2 pi q / Nu)
  float* sn = cs + Nu;                // sin(2 pi q / Nu)
  __shared__ float cre[4][NMAX / 2 + 1], cim[4][NMAX / 2 + 1];
  __shared__ double fl[2 * NMAX], gsum[2], cmean[2], red[8];
  const double* T = tab + vi.toff[v];
  for (int q = tid; q < Nu; q += blockDim.x) sincospif(2.f * q / Nu, &sn[q], &cs[q]);
  for (int r = tid; r < 2 * N; r += blockDim.x) fl[r] = f[2 * o + r];
  // Fourier coefficients of x, y, f_x, f_y (k = 0..N/2), FP64 sums; the curve's relative to its mean point
  const int nk = N / 2 + 1;
  for (int e = tid; e < 4 * nk; e += blockDim.x) {
    const int comp = e / nk, k = e - comp * nk;
    const double* sv = (comp < 2) ? (xy + 2 * o + comp * N) : (f + 2 * o + (comp - 2) * N);
    double re = 0.0, im = 0.0;
    int m = 0;
    for (int j = 0; j < N; ++j) {
      re = fma(sv[j], T[15 * N + m], re);
      im = fma(-sv[j], T[16 * N + m], im);
      m += k;
      if (m >= N) m -= N;
    }
    if (comp < 2 && k == 0) cmean[comp] = re / N;
    cre[comp][k] = (comp < 2 && k == 0) ? 0.f : (float)(re / N);
    cim[comp][k] = (float)(im / N);
    if (MODE == NEAR_YZ && comp < 2) {
      double* Y = nb.layer + 30 * o + (comp == 0 ? YzLayout{N}.cx() : YzLayout{N}.cy());
      Y[2 * k] = re / N;
      Y[2 * k + 1] = im / N;
    }
  }
  __syncthreads();
  if constexpr (MODE == NEAR_LEARNED) {  // the learned layers are those of the density's modes <= Kf: truncate it
    for (int e = tid; e < 2 * nk; e += blockDim.x) {
      const int comp = 2 + e / nk, k = e - (comp - 2) * nk;
      if (k > nn.Kf) { cre[comp][k] = 0.f; cim[comp][k] = 0.f; }
    }
    __syncthreads();
  }
  const double cx = cmean[0], cy = cmean[1];
  // upsampled curve (relative to the mean point), its speed, and g = f |X_alpha| (2 pi / Nu) / (4 pi mu)
  const float cw = (float)(2.0 * VS_PI / Nu / (4.0 * VS_PI * mu));
  double gxs = 0.0, gys = 0.0;
  float r2max = 0.f;
  for (int q = tid; q < Nu; q += blockDim.x) {
    float val[4], dx = 0.f, dy = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) val[c] = cre[c][0];
    int idx = 0;
    for (int k = 1; k < N / 2; ++k) {
      idx += q;
      if (idx >= Nu) idx %= Nu;
      const float ck = cs[idx], sk = sn[idx];
#pragma unroll
      for (int c = 0; c < 4; ++c) val[c] += 2.f * (cre[c][k] * ck - cim[c][k] * sk);
      dx -= 2.f * k * (cre[0][k] * sk + cim[0][k] * ck);
      dy -= 2.f * k * (cre[1][k] * sk + cim[1][k] * ck);
    }
    const int iN = (int)(((int64_t)q * (N / 2)) % Nu);
#pragma unroll
    for (int c = 0; c < 4; ++c) val[c] += cre[c][N / 2] * cs[iN];
    dx -= cre[0][N / 2] * (N / 2) * sn[iN];
    dy -= cre[1][N / 2] * (N / 2) * sn[iN];
    const float w = sqrtf(dx * dx + dy * dy) * cw;
    src[q] = make_float4(val[0], val[1], val[2] * w, val[3] * w);
    gxs += (double)(val[2] * w);
    gys += (double)(val[3] * w);
    r2max = fmaxf(r2max, val[0] * val[0] + val[1] * val[1]);
  }
  gxs = block_sum(gxs, red);
  gys = block_sum(gys, red);
  const double rmax = block_max((double)r2max, red);
  if (tid == 0) {
    gsum[0] = gxs;
    gsum[1] = gys;
  }
  __syncthreads();
  const double h = length[v] / N;
  const float reach2 = (float)(rmax + h * h);
  double* L = nb.layer + 30 * o;
  double* LX = L;
  double* LY = L + 5 * N;
  double* UX = L + 10 * N;
  double* UY = L + 15 * N;
  // S at slot s: FP64, or (mixed-precision path, scratch32 set) the FP32 split S_hi + S_lo
  const int64_t NN = (int64_t)N * N;
  const double* S = scratch + vi.moff[v] + (MatLayout::slot(s) + MatLayout::S) * NN;
  const float* Sh = scratch32 ? scratch32 + vi.moff[v] + (MatLayout::slot(s) + MatLayout::S) * NN : nullptr;
  const float* Sl = scratch32 ? scratch32 + vi.moff[v] + (MatLayout::slot(s) + MatLayout::SL) * NN : nullptr;
  const float hl2 = -0.34657359027997264f;  // -ln(2)/2: -log|r| = hl2 log2|r|^2
  if constexpr (MODE == NEAR_YZ) {
    // the on-curve single layer u0 = S f, its Fourier coefficients, the sums and the upsampled sources
    __shared__ double u0[2 * NMAX];
    for (int r = tid; r < 2 * N; r += blockDim.x) {
      double a = 0.0;
      for (int k = 0; k < 2 * N; ++k) {
        const int64_t e = (int64_t)r * 2 * N + k;
        a = fma(Sh ? (double)Sh[e] + (double)Sl[e] : S[e], fl[k], a);
      }
      u0[r] = a;
    }
    __syncthreads();
    const YzLayout lay{N};
    double* Yv = nb.layer + 30 * o;
    for (int e = tid; e < 2 * nk; e += blockDim.x) {
      const int comp = e / nk, k = e - comp * nk;
      double re = 0.0, im = 0.0;
      int m = 0;
      for (int j = 0; j < N; ++j) {
        re = fma(u0[comp * N + j], T[15 * N + m], re);
        im = fma(-u0[comp * N + j], T[16 * N + m], im);
        m += k;
        if (m >= N) m -= N;
      }
      double* C = Yv + (comp == 0 ? lay.ux() : lay.uy());
      C[2 * k] = re / N;
      C[2 * k + 1] = im / N;
    }
    if (tid == 0) {
      double* mi = Yv + lay.misc();
      mi[0] = gsum[0];
      mi[1] = gsum[1];
      mi[2] = cx;
      mi[3] = cy;
      mi[4] = (double)reach2;
    }
    float4* so = reinterpret_cast<float4*>(Yv + lay.src());
    for (int q = tid; q < Nu; q += blockDim.x) so[q] = src[q];
    return;
  }
  if constexpr (MODE == NEAR_LEARNED) {
    for (int e = tid; e < 5 * N; e += blockDim.x) {
      const int lay = e / N, j = e - lay * N;
      const double d = c_layer_d[lay] * h;
      LX[e] = xy[2 * o + j] + d * g.ty[o + j];
      LY[e] = xy[2 * o + N + j] - d * g.tx[o + j];
    }
    near_learned_layers(nn, v, N, o, T, f, g, length[v], mu, gsum, UX, UY);
    return;
  }
  for (int e = tid; e < 5 * N; e += blockDim.x) {
    const int lay = e / N, j = e - lay * N;
    const double d = c_layer_d[lay] * h;
    const double nx = g.ty[o + j], ny = -g.tx[o + j];
    const double px = xy[2 * o + j] + d * nx, py = xy[2 * o + N + j] + d * ny;
    LX[e] = px;
    LY[e] = py;
    double ax = 0.0, ay = 0.0;
    if (lay == 2) {  // on the curve: S f
      for (int k = 0; k < 2 * N; ++k) {
        const int64_t ex = (int64_t)j * 2 * N + k, ey = (int64_t)(N + j) * 2 * N + k;
        const double sx = Sh ? (double)Sh[ex] + (double)Sl[ex] : S[ex];
        const double sy = Sh ? (double)Sh[ey] + (double)Sl[ey] : S[ey];
        ax = fma(sx, fl[k], ax);
        ay = fma(sy, fl[k], ay);
      }
    } else {  // off the curve: FP32 trapezoid sums on the upsampled curve
      const float tx = (float)(px - cx), ty = (float)(py - cy);
      float le;
      const float sc = pow2_scale(fmaf(tx, tx, ty * ty) + reach2, le);
      float lx = 0.f, ly = 0.f, qx = 0.f, qy = 0.f;
      for (int m = 0; m < Nu; ++m) {
        const float4 sm = src[m];
        const float rx = tx - sm.x, ry = ty - sm.y;
        const float r2 = fmaf(rx, rx, ry * ry);
        const float lg = fast_lg2(r2 * sc);
        const float q = fmaf(rx, sm.z, ry * sm.w) * fast_rcp(r2);
        lx = fmaf(lg, sm.z, lx);
        ly = fmaf(lg, sm.w, ly);
        qx = fmaf(q, rx, qx);
        qy = fmaf(q, ry, qy);
      }
      ax = (double)hl2 * ((double)lx + (double)le * gsum[0]) + (double)qx;
      ay = (double)hl2 * ((double)ly + (double)le * gsum[1]) + (double)qy;
    }
    UX[e] = ax;
    UY[e] = ay;
  }
}

// Ying-Zorin evaluation (Sec. 2.2.2, Fig. fig:near-singular; the near-singular scheme of the paper's BIEM
// ground truth): for every near (target, source vesicle) pair, u += S[X_v, f_v](x) by
//  1. the closest point x0 = X(alpha0) of the source's trigonometric interpolant (Newton on
//     (X - x) . X' = 0 from the nearest point, FP64);
//  2. the on-curve single layer at alpha0 from the Fourier coefficients of u0 = S f;
//  3. the single layer at x0 + s i beta h n, i = 1..YZ_M (s: the target's side), by FP32 trapezoid sums on
//     the upsampled curve with the far field's log scaling;
//  4. the interpolating polynomial in the distance t = |x - x0| (Lagrange form, FP64).
// One warp per target point (grid-stride over targets); the lanes split the modes and the upsampled sources.
constexpr int YZ_M = 6;
constexpr double YZ_BETA = 0.25;
constexpr int YZ_NEWTON = 30;

__device__ __forceinline__ double warp_sum_all(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// X, X', X'' of the interpolant with coefficients C (re, im pairs, k = 0..N/2) at alpha: each lane sums its
// modes, the warp adds them (all lanes get the totals). The Nyquist mode enters the value only.
__device__ inline void yz_curve(const double* C, int N, double a, double& v, double& d1, double& d2) {
  const int lane = threadIdx.x & 31;
  double sv = 0.0, s1 = 0.0, s2 = 0.0;
  for (int k = lane; k <= N / 2; k += 32) {
    double sn, cs;
    sincos(k * a, &sn, &cs);
    const double re = C[2 * k], im = C[2 * k + 1];
    const double c = re * cs - im * sn;  // Re(c_k e^{ik a})
    if (k == 0) {
      sv += re;
    } else if (k == N / 2) {
      sv += re * cs;
    } else {
      sv += 2.0 * c;
      s1 += -2.0 * k * (re * sn + im * cs);
      s2 += -2.0 * (double)k * k * c;
    }
  }
  v = warp_sum_all(sv);
  d1 = warp_sum_all(s1);
  d2 = warp_sum_all(s2);
}

__global__ void __launch_bounds__(128) k_near_yz(int64_t P, const int32_t* __restrict__ owner,
                                                 const int64_t* __restrict__ off, const int32_t* __restrict__ Nv,
                                                 const int* __restrict__ near_cnt, const int* __restrict__ near_v,
                                                 const double* __restrict__ xy, const double* __restrict__ length,
                                                 const double* __restrict__ layer, double* __restrict__ u) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < P; t += warps) {
    const int cnt = min(near_cnt[t], MAX_NEAR);
    if (cnt == 0) continue;
    const int a = owner[t];
    const int64_t oa = off[a];
    const int Na = Nv[a];
    const int ia = (int)(t - oa);
    const double px = xy[2 * oa + ia], py = xy[2 * oa + Na + ia];
    double ax = 0.0, ay = 0.0;
    for (int c = 0; c < cnt; ++c) {
      const int v = near_v[t * MAX_NEAR + c];
      const int N = Nv[v];
      const int64_t o = off[v];
      const YzLayout lay{N};
      const double* Y = layer + 30 * o;
      // 1. the nearest of the N points, then Newton on the interpolant
      double best = 1e300;
      int jb = 0;
      for (int j = lane; j < N; j += 32) {
        const double dx = xy[2 * o + j] - px, dy = xy[2 * o + N + j] - py;
        const double d2 = dx * dx + dy * dy;
        if (d2 < best) { best = d2; jb = j; }
      }
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, s);
        const int oj = __shfl_xor_sync(0xffffffffu, jb, s);
        if (ob < best || (ob == best && oj < jb)) { best = ob; jb = oj; }
      }
      double al = 2.0 * VS_PI * jb / N;
      double X, X1, X2, Yc, Y1, Y2;
      for (int it = 0; it < YZ_NEWTON; ++it) {
        yz_curve(Y + lay.cx(), N, al, X, X1, X2);
        yz_curve(Y + lay.cy(), N, al, Yc, Y1, Y2);
        const double g = (X - px) * X1 + (Yc - py) * Y1;
        const double gp = X1 * X1 + Y1 * Y1 + (X - px) * X2 + (Yc - py) * Y2;
        const double step = g / gp;
        al -= step;
        if (fabs(step) < 1e-15) break;
      }
      yz_curve(Y + lay.cx(), N, al, X, X1, X2);
      yz_curve(Y + lay.cy(), N, al, Yc, Y1, Y2);
      const double sp = sqrt(X1 * X1 + Y1 * Y1);
      const double nx = Y1 / sp, ny = -X1 / sp;
      const double sd = ((px - X) * nx + (py - Yc) * ny) >= 0.0 ? 1.0 : -1.0;
      const double tq = sqrt((px - X) * (px - X) + (py - Yc) * (py - Yc));
      // 2. the on-curve value at alpha0
      double vx[YZ_M + 1], vy[YZ_M + 1], d;
      yz_curve(Y + lay.ux(), N, al, vx[0], d, d);
      yz_curve(Y + lay.uy(), N, al, vy[0], d, d);
      // 3. the points along the normal: FP32 trapezoid sums on the upsampled curve
      const double* mi = Y + lay.misc();
      const double gsx = mi[0], gsy = mi[1], cx = mi[2], cy = mi[3];
      const float reach2 = (float)mi[4];
      const float4* src = reinterpret_cast<const float4*>(Y + lay.src());
      const int Nu = near_rho(N) * N;
      const double h = length[v] / N;
      const float hl2 = -0.34657359027997264f;
#pragma unroll
      for (int i = 1; i <= YZ_M; ++i) {
        const double di = sd * i * YZ_BETA * h;
        const float tx = (float)(X + di * nx - cx), ty = (float)(Yc + di * ny - cy);
        float le;
        const float sc = pow2_scale(fmaf(tx, tx, ty * ty) + reach2, le);
        float lx = 0.f, ly = 0.f, qx = 0.f, qy = 0.f;
        for (int m = lane; m < Nu; m += 32) {
          const float4 sm = src[m];
          const float rx = tx - sm.x, ry = ty - sm.y;
          const float r2 = fmaf(rx, rx, ry * ry);
          const float lg = fast_lg2(r2 * sc);
          const float q = fmaf(rx, sm.z, ry * sm.w) * fast_rcp(r2);
          lx = fmaf(lg, sm.z, lx);
          ly = fmaf(lg, sm.w, ly);
          qx = fmaf(q, rx, qx);
          qy = fmaf(q, ry, qy);
        }
        const double Lx = warp_sum_all((double)lx), Ly = warp_sum_all((double)ly);
        const double Qx = warp_sum_all((double)qx), Qy = warp_sum_all((double)qy);
        vx[i] = (double)hl2 * (Lx + (double)le * gsx) + Qx;
        vy[i] = (double)hl2 * (Ly + (double)le * gsy) + Qy;
      }
      // 4. Lagrange interpolation at t in units of beta h
      const double tt = tq / (YZ_BETA * h);
#pragma unroll
      for (int i = 0; i <= YZ_M; ++i) {
        double w = 1.0;
#pragma unroll
        for (int j = 0; j <= YZ_M; ++j)
          if (j != i) w *= (tt - j) / (double)(i - j);
        ax = fma(w, vx[i], ax);
        ay = fma(w, vy[i], ay);
      }
    }
    if (lane == 0) {
      u[2 * oa + ia] += ax;
      u[2 * oa + Na + ia] += ay;
    }
  }
}

// Row v, columns [col, col + 2 (2K + 1)) of `rows` = the velocity features (modes <= K; a_0..a_K, b_1..b_K
// of x, then of y) of layer d's velocities in nb.layer, for the vesicles flagged in has_near (the training
// rows of the learned near field: the layers of the standardised points, whose labels are the frame's).
__global__ void __launch_bounds__(NMAX) k_layer_features(VesIndex vi, const int* __restrict__ has_near,
                                                         const double* __restrict__ layer, int d,
                                                         const double* __restrict__ tab, int K,
                                                         float* __restrict__ rows, int64_t ld, int col) {
  __shared__ double u[2][NMAX];
  const int v = vi.vid(blockIdx.x);
  if (!has_near[v]) return;
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int t = threadIdx.x;
  const double* T = tab + vi.toff[v];
  const double* L = layer + 30 * o;
  if (t < N) {
    u[0][t] = L[10 * N + d * N + t];
    u[1][t] = L[15 * N + d * N + t];
  }
  __syncthreads();
  const int per = 2 * K + 1;
  float* row = rows + (int64_t)v * ld + col;
  for (int e = t; e < 2 * per; e += blockDim.x) {
    const int c = e / per, r = e - c * per;
    const int q = r <= K ? r : r - K;
    const int off = r <= K ? 15 * N : 16 * N;
    double acc = 0.0;
    int m = 0;
    for (int j = 0; j < N; ++j) {
      acc = fma(u[c][j], T[off + m], acc);
      m += q;
      if (m >= N) m -= N;
    }
    row[e] = (float)((r <= K ? acc : -acc) / N);
  }
}

// FP32 Cholesky of (Phi + lam I) and the two RBF weight vectors for 5N <= 320, the lower triangle held
// packed in shared memory (row i at i (i + 1) / 2; dynamic shared memory near_rbf_smem(5N) bytes). One CTA
// per near vesicle, right-looking and blocked by panels of RBF_NB columns: warp 0 factors the panel's
// diagonal block (a column a lane, in registers), one thread a row solves the panel below it against that
// block (also copied, transposed, to a panel buffer), and the trailing triangle takes the panel's
// rank-RBF_NB update in 4 x 4 register tiles; three barriers a panel instead of two a column. The
// triangular solves go by the same panels (warp 0 the diagonal block, every thread a row of the update
// below or above it), and one step of iterative refinement follows (the residual with Phi formed again),
// which removes the factorisation's rounding growth from the weights. The coordinate differences are taken
// in float pairs (hi + lo of each layer point relative to the first), accurate to FP32 in the difference.
constexpr int NEAR_RBF_SMEM_N = 320;
constexpr int RBF_NB = 16;  // panel width
// The packed triangle (n (n + 1) / 2 floats, rounded up to a multiple of 4), then the panel buffer
// (RBF_NB rows of rbf_ld(n) floats; in the solves: the coordinates and the vectors).
__host__ __device__ inline int rbf_ld(int n) { return (n + 3) & ~3; }
__host__ __device__ inline size_t rbf_tri(int n) { return ((size_t)n * (n + 1) / 2 + 3) & ~(size_t)3; }
inline size_t near_rbf_smem(int n) { return (rbf_tri(n) + (size_t)RBF_NB * rbf_ld(n)) * sizeof(float); }

__device__ __forceinline__ float rbf_phi(const float* c, int ld, int i, int j, float ie2) {
  // c: x hi, x lo, y hi, y lo rows of ld floats
  const float dx = (c[i] - c[j]) + (c[ld + i] - c[ld + j]);
  const float dy = (c[2 * ld + i] - c[2 * ld + j]) + (c[3 * ld + i] - c[3 * ld + j]);
  float p = expf(-(dx * dx + dy * dy) * ie2);
  if (i == j) p += (float)NEAR_RBF_NUGGET;
  return p;
}

// The layer points relative to the first as float pairs into c (four rows of ld floats).
__device__ __forceinline__ void rbf_coords(const double* LX, const double* LY, int n, int ld, float* c) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = LX[i] - LX[0], y = LY[i] - LY[0];
    const float xh = (float)x, yh = (float)y;
    c[i] = xh;
    c[ld + i] = (float)(x - (double)xh);
    c[2 * ld + i] = yh;
    c[3 * ld + i] = (float)(y - (double)yh);
  }
}

// Solves L L^T z = b in place for two vectors (b1, b2 in shared memory), L packed in sA, by panels of RBF_NB:
// forward, then backward; all threads of the CTA (two barriers a panel and direction).
__device__ void rbf_solve2(const float* sA, int n, float* b1, float* b2) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int c0 = 0; c0 < n; c0 += RBF_NB) {  // forward: L y = b
    const int w = min(RBF_NB, n - c0), c1 = c0 + w;
    if (wid == 0) {  // lane r: row c0 + r of the diagonal block; y_t broadcast as it is found
      const int i = c0 + lane;
      const float* row = sA + (size_t)i * (i + 1) / 2 + c0;
      float a1 = lane < w ? b1[i] : 0.f, a2 = lane < w ? b2[i] : 0.f;
      const float dii = lane < w ? row[lane] : 1.f;
#pragma unroll
      for (int t = 0; t < RBF_NB; ++t) {
        if (t >= w) break;
        if (lane == t) { a1 /= dii; a2 /= dii; }
        const float y1 = __shfl_sync(0xffffffffu, a1, t), y2 = __shfl_sync(0xffffffffu, a2, t);
        if (lane > t && lane < w) {
          const float l = row[t];
          a1 = fmaf(-l, y1, a1);
          a2 = fmaf(-l, y2, a2);
        }
      }
      if (lane < w) { b1[i] = a1; b2[i] = a2; }
    }
    __syncthreads();
    for (int i = c1 + tid; i < n; i += blockDim.x) {
      const float* row = sA + (size_t)i * (i + 1) / 2 + c0;
      float s1 = b1[i], s2 = b2[i];
      for (int t = 0; t < w; ++t) {
        s1 = fmaf(-row[t], b1[c0 + t], s1);
        s2 = fmaf(-row[t], b2[c0 + t], s2);
      }
      b1[i] = s1;
      b2[i] = s2;
    }
    __syncthreads();
  }
  const int last = ((n - 1) / RBF_NB) * RBF_NB;
  for (int c0 = last; c0 >= 0; c0 -= RBF_NB) {  // backward: L^T z = y
    const int w = min(RBF_NB, n - c0), c1 = c0 + w;
    if (wid == 0) {  // lane j: unknown c0 + j; z_i broadcast as it is found, from the last row up
      const int j = c0 + lane;
      float a1 = lane < w ? b1[j] : 0.f, a2 = lane < w ? b2[j] : 0.f;
      const float djj = lane < w ? sA[(size_t)j * (j + 1) / 2 + j] : 1.f;
#pragma unroll
      for (int t = RBF_NB - 1; t >= 0; --t) {
        if (t >= w) continue;
        if (lane == t) { a1 /= djj; a2 /= djj; }
        const float z1 = __shfl_sync(0xffffffffu, a1, t), z2 = __shfl_sync(0xffffffffu, a2, t);
        if (lane < t) {  // L[c0 + t][c0 + lane]
          const float l = sA[(size_t)(c0 + t) * (c0 + t + 1) / 2 + c0 + lane];
          a1 = fmaf(-l, z1, a1);
          a2 = fmaf(-l, z2, a2);
        }
      }
      if (lane < w) { b1[j] = a1; b2[j] = a2; }
    }
    __syncthreads();
    for (int k = tid; k < c0; k += blockDim.x) {  // earlier unknowns: y_k -= sum_i L[i][k] z_i
      float s1 = b1[k], s2 = b2[k];
      for (int t = 0; t < w; ++t) {
        const float l = sA[(size_t)(c0 + t) * (c0 + t + 1) / 2 + k];
        s1 = fmaf(-l, b1[c0 + t], s1);
        s2 = fmaf(-l, b2[c0 + t], s2);
      }
      b1[k] = s1;
      b2[k] = s2;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(512) k_near_rbf_smem(VesIndex vi, const int* __restrict__ has_near,
                                                       const double* __restrict__ length, NearBufs nb,
                                                       unsigned* err) {
  extern __shared__ float sA[];
  __shared__ int bad;
  const int v = vi.vid(blockIdx.x);
  if (!has_near[v]) return;
  const int N = vi.N[v];
  const int n = 5 * N;
  const int64_t o = vi.off[v];
  float* Pt = sA + rbf_tri(n);  // [RBF_NB][ld]: the panel's rows below its diagonal block, transposed
  const int ld = rbf_ld(n);
  const double h = length[v] / N;
  const float ie2 = (float)(1.0 / (NEAR_RBF_C * h * NEAR_RBF_C * h));
  double* L = nb.layer + 30 * o;
  const double* LX = L;
  const double* LY = L + 5 * N;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) bad = 0;
  rbf_coords(LX, LY, n, ld, Pt);
  __syncthreads();
  for (int i = wid; i < n; i += nw) {
    float* row = sA + (size_t)i * (i + 1) / 2;
    for (int j = lane; j <= i; j += 32) row[j] = rbf_phi(Pt, ld, i, j, ie2);
  }
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += RBF_NB) {
    const int w = min(RBF_NB, n - c0), c1 = c0 + w, m = n - c1;
    if (wid == 0) {  // diagonal block: lane c holds column c0 + c (rows c0 + r, r >= c)
      float a[RBF_NB];
#pragma unroll
      for (int r = 0; r < RBF_NB; ++r)
        a[r] = (lane < w && r < w && r >= lane) ? sA[(size_t)(c0 + r) * (c0 + r + 1) / 2 + c0 + lane] : 0.f;
#pragma unroll
      for (int k = 0; k < RBF_NB; ++k) {
        if (k >= w) break;
        const float dkk = __shfl_sync(0xffffffffu, a[k], k);
        if (!(dkk > 0.f) && lane == 0) bad = 1;
        const float d = dkk > 0.f ? sqrtf(dkk) : 1.f;
        if (lane == k) {
          const float inv = 1.f / d;
#pragma unroll
          for (int r = 0; r < RBF_NB; ++r) a[r] = (r == k) ? d : (r > k ? a[r] * inv : a[r]);
        }
        // column j = lane > k: a[r] -= L[r][k] L[j][k] for r >= j (column k sits in lane k; L[j][k] arrives
        // at r == j, before the first r it is needed for)
        float ljk = 0.f;
#pragma unroll
        for (int r = 0; r < RBF_NB; ++r) {
          const float lrk = __shfl_sync(0xffffffffu, a[r], k);
          if (r == lane) ljk = lrk;
          if (lane > k && lane < w && r >= lane) a[r] = fmaf(-lrk, ljk, a[r]);
        }
      }
      if (lane < w)
#pragma unroll
        for (int r = 0; r < RBF_NB; ++r)
          if (r < w && r >= lane) sA[(size_t)(c0 + r) * (c0 + r + 1) / 2 + c0 + lane] = a[r];
    }
    __syncthreads();
    if (m == 0) break;
    // the panel below the diagonal block: row i solves L[i][c0..c1) L_kk^T = A[i][c0..c1)
    for (int q = tid; q < m; q += blockDim.x) {
      const int i = c1 + q;
      float* row = sA + (size_t)i * (i + 1) / 2 + c0;
      float x[RBF_NB];
#pragma unroll
      for (int j = 0; j < RBF_NB; ++j) {
        if (j >= w) break;
        float acc = row[j];
        const float* lj = sA + (size_t)(c0 + j) * (c0 + j + 1) / 2 + c0;  // row c0 + j of the diagonal block
#pragma unroll
        for (int t = 0; t < RBF_NB; ++t)
          if (t < j) acc = fmaf(-x[t], lj[t], acc);
        x[j] = acc / lj[j];
      }
#pragma unroll
      for (int j = 0; j < RBF_NB; ++j)
        if (j < w) {
          row[j] = x[j];
          Pt[j * ld + q] = x[j];
        }
    }
    __syncthreads();
    // trailing triangle: A[i][j] -= sum_t L[i][t] L[j][t] over the panel columns t, tiles of 4 x 4 (tile I >= J)
    const int mb = (m + 3) >> 2;
    const int ntile = mb * (mb + 1) / 2;
    for (int t = tid; t < ntile; t += blockDim.x) {
      int I = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
      while (I * (I + 1) / 2 > t) --I;
      while ((I + 1) * (I + 2) / 2 <= t) ++I;
      const int J = t - I * (I + 1) / 2;
      float acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
      for (int u = 0; u < w; ++u) {  // entries past m in the last tile are stale and only reach discarded sums
        const float4 pi = *reinterpret_cast<const float4*>(&Pt[u * ld + 4 * I]);
        const float4 pj = *reinterpret_cast<const float4*>(&Pt[u * ld + 4 * J]);
        const float vi[4] = {pi.x, pi.y, pi.z, pi.w}, vj[4] = {pj.x, pj.y, pj.z, pj.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(vi[a], vj[b], acc[a][b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int i = c1 + 4 * I + a;
        if (4 * I + a >= m) continue;
        float* row = sA + (size_t)i * (i + 1) / 2;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int j = c1 + 4 * J + b;
          if (4 * J + b < m && j <= i) row[j] -= acc[a][b];
        }
      }
    }
    __syncthreads();
  }
  if (bad && tid == 0) atomicOr(err, ERR_PIVOT);
  // the panel buffer now holds the coordinates (4 ld), the weights (2 ld) and the residuals (2 ld)
  float* crd = Pt;
  float* w1 = Pt + 4 * ld;
  float* w2 = w1 + ld;
  float* r1 = w2 + ld;
  float* r2 = r1 + ld;
  const double* UX = L + 10 * N;
  const double* UY = L + 15 * N;
  rbf_coords(LX, LY, n, ld, crd);
  for (int i = tid; i < n; i += blockDim.x) { w1[i] = (float)UX[i]; w2[i] = (float)UY[i]; }
  __syncthreads();
  rbf_solve2(sA, n, w1, w2);
  // refinement: r = u - (Phi + lam I) w with the same FP32 Phi formed again, its products and sums
  // compensated (the exact product error by fma, Neumaier sums, lanes combined in FP64), w += (L L^T)^{-1} r
  for (int i = wid; i < n; i += nw) {
    float s1 = 0.f, c1 = 0.f, s2 = 0.f, c2 = 0.f;
    for (int j = lane; j < n; j += 32) {
      const float p = rbf_phi(crd, ld, i, j, ie2);
      const float q1 = p * w1[j], q2 = p * w2[j];
      c1 += fmaf(p, w1[j], -q1);
      c2 += fmaf(p, w2[j], -q2);
      neumaier_add(s1, c1, q1);
      neumaier_add(s2, c2, q2);
    }
    double d1 = (double)s1 + (double)c1, d2 = (double)s2 + (double)c2;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      d1 += __shfl_xor_sync(0xffffffffu, d1, off);
      d2 += __shfl_xor_sync(0xffffffffu, d2, off);
    }
    if (lane == 0) {
      r1[i] = (float)(UX[i] - d1);
      r2[i] = (float)(UY[i] - d2);
    }
  }
  __syncthreads();
  rbf_solve2(sA, n, r1, r2);
  double* WX = L + 20 * N;
  double* WY = L + 25 * N;
  for (int i = tid; i < n; i += blockDim.x) {
    WX[i] = (double)w1[i] + (double)r1[i];
    WY[i] = (double)w2[i] + (double)r2[i];
  }
}

// FP32 Cholesky of (Phi + lam I) and the two RBF weight vectors. One CTA per near vesicle.
__global__ void __launch_bounds__(256) k_near_rbf(VesIndex vi, const int* __restrict__ has_near,
                                                  const double* __restrict__ length, NearBufs nb,
                                                  unsigned* err) {
  __shared__ float colk[5 * NMAX];
  __shared__ float y1[5 * NMAX], y2[5 * NMAX];
  __shared__ int bad;
  const int v = vi.vid(blockIdx.x);
  if (!has_near[v]) return;
  const int N = vi.N[v];
  const int n = 5 * N;
  const int64_t o = vi.off[v];
  const double h = length[v] / N;
  const double ie2 = 1.0 / (NEAR_RBF_C * h * NEAR_RBF_C * h);
  double* L = nb.layer + 30 * o;
  const double* LX = L;
  const double* LY = L + 5 * N;
  float* A = nb.phi + vi.moff[v];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) bad = 0;
  for (int i = wid; i < n; i += nw)
    for (int j = lane; j <= i; j += 32) {
      const double dx = LX[i] - LX[j], dy = LY[i] - LY[j];
      double p = exp(-(dx * dx + dy * dy) * ie2);
      if (i == j) p += NEAR_RBF_NUGGET;
      A[(int64_t)i * n + j] = (float)p;
    }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const float dkk = A[(int64_t)k * n + k];
    const float d = dkk > 0.f ? sqrtf(dkk) : 1.f;
    if (tid == 0 && !(dkk > 0.f)) bad = 1;
    const float inv = 1.f / d;
    for (int i = k + 1 + tid; i < n; i += blockDim.x) {
      const float l = A[(int64_t)i * n + k] * inv;
      A[(int64_t)i * n + k] = l;
      colk[i] = l;
    }
    __syncthreads();
    if (tid == 0) A[(int64_t)k * n + k] = d;
    for (int i = k + 1 + wid; i < n; i += nw) {
      const float li = colk[i];
      for (int j = k + 1 + lane; j <= i; j += 32) A[(int64_t)i * n + j] = fmaf(-li, colk[j], A[(int64_t)i * n + j]);
    }
    __syncthreads();
  }
  if (bad && tid == 0) atomicOr(err, ERR_PIVOT);
  // forward L y = u, backward L^T w = y (warp 0, row dot products)
  const double* UX = L + 10 * N;
  const double* UY = L + 15 * N;
  for (int i = tid; i < n; i += blockDim.x) { y1[i] = (float)UX[i]; y2[i] = (float)UY[i]; }
  __syncthreads();
  if (wid == 0) {
    for (int i = 0; i < n; ++i) {
      float s1 = 0.f, s2 = 0.f;
      for (int k = lane; k < i; k += 32) {
        const float a = A[(int64_t)i * n + k];
        s1 = fmaf(a, y1[k], s1);
        s2 = fmaf(a, y2[k], s2);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
      }
      if (lane == 0) {
        const float di = A[(int64_t)i * n + i];
        y1[i] = (y1[i] - s1) / di;
        y2[i] = (y2[i] - s2) / di;
      }
      __syncwarp();
    }
    for (int i = n - 1; i >= 0; --i) {
      float s1 = 0.f, s2 = 0.f;
      for (int k = i + 1 + lane; k < n; k += 32) {
        const float a = A[(int64_t)k * n + i];
        s1 = fmaf(a, y1[k], s1);
        s2 = fmaf(a, y2[k], s2);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
      }
      if (lane == 0) {
        const float di = A[(int64_t)i * n + i];
        y1[i] = (y1[i] - s1) / di;
        y2[i] = (y2[i] - s2) / di;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  double* WX = L + 20 * N;
  double* WY = L + 25 * N;
  for (int i = tid; i < n; i += blockDim.x) { WX[i] = y1[i]; WY[i] = y2[i]; }
}

// u(x_t) += RBF interpolant of each near vesicle's layer velocities.
__global__ void __launch_bounds__(128) k_near_apply(int64_t P, const int32_t* __restrict__ owner,
                                                    const int64_t* __restrict__ voff, const int32_t* __restrict__ Nv,
                                                    const int* __restrict__ near_cnt, const int* __restrict__ near_v,
                                                    const double* __restrict__ xy, const double* __restrict__ length,
                                                    NearBufs nb, double* __restrict__ u) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P) return;
  const int c = near_cnt[t];
  if (c == 0) return;
  const int tv = owner[t];
  const int64_t to = voff[tv];
  const int tN = Nv[tv];
  const double px = xy[2 * to + (t - to)], py = xy[2 * to + tN + (t - to)];
  double ax = 0.0, ay = 0.0;
  for (int k = 0; k < c; ++k) {
    const int v = near_v[t * MAX_NEAR + k];
    const int N = Nv[v];
    const double h = length[v] / N;
    const double ie2 = 1.0 / (NEAR_RBF_C * h * NEAR_RBF_C * h);
    const double* L = nb.layer + 30 * voff[v];
    for (int b = 0; b < 5 * N; ++b) {
      const double dx = px - L[b], dy = py - L[5 * N + b];
      const double p = exp(-(dx * dx + dy * dy) * ie2);
      ax = fma(p, L[20 * N + b], ax);
      ay = fma(p, L[25 * N + b], ay);
    }
  }
  u[2 * to + (t - to)] += ax;
  u[2 * to + tN + (t - to)] += ay;
}

}  // namespace vs
