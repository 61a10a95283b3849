// Per-vesicle geometry, membrane force and background flow (Sec. 2.2.1, Eq. elastic_force,
// Sec. 5.3-5.5). One CTA of NMAX threads per vesicle, one or two threads per point.
#pragma once
#include "common.cuh"
#include "dfloat.cuh"

namespace vs {

struct FlowDev {
  int kind;        // 0 none, 1 shear, 2 Taylor-Green, 3 Poiseuille
  double p0, p1;
};

__device__ __forceinline__ double2 background_flow(const FlowDev& f, double x, double y) {
  switch (f.kind) {
    case 1: return make_double2(f.p0 * y, 0.0);
    case 2: {
      const double a = VS_PI * x / f.p1, b = VS_PI * y / f.p1;
      return make_double2(f.p0 * sin(a) * cos(b), -f.p0 * cos(a) * sin(b));
    }
    case 3: {
      const double r = y / f.p1;
      return make_double2(f.p0 * (1.0 - r * r), 0.0);
    }
    default: return make_double2(0.0, 0.0);
  }
}

// Geometry outputs at the N points of every vesicle.
struct GeomOut {
  double* sa;   // |X_alpha|
  double* tx;   // X_s
  double* ty;
  double* bx;   // X_ssss
  double* by;
  double* area;    // [M]
  double* length;  // [M]
  float4* g32;     // FP32 (1/|X_alpha|, x_s, y_s, 0) for the FP32 operator products (may be null)
  float4* sdf;     // 3 per point, double-float pairs for the self matrix (may be null):
                   //   (x - x_0, y - y_0), (|X_alpha| / (4 pi mu), -R(0)/2 - (2 pi/N) log|X_alpha|), (x_s, y_s)
  const int* active;  // null, or only vesicles with active[v] != 0 are processed
  const float4* logtab;  // the double-float logarithm's table (log_df) for the self-matrix diagonal, or null
                         // (then an FP64 logarithm)
};

// Force/source outputs (only written when `f` is non-null). With f_in non-null the density is
// taken from f_in instead of the membrane force.
struct ForceOut {
  double* f;           // f = -kappa X_ssss + (sigma X_s)_s, CSR blocks [f_x(N), f_y(N)] per vesicle
  double* u;           // velocity accumulator (CSR blocks): initialised to u_inf(X)
  float4* src;         // (x - c_v, y - c_v, g_x, g_y), g = f |X_alpha| (2 pi/N) / (4 pi mu)
  double2* centre;     // c_v (mean of the points) [M]
  float4* centre32;    // (hi_x, hi_y, lo_x, lo_y) float split of c_v [M]
  float2* h2;          // ((L_v/N_v)^2, reach^2) [M]: reach = (max_j |X_vj - c_v| + L_v/N_v)(1 + 1e-3), a
                       // bound beyond which no point of v is within L_v/N_v
  double* g64;         // FP64 copy of g, CSR blocks (for the FP64 far-field variant)
  float2* gsum;        // sum_j g_j of each vesicle, summed in FP64 [M] (the FP32 far field adds the common
                       // part of its logarithms once per vesicle pair with it)
};

// Part of the circulant product out_i = sum_j d[(i - j) mod N] v_j over the terms j in [jb, je), in
// double-float like circ_df (compensated chunks of DF_CHUNK folded into a double-float total).
__device__ __forceinline__ float2 circ_df_part(const float2* d, const float2* v, int N, int i, int jb, int je) {
  float2 tot = make_float2(0.f, 0.f);
  int m = i - jb;
  if (m < 0) m += N;
  for (int j0 = jb; j0 < je; j0 += DF_CHUNK) {
    Dot2 a;
    const int j1 = min(j0 + DF_CHUNK, je);
    for (int j = j0; j < j1; ++j) {
      a.add(d[m], v[j]);
      m = (m == 0) ? N - 1 : m - 1;
    }
    tot = df_add(tot, a.value());
  }
  return tot;
}

// The circulant products of two vectors at point i, by the P halves of the CTA (half h = thread / (NMAX / P)):
// P = 1 is circ_df; with P = 2 each half sums half of the terms, the second half hands its parts over through
// shared memory (px, py) and the first half gets (first half's terms) + (second half's terms). Called by every
// thread; ends with a barrier after the last read of v1 and v2; the results are valid in half 0 where act.
template <int P>
__device__ __forceinline__ void circ_pts2(const float2* d, const float2* v1, const float2* v2, int N, int i, int h,
                                          bool act, float2* px, float2* py, float2& o1, float2& o2) {
  o1 = o2 = make_float2(0.f, 0.f);
  if constexpr (P == 1) {
    if (act) {
      o1 = circ_df(d, v1, N, i);
      o2 = circ_df(d, v2, N, i);
    }
    __syncthreads();  // as with P = 2: every read of v1, v2 ends here
  } else {
    const int half = N / 2, jb = h * half, je = h ? N : half;
    float2 a = make_float2(0.f, 0.f), b = a;
    if (act) {
      a = circ_df_part(d, v1, N, i, jb, je);
      b = circ_df_part(d, v2, N, i, jb, je);
      if (h) { px[i] = a; py[i] = b; }
    }
    __syncthreads();
    if (act && !h) {
      o1 = df_add(a, px[i]);
      o2 = df_add(b, py[i]);
    }
  }
}

// Block-wide sums of four doubles over the first nw warps of the CTA (the others hold no values and skip the
// shuffles; each sum in the same order as block_sum); red holds 4 doubles per warp. All threads get them.
__device__ inline double4 block_sum4(double4 v, double* red, int nw) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid < nw) {
    v.x = warp_sum(v.x);
    v.y = warp_sum(v.y);
    v.z = warp_sum(v.z);
    v.w = warp_sum(v.w);
  }
  __syncthreads();
  if (lane == 0 && wid < nw) {
    red[4 * wid] = v.x; red[4 * wid + 1] = v.y; red[4 * wid + 2] = v.z; red[4 * wid + 3] = v.w;
  }
  __syncthreads();
  double4 t = make_double4(0.0, 0.0, 0.0, 0.0);
  for (int w = 0; w < nw; ++w) {
    t.x += red[4 * w]; t.y += red[4 * w + 1]; t.z += red[4 * w + 2]; t.w += red[4 * w + 3];
  }
  return t;
}

// One CTA of NMAX threads per vesicle. With P = 2 (every vesicle of at most NMAX / 2 points) both halves of the
// CTA take point i = thread mod (NMAX / 2) and each sums half of every circulant product, while the per-point
// FP64 work (on a pipe at 1/64 of the FP32 rate) stays with the first half, so that it costs no more warp
// instructions than with one thread a point; P = 1 gives thread i point i.
template <int P>
__global__ void __launch_bounds__(NMAX) k_geometry(VesIndex vi, const double* __restrict__ xy,
                                                   const double* __restrict__ sigma,
                                                   const double* __restrict__ tab, double kappa,
                                                   double mu, FlowDev flow, GeomOut g,
                                                   ForceOut fo, const double* __restrict__ f_in) {
  // the circulant products run in double-float (FP64 is 1/64 of the FP32 rate on this part), on the
  // positions relative to point 0 (the derivatives do not see the constant)
  constexpr int HALF = NMAX / P, NW = HALF / 32;
  __shared__ double xs[NMAX], ys[NMAX], red[4 * (NMAX / 32)];
  __shared__ float2 dd[NMAX], w1[NMAX], w2[NMAX], p1[NMAX], p2[NMAX];
  __shared__ double cst[3];  // 2 pi / N, 1 / N, 1 / (4 pi mu): one FP64 division each per vesicle
  const int v = vi.vid(blockIdx.x);
  if (g.active && !g.active[v]) return;
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int i = threadIdx.x % HALF, h = threadIdx.x / HALF;
  const bool act = i < N, own = act && h == 0;  // own: the thread that does point i's FP64 work and writes it
  const double* T = tab + vi.toff[v];
  if (threadIdx.x == 0) {
    cst[0] = 2.0 * VS_PI / N;
    cst[1] = 1.0 / N;
    cst[2] = 1.0 / (4.0 * VS_PI * mu);
  }
  float2 px = make_float2(0.f, 0.f), py = px;
  if (own) {
    dd[i] = df_of(T[i]);
    xs[i] = xy[2 * o + i];
    ys[i] = xy[2 * o + N + i];
  }
  __syncthreads();
  if (own) {
    px = w1[i] = df_of(xs[i] - xs[0]);
    py = w2[i] = df_of(ys[i] - ys[0]);
  }
  __syncthreads();
  float2 xad, yad;
  circ_pts2<P>(dd, w1, w2, N, i, h, act, p1, p2, xad, yad);
  // speed, its reciprocal and the unit tangent in double-float (no FP64 square root or division per point)
  double xa = 0.0, ya = 0.0, sa = 1.0, tx = 0.0, ty = 0.0;
  float2 sad = make_float2(1.f, 0.f), isd = sad, txd = make_float2(0.f, 0.f), tyd = txd;
  const double dal = cst[0], i4pm = cst[2];
  double4 mine = make_double4(0.0, 0.0, 0.0, 0.0);
  if (own) {
    sad = df_sqrt(df_add(df_mul(xad, xad), df_mul(yad, yad)));
    isd = df_rcp(sad);
    txd = df_mul(xad, isd);
    tyd = df_mul(yad, isd);
    xa = df_val(xad); ya = df_val(yad); sa = df_val(sad); tx = df_val(txd); ty = df_val(tyd);
    mine = make_double4(0.5 * (xs[i] * ya - ys[i] * xa) * dal, sa * dal, xs[i], ys[i]);
  }
  const double4 sums = block_sum4(mine, red, NW);
  const double area = sums.x, length = sums.y, cxs = sums.z, cys = sums.w;
  // X_ssss: four applications of D_s = diag(1/sa) D_alpha to each coordinate (w1, w2 hold px, py)
  float2 bxd = px, byd = py;
  for (int r = 0; r < 4; ++r) {
    __syncthreads();
    float2 cx2, cy2;
    circ_pts2<P>(dd, w1, w2, N, i, h, act, p1, p2, cx2, cy2);
    if (own) {  // every read of w1, w2 in this pass ended at the barrier inside circ_pts2
      bxd = df_mul(cx2, isd);
      byd = df_mul(cy2, isd);
      w1[i] = bxd;
      w2[i] = byd;
    }
  }
  const double bx = df_val(bxd), by = df_val(byd);
  if (own) {
    g.sa[o + i] = sa;
    g.tx[o + i] = tx;
    g.ty[o + i] = ty;
    g.bx[o + i] = bx;
    g.by[o + i] = by;
    if (g.g32) g.g32[o + i] = make_float4(isd.x, txd.x, tyd.x, 0.f);
    if (g.sdf) {  // once per point here instead of once per tile in the self matrix (FP64 is slow)
      const float2 c = df_mul(sad, df_of(i4pm));
      const float2 lpd = g.logtab ? df_add(df_of(-0.5 * T[N]), df_mul(df_of(-dal), log_df(sad, g.logtab)))
                                  : df_of(-0.5 * T[N] - dal * log(sa));
      float4* q = g.sdf + 3 * (o + i);
      q[0] = make_float4(px.x, px.y, py.x, py.y);
      q[1] = make_float4(c.x, c.y, lpd.x, lpd.y);
      q[2] = make_float4(txd.x, txd.y, tyd.x, tyd.y);
    }
  }
  if (threadIdx.x == 0) {
    g.area[v] = area;
    g.length[v] = length;
  }
  if (fo.f == nullptr) return;
  // force: f = -kappa X_ssss + D_s(sigma X_s)
  __syncthreads();  // the last pass's reads of w1, w2 ended; X_ssss no longer needed there
  if (own) {
    const double sg = sigma ? sigma[o + i] : 0.0;  // sigma may be null with f_in
    w1[i] = df_of(sg * tx);
    w2[i] = df_of(sg * ty);
  }
  __syncthreads();
  double fx = 0.0, fy = 0.0;
  if (f_in) {  // caller-supplied density (far-field evaluation of a given force)
    if (own) {
      fx = f_in[2 * o + i];
      fy = f_in[2 * o + N + i];
    }
  } else {
    float2 tsx, tsy;
    circ_pts2<P>(dd, w1, w2, N, i, h, act, p1, p2, tsx, tsy);
    if (own) {
      fx = -kappa * bx + df_val(df_mul(tsx, isd));
      fy = -kappa * by + df_val(df_mul(tsy, isd));
    }
  }
  const double cx = cxs * cst[1], cy = cys * cst[1];
  const double c = sa * dal * i4pm;
  double4 m2 = make_double4(0.0, 0.0, 0.0, 0.0);
  if (own) m2 = make_double4(fx * c, fy * c, 0.0, 0.0);
  const double4 gs = block_sum4(m2, red, NW);
  // reach of the vesicle (max distance of a point from c_v) by warp maxima over the first half
  double r2 = own ? (xs[i] - cx) * (xs[i] - cx) + (ys[i] - cy) * (ys[i] - cy) : 0.0;
  if ((int)(threadIdx.x >> 5) < NW)
    for (int off = 16; off > 0; off >>= 1) r2 = fmax(r2, __shfl_xor_sync(0xffffffffu, r2, off));
  __syncthreads();
  if ((threadIdx.x & 31) == 0 && (int)(threadIdx.x >> 5) < NW) red[threadIdx.x >> 5] = r2;
  __syncthreads();
  double rho2 = red[0];
  for (int w = 1; w < NW; ++w) rho2 = fmax(rho2, red[w]);
  if (own) {
    fo.f[2 * o + i] = fx;
    fo.f[2 * o + N + i] = fy;
    const double2 ub = background_flow(flow, xs[i], ys[i]);
    fo.u[2 * o + i] = ub.x;
    fo.u[2 * o + N + i] = ub.y;
    fo.g64[2 * o + i] = fx * c;
    fo.g64[2 * o + N + i] = fy * c;
    fo.src[o + i] = make_float4((float)(xs[i] - cx), (float)(ys[i] - cy), (float)(fx * c), (float)(fy * c));
  }
  if (threadIdx.x == 0) {
    fo.centre[v] = make_double2(cx, cy);
    const float hx = (float)cx, hy = (float)cy;
    fo.centre32[v] = make_float4(hx, hy, (float)(cx - (double)hx), (float)(cy - (double)hy));
    const double hs = length / N;
    const double reach = (sqrt(rho2) + hs) * (1.0 + 1e-3);
    fo.h2[v] = make_float2((float)(hs * hs), (float)(reach * reach));
    fo.gsum[v] = make_float2((float)gs.x, (float)gs.y);
  }
}

// Launch of k_geometry over M vesicles of at most nmax points (two threads a point when they fit).
inline void launch_geometry(int M, int nmax, cudaStream_t st, const VesIndex& vi, const double* xy, const double* sigma,
                            const double* tab, double kappa, double mu, FlowDev flow, const GeomOut& g,
                            const ForceOut& fo, const double* f_in) {
  if (2 * nmax <= NMAX)
    k_geometry<2><<<M, NMAX, 0, st>>>(vi, xy, sigma, tab, kappa, mu, flow, g, fo, f_in);
  else
    k_geometry<1><<<M, NMAX, 0, st>>>(vi, xy, sigma, tab, kappa, mu, flow, g, fo, f_in);
}

}  // namespace vs
