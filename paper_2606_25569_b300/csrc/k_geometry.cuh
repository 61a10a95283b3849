// Per-vesicle geometry, membrane force and background flow (Sec. 2.2.1, Eq. elastic_force,
// Sec. 5.3-5.5). One CTA of NMAX threads per vesicle, thread j owns point j.
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

__global__ void __launch_bounds__(NMAX) k_geometry(VesIndex vi, const double* __restrict__ xy,
                                                   const double* __restrict__ sigma,
                                                   const double* __restrict__ tab, double kappa,
                                                   double mu, FlowDev flow, GeomOut g,
                                                   ForceOut fo, const double* __restrict__ f_in) {
  // the circulant products run in double-float (FP64 is 1/64 of the FP32 rate on this part), on the
  // positions relative to point 0 (the derivatives do not see the constant)
  __shared__ double xs[NMAX], ys[NMAX], red[NMAX / 32];
  __shared__ float2 dd[NMAX], w1[NMAX], w2[NMAX];
  const int v = vi.vid(blockIdx.x);
  if (g.active && !g.active[v]) return;
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int i = threadIdx.x;
  const bool act = i < N;
  const double* T = tab + vi.toff[v];
  if (act) {
    dd[i] = df_of(T[i]);
    xs[i] = xy[2 * o + i];
    ys[i] = xy[2 * o + N + i];
  }
  __syncthreads();
  float2 px = make_float2(0.f, 0.f), py = px;
  if (act) {
    px = w1[i] = df_of(xs[i] - xs[0]);
    py = w2[i] = df_of(ys[i] - ys[0]);
  }
  __syncthreads();
  double xa = 0.0, ya = 0.0;
  if (act) {
    xa = df_val(circ_df(dd, w1, N, i));
    ya = df_val(circ_df(dd, w2, N, i));
  }
  const double sa = act ? sqrt(xa * xa + ya * ya) : 1.0;
  const double isa = 1.0 / sa;
  const float2 isd = df_of(isa);
  const double tx = xa * isa, ty = ya * isa;
  const double dal = 2.0 * VS_PI / N;
  const double area = block_sum(act ? 0.5 * (xs[i] * ya - ys[i] * xa) * dal : 0.0, red);
  const double length = block_sum(act ? sa * dal : 0.0, red);
  const double cxs = block_sum(act ? xs[i] : 0.0, red);
  const double cys = block_sum(act ? ys[i] : 0.0, red);
  // X_ssss: four applications of D_s = diag(1/sa) D_alpha to each coordinate
  float2 bxd = act ? w1[i] : make_float2(0.f, 0.f), byd = act ? w2[i] : make_float2(0.f, 0.f);
  for (int r = 0; r < 4; ++r) {
    __syncthreads();
    if (act) { w1[i] = bxd; w2[i] = byd; }
    __syncthreads();
    if (act) {
      bxd = df_mul(circ_df(dd, w1, N, i), isd);
      byd = df_mul(circ_df(dd, w2, N, i), isd);
    }
  }
  const double bx = df_val(bxd), by = df_val(byd);
  if (act) {
    g.sa[o + i] = sa;
    g.tx[o + i] = tx;
    g.ty[o + i] = ty;
    g.bx[o + i] = bx;
    g.by[o + i] = by;
    if (g.g32) g.g32[o + i] = make_float4((float)(1.0 / sa), (float)tx, (float)ty, 0.f);
    if (g.sdf) {  // once per point here instead of once per tile in the self matrix (FP64 is slow)
      const float2 c = df_of(sa / (4.0 * VS_PI * mu));
      const float2 lpd = g.logtab ? df_add(df_of(-0.5 * T[N]), df_mul(df_of(-dal), log_df(df_of(sa), g.logtab)))
                                  : df_of(-0.5 * T[N] - dal * log(sa));
      const float2 a = df_of(tx), b = df_of(ty);
      float4* q = g.sdf + 3 * (o + i);
      q[0] = make_float4(px.x, px.y, py.x, py.y);
      q[1] = make_float4(c.x, c.y, lpd.x, lpd.y);
      q[2] = make_float4(a.x, a.y, b.x, b.y);
    }
  }
  if (i == 0) {
    g.area[v] = area;
    g.length[v] = length;
  }
  if (fo.f == nullptr) return;
  // force: f = -kappa X_ssss + D_s(sigma X_s)
  const double sg = (act && sigma) ? sigma[o + i] : 0.0;  // sigma may be null with f_in
  __syncthreads();
  if (act) { w1[i] = df_of(sg * tx); w2[i] = df_of(sg * ty); }
  __syncthreads();
  double fx = 0.0, fy = 0.0;
  if (act) {
    if (f_in) {  // caller-supplied density (far-field evaluation of a given force)
      fx = f_in[2 * o + i];
      fy = f_in[2 * o + N + i];
    } else {
      fx = -kappa * bx + df_val(df_mul(circ_df(dd, w1, N, i), isd));
      fy = -kappa * by + df_val(df_mul(circ_df(dd, w2, N, i), isd));
    }
  }
  const double cx = cxs / N, cy = cys / N;
  const double rho2 = block_max(act ? (xs[i] - cx) * (xs[i] - cx) + (ys[i] - cy) * (ys[i] - cy) : 0.0, red);
  const double c = sa * dal / (4.0 * VS_PI * mu);
  const double gsx = block_sum(act ? fx * c : 0.0, red);
  const double gsy = block_sum(act ? fy * c : 0.0, red);
  if (act) {
    fo.f[2 * o + i] = fx;
    fo.f[2 * o + N + i] = fy;
    const double2 ub = background_flow(flow, xs[i], ys[i]);
    fo.u[2 * o + i] = ub.x;
    fo.u[2 * o + N + i] = ub.y;
    fo.g64[2 * o + i] = fx * c;
    fo.g64[2 * o + N + i] = fy * c;
    fo.src[o + i] = make_float4((float)(xs[i] - cx), (float)(ys[i] - cy), (float)(fx * c), (float)(fy * c));
  }
  if (i == 0) {
    fo.centre[v] = make_double2(cx, cy);
    const float hx = (float)cx, hy = (float)cy;
    fo.centre32[v] = make_float4(hx, hy, (float)(cx - (double)hx), (float)(cy - (double)hy));
    const double h = length / N;
    const double reach = (sqrt(rho2) + h) * (1.0 + 1e-3);
    fo.h2[v] = make_float2((float)(h * h), (float)(reach * reach));
    fo.gsum[v] = make_float2((float)gsx, (float)gsy);
  }
}

}  // namespace vs
