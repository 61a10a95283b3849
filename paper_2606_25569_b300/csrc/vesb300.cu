// C ABI and host orchestration of the vesicle-suspension step (Algorithm 1 with exact operators).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/vesb300.h"
#include "common.cuh"
#include "k_dense.cuh"
#include "k_farfield.cuh"
#include "k_farfield_sym.cuh"
#include "k_farfield_loc.cuh"
#include "k_fftree.cuh"
#include "k_fused.cuh"
#include "k_geometry.cuh"
#include "k_implicit.cuh"
#include "k_ivnet.cuh"
#include "k_mlp.cuh"
#include "k_mp.cuh"
#include "k_near.cuh"
#include "k_probe.cuh"
#include "k_selfmat.cuh"
#include "k_standardize.cuh"
#include "k_flow.cuh"
#include "k_tcgemm.cuh"
#include "k_vesicle.cuh"
#include "tables.cuh"

using namespace vs;

// Hybrid steps relax exactly every vesicle within this many point spacings h = L/N (the larger of the two
// vesicles') of another vesicle.
constexpr double HYBRID_EXACT_GAP = 4.0;  // default of vs_params.exact_gap
constexpr int CORR_NEWTON_ITERS = 16;  // Newton steps on the KKT system (linear convergence with the FP32 Jacobian)

namespace {

// ---------------------------------------------------------------------------------------------
// layout shared by suspensions and far-field plans
struct Layout {
  int M = 0;
  int64_t P = 0;
  int nmax = 0;
  std::vector<int32_t> N;
  std::vector<int64_t> off, moff, toff;
  std::vector<int32_t> owner, chunk, chunk1k;  // far-field source chunks of at most 2048 / 1024 points
  std::vector<double> tab;
  std::vector<int32_t> order;  // vesicles by point count, descending (empty when all counts are equal)
};

// Greedy chunks of whole vesicles with at most `limit` points each: boundaries in vesicles.
std::vector<int32_t> source_chunks(const std::vector<int32_t>& N, int limit) {
  std::vector<int32_t> c{0};
  int64_t acc = 0;
  for (int v = 0; v < (int)N.size(); ++v) {
    if (acc + N[v] > limit) { c.push_back(v); acc = 0; }
    acc += N[v];
  }
  c.push_back((int32_t)N.size());
  return c;
}

bool build_layout(const int64_t* offsets, int M, Layout& L, std::string& msg) {
  if (M < 1 || offsets == nullptr) { msg = "M must be >= 1 and offsets non-null"; return false; }
  if (offsets[0] != 0) { msg = "offsets[0] must be 0"; return false; }
  L.M = M;
  L.N.resize(M);
  L.off.resize(M + 1);
  L.moff.resize(M + 1);
  L.toff.resize(M);
  std::map<int, int64_t> tpos;
  int64_t moff = 0;
  for (int v = 0; v < M; ++v) {
    const int64_t n = offsets[v + 1] - offsets[v];
    if (n < 8 || n > NMAX || (n & 1)) {
      char b[160];
      snprintf(b, sizeof b, "vesicle %d has %lld points; need an even count in [8, %d]", v, (long long)n, NMAX);
      msg = b;
      return false;
    }
    L.N[v] = (int32_t)n;
    L.off[v] = offsets[v];
    L.moff[v] = moff;
    moff += MatLayout::TOTAL * n * n;
    if (!tpos.count((int)n)) {
      tpos[(int)n] = (int64_t)L.tab.size();
      L.tab.resize(L.tab.size() + TAB_STRIDE * n);
      build_tables((int)n, L.tab.data() + tpos[(int)n]);
    }
    L.toff[v] = tpos[(int)n];
    L.nmax = std::max(L.nmax, (int)n);
  }
  L.off[M] = offsets[M];
  L.moff[M] = moff;
  L.P = offsets[M];
  L.owner.resize(L.P);
  for (int v = 0; v < M; ++v)
    for (int64_t p = L.off[v]; p < L.off[v + 1]; ++p) L.owner[p] = v;
  L.chunk = source_chunks(L.N, FF_CHUNK);
  L.chunk1k = source_chunks(L.N, 1024);
  // per-vesicle launches take the largest vesicles first (longest work first shortens the tail)
  L.order.clear();
  if (*std::min_element(L.N.begin(), L.N.end()) != L.nmax) {
    L.order.resize(M);
    for (int v = 0; v < M; ++v) L.order[v] = v;
    std::stable_sort(L.order.begin(), L.order.end(), [&](int a, int b) { return L.N[a] > L.N[b]; });
  }
  return true;
}

template <class T>
cudaError_t dalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  return cudaMalloc((void**)p, n * sizeof(T));
}

template <class T>
cudaError_t upload(T* d, const T* h, size_t n, cudaStream_t s) {
  return cudaMemcpyAsync(d, h, n * sizeof(T), cudaMemcpyHostToDevice, s);
}

struct DevLayout {
  int32_t* N = nullptr;
  int64_t* off = nullptr;
  int64_t* moff = nullptr;
  int64_t* toff = nullptr;
  int32_t* owner = nullptr;
  int32_t* chunk = nullptr;
  int32_t* chunk1k = nullptr;
  double* tab = nullptr;
  float* tab32 = nullptr;  // FP32 copy of tab (FP32 operator products)
  float4* logtab = nullptr;  // (log c_k, 1/c_k) as FP32 pairs, c_k = 1 + (k + 1/2)/LOG_TAB (log_df)
  float2* tabdf = nullptr;   // double-float copy of tab (hi, lo)
  int32_t* order = nullptr;
  VesIndex vi() const { return VesIndex{N, off, moff, toff, order}; }
  void release() {
    cudaFree(N); cudaFree(off); cudaFree(moff); cudaFree(toff);
    cudaFree(owner); cudaFree(chunk); cudaFree(chunk1k); cudaFree(tab); cudaFree(tab32); cudaFree(logtab);
    cudaFree(tabdf); cudaFree(order);
    *this = DevLayout{};
  }
};

cudaError_t upload_layout(const Layout& L, DevLayout& D, cudaStream_t s) {
  cudaError_t e;
#define VS_TRY(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
  VS_TRY(dalloc(&D.N, L.M));
  VS_TRY(dalloc(&D.off, L.M + 1));
  VS_TRY(dalloc(&D.moff, L.M + 1));
  VS_TRY(dalloc(&D.toff, L.M));
  if (!L.order.empty()) {
    VS_TRY(dalloc(&D.order, L.M));
    VS_TRY(upload(D.order, L.order.data(), L.M, s));
  }
  VS_TRY(dalloc(&D.owner, L.P));
  VS_TRY(dalloc(&D.chunk, L.chunk.size()));
  VS_TRY(dalloc(&D.chunk1k, L.chunk1k.size()));
  VS_TRY(upload(D.chunk1k, L.chunk1k.data(), L.chunk1k.size(), s));
  VS_TRY(dalloc(&D.tab, L.tab.size()));
  VS_TRY(upload(D.N, L.N.data(), L.M, s));
  VS_TRY(upload(D.off, L.off.data(), L.M + 1, s));
  VS_TRY(upload(D.moff, L.moff.data(), L.M + 1, s));
  VS_TRY(upload(D.toff, L.toff.data(), L.M, s));
  VS_TRY(upload(D.owner, L.owner.data(), L.P, s));
  VS_TRY(upload(D.chunk, L.chunk.data(), L.chunk.size(), s));
  VS_TRY(upload(D.tab, L.tab.data(), L.tab.size(), s));
  std::vector<float> t32(L.tab.begin(), L.tab.end());
  VS_TRY(dalloc(&D.tab32, t32.size()));
  VS_TRY(upload(D.tab32, t32.data(), t32.size(), s));
  std::vector<float2> tdf(L.tab.size());
  for (size_t k = 0; k < L.tab.size(); ++k) {
    const float hi = (float)L.tab[k];
    tdf[k] = make_float2(hi, (float)(L.tab[k] - (double)hi));
  }
  VS_TRY(dalloc(&D.tabdf, tdf.size()));
  VS_TRY(upload(D.tabdf, tdf.data(), tdf.size(), s));
  std::vector<float4> lt(LOG_TAB);
  for (int k = 0; k < LOG_TAB; ++k) {
    const long double c = 1.0L + (k + 0.5L) / LOG_TAB, lc = std::log(c), rc = 1.0L / c;
    const float lh = (float)lc, rh = (float)rc;
    lt[k] = make_float4(lh, (float)(lc - lh), rh, (float)(rc - rh));
  }
  VS_TRY(dalloc(&D.logtab, LOG_TAB));
  VS_TRY(upload(D.logtab, lt.data(), LOG_TAB, s));
#undef VS_TRY
  return cudaStreamSynchronize(s);
}

// Per-point and per-vesicle work buffers used by the force / far-field stage.
struct SourceBufs {
  double* f = nullptr;
  double* g64 = nullptr;
  float4* src = nullptr;
  double2* centre = nullptr;
  float4* centre32 = nullptr;
  float2* h2 = nullptr;
  float2* gsum = nullptr;
  int* near_cnt = nullptr;
  int* near_v = nullptr;
  double *sa = nullptr, *tx = nullptr, *ty = nullptr, *bx = nullptr, *by = nullptr;
  double *area = nullptr, *length = nullptr;
  float4* g32 = nullptr;
  float4* sdf = nullptr;
  float4* mpcoef = nullptr;  // multipole far field: per vesicle (FF_MP_P + 1) x 2 float4 coefficients
  float2* mpa0 = nullptr;    // and its total density A_0
  float* mploc = nullptr;    // per target vesicle: local expansion of the separated sources
  int* mpncnt = nullptr;     // and its list of the other source vesicles
  int* mplist = nullptr;
  // cluster tree of the multipole far field (k_fftree.cuh), allocated when it is used
  double2 *vraw = nullptr, *t_cen = nullptr, *t_raw = nullptr;
  int *t_order = nullptr, *t_owner = nullptr, *t_lstart = nullptr, *t_parent = nullptr, *t_first = nullptr;
  int *t_nchild = nullptr;
  int2* t_range = nullptr;
  float4 *t_cen32 = nullptr, *t_coef = nullptr;
  float* t_rad = nullptr;
  float2* t_a0 = nullptr;
  int64_t t_max = 0;
  cudaError_t alloc_tree(int M) {
    cudaError_t e;
#define VS_TRY(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
    t_max = tree_max_boxes(M);
    VS_TRY(dalloc(&vraw, (size_t)M * 3 * TREE_K)); VS_TRY(dalloc(&t_order, M)); VS_TRY(dalloc(&t_owner, M));
    VS_TRY(dalloc(&t_lstart, TREE_LMAX + 2)); VS_TRY(dalloc(&t_range, t_max)); VS_TRY(dalloc(&t_parent, t_max));
    VS_TRY(dalloc(&t_first, t_max)); VS_TRY(dalloc(&t_nchild, t_max)); VS_TRY(dalloc(&t_cen, t_max));
    VS_TRY(dalloc(&t_cen32, t_max)); VS_TRY(dalloc(&t_rad, t_max)); VS_TRY(dalloc(&t_raw, t_max * 3 * TREE_K));
    VS_TRY(dalloc(&t_coef, t_max * 2 * (FF_MP_P + 1))); VS_TRY(dalloc(&t_a0, t_max));
#undef VS_TRY
    return cudaSuccess;
  }
  FfTreeArgs tree(int M) const {
    return FfTreeArgs{M, t_max, centre, centre32, h2, vraw, t_order, t_owner, t_lstart, t_range, t_parent, t_first,
                      t_nchild, t_cen, t_cen32, t_rad, t_raw, t_coef, t_a0};
  }
  cudaError_t alloc(int64_t P, int M) {
    cudaError_t e;
#define VS_TRY(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
    VS_TRY(dalloc(&f, 2 * P)); VS_TRY(dalloc(&g64, 2 * P)); VS_TRY(dalloc(&src, P));
    VS_TRY(dalloc(&centre, M)); VS_TRY(dalloc(&centre32, M)); VS_TRY(dalloc(&h2, M));
    VS_TRY(dalloc(&gsum, M));
    VS_TRY(dalloc(&near_cnt, P)); VS_TRY(dalloc(&near_v, P * MAX_NEAR));
    VS_TRY(dalloc(&sa, P)); VS_TRY(dalloc(&tx, P)); VS_TRY(dalloc(&ty, P));
    VS_TRY(dalloc(&bx, P)); VS_TRY(dalloc(&by, P));
    VS_TRY(dalloc(&area, M)); VS_TRY(dalloc(&length, M)); VS_TRY(dalloc(&g32, P));
    VS_TRY(dalloc(&sdf, 3 * P));
    VS_TRY(dalloc(&mpcoef, (int64_t)M * (FF_MP_P + 1) * 2)); VS_TRY(dalloc(&mpa0, M));
    VS_TRY(dalloc(&mploc, (int64_t)M * ffl_floats(FF_MP_P))); VS_TRY(dalloc(&mpncnt, M));
    VS_TRY(dalloc(&mplist, (int64_t)M * FFL_LIST));
#undef VS_TRY
    return cudaSuccess;
  }
  void release() {
    cudaFree(f); cudaFree(g64); cudaFree(src); cudaFree(centre); cudaFree(centre32); cudaFree(h2);
    cudaFree(gsum);
    cudaFree(near_cnt); cudaFree(near_v); cudaFree(sa); cudaFree(tx); cudaFree(ty); cudaFree(bx);
    cudaFree(by); cudaFree(area); cudaFree(length); cudaFree(g32); cudaFree(sdf);
    cudaFree(mpcoef); cudaFree(mpa0); cudaFree(mploc); cudaFree(mpncnt); cudaFree(mplist);
    cudaFree(vraw); cudaFree(t_order); cudaFree(t_owner); cudaFree(t_lstart); cudaFree(t_range); cudaFree(t_parent);
    cudaFree(t_first); cudaFree(t_nchild); cudaFree(t_cen); cudaFree(t_cen32); cudaFree(t_rad); cudaFree(t_raw);
    cudaFree(t_coef); cudaFree(t_a0);
    *this = SourceBufs{};
  }
  GeomOut geom() const { return GeomOut{sa, tx, ty, bx, by, area, length, g32, sdf}; }
  FfLocArgs loc(int M) const { return FfLocArgs{M, centre32, h2, mpcoef, mpa0, mploc, mpncnt, mplist}; }
  PointGeom pg() const { return PointGeom{sa, tx, ty}; }
};

}  // namespace

// ---------------------------------------------------------------------------------------------
// Optional per-kernel CUDA-event timing on the handle's stream.
struct Prof {
  bool on = false;
  std::vector<std::string> names;
  std::vector<double> total_ms;
  std::vector<int64_t> count;
  std::vector<cudaEvent_t> pool;
  std::vector<int> rec_id;  // name id per recorded pair (events 2k, 2k+1 of the pool)
  int id(const char* n) {
    for (size_t i = 0; i < names.size(); ++i)
      if (names[i] == n) return (int)i;
    names.push_back(n);
    total_ms.push_back(0.0);
    count.push_back(0);
    return (int)names.size() - 1;
  }
};

struct vs_mlp {
  std::vector<int> dims;            // d_0 .. d_L
  int L = 0, Bcap = 0, ncomp = 1;
  float beta = 1.f;
  int64_t nparam = 0;
  std::vector<int64_t> woff, boff;  // offsets of W_l, b_l in the flat parameter vector
  cudaStream_t stream = nullptr;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  std::vector<__nv_bfloat16*> Wb, WbT, H, HT;
  float* yhat = nullptr;
  float *g32[2] = {nullptr, nullptr};
  __nv_bfloat16 *gbf[2] = {nullptr, nullptr}, *gbfT[2] = {nullptr, nullptr};
  float *loss_b = nullptr, *loss = nullptr;
  // per-feature affine maps: [in_shift d_0 | in_scale d_0 | out_shift d_L | out_scale d_L | 1/out_scale d_L]
  float* aff = nullptr;
  bool has_in = false, has_out = false;
  float* ynorm = nullptr;             // targets in output coordinates (Bcap x d_L)
  double* stats = nullptr;            // column means and deviations (2 max(d_0, d_L))
  unsigned* err = nullptr;
  int64_t t = 0;
  int64_t launches = 0;
  std::string msg;
};

// Symmetric FP32 far field (k_farfield_sym): tile list, tile counter and per-chunk partial sums; R = points
// per lane (N / 32), 0 when the suspension or plan uses another far-field kernel.
// Symmetric FP32 far field (k_farfield_sym): the symmetric order, chunks, and the tiles of each pair of
// classes (rows of rr[k] segments, columns of rc[k]).
constexpr int FFS_NPAIR = 6;
struct FfSymState {
  bool on = false;
  int V = FFS_V;        // vesicles per chunk
  int per_sm = 0;       // persistent CTAs per SM (0: as many as fit)
  bool padded = false;  // some N is not a multiple of 32 or the order is not the identity: k_ffs_pad runs
  int nchunk = 0;
  int slots = 0;        // partial-sum slots per point: nchunk, or the group size S of the phased evaluation
  bool phased = false;
  // one persistent launch per pair of classes with tiles, per phase (one phase when not phased)
  struct Launch { int rr, rc, ntile, grid; int64_t tile_off; };
  struct Phase { int first, count, ga, gb, na, nb; };
  std::vector<Launch> launch;
  std::vector<Phase> phase;
  int2* tiles = nullptr;
  unsigned* ctr = nullptr;  // [launch.size()]
  int* pchunk = nullptr;    // chunk of each point (phased only)
  float4* part = nullptr;
  float4* psrc = nullptr;   // padded sources (padded only)
  int* vid = nullptr;
  int64_t *poff = nullptr, *roff = nullptr;
  int* nreal = nullptr;
  int2* chunk = nullptr;
  void release() {
    cudaFree(tiles); cudaFree(ctr); cudaFree(part); cudaFree(psrc); cudaFree(vid); cudaFree(poff); cudaFree(roff);
    cudaFree(nreal); cudaFree(chunk); cudaFree(pchunk);
    *this = FfSymState{};
  }
};

// Restarted GMRES of the fully implicit step (mode 2): settings, device work vectors and statistics.
struct GmresState {
  double tol = 1e-10;        // relative residual ||b - A z|| / ||b|| to reach
  int restart = 30;          // Krylov vectors per cycle
  int max_iter = 300;        // iterations (matrix-vector products in cycles) per step
  int64_t n = 0;             // 3 P
  int G = 0;                 // CTAs of the vector kernels
  int alloc_restart = 0;
  double *V = nullptr;       // (restart + 1) x n Krylov basis
  double *Z = nullptr;       // restart x n preconditioned basis vectors (flexible GMRES)
  int64_t ainv = 0;          // FP32 inverse of the relaxation matrix in the FP32 scratch (mixed precision)
  double *w = nullptr, *z = nullptr, *b = nullptr, *t1 = nullptr;
  double *part = nullptr;    // (restart + 1) x G partial dot products
  double *hd = nullptr;      // Hessenberg column (restart + 2), then the first pass's coefficients
  double *hd2 = nullptr;     // second Gram-Schmidt pass's coefficients / the update coefficients y
  double *hh = nullptr;      // pinned host copy of a Hessenberg column (restart + 2)
  int last_iters = 0;
  double last_res = 0.0;
  int64_t total_iters = 0;
  void release() {
    cudaFree(V); cudaFree(Z); cudaFree(w); cudaFree(z); cudaFree(b); cudaFree(t1); cudaFree(part);
    cudaFree(hd); cudaFree(hd2);
    if (hh) cudaFreeHost(hh);
    V = Z = w = z = b = t1 = part = hd = hd2 = hh = nullptr;
    alloc_restart = 0;
  }
};

struct vs_suspension {
  Layout L;
  DevLayout D;
  SourceBufs B;
  vs_params p{};
  vs_flow flow{};
  cudaStream_t stream = nullptr;
  double *xy = nullptr, *xy_star = nullptr, *xy_next = nullptr, *sigma = nullptr;
  double *u = nullptr, *u_r = nullptr, *A0 = nullptr, *L0 = nullptr, *scratch = nullptr;
  float* scratch32 = nullptr;      // FP32 operator copies / factorisations (mixed-precision path)
  int* piv32 = nullptr;
  int *piv = nullptr, *dirty = nullptr, *fired = nullptr;
  unsigned* err = nullptr;
  int* has_near = nullptr;
  int* involved = nullptr;         // vesicles in a near pair this step (hybrid: they relax exactly)
  unsigned long long* fb_acc = nullptr;  // [0] vesicles taking the exact fallback, summed over steps; [1] steps
  int64_t learned_steps = 0;       // steps whose relaxation was the learned map
  NearBufs nb{nullptr, nullptr};
  double* corr = nullptr;          // correction state (6 N + 16 doubles per vesicle)
  int *cactive = nullptr, *cpiv = nullptr;
  float* xin = nullptr;            // network input rows (M x feature width)
  StdFrame* frames = nullptr;      // standardisation frames (M)
  struct vs_mlp* net = nullptr;    // learned relaxation map (hybrid mode), borrowed
  double net_scale = 1.0;
  int net_kmax = 0;
  struct vs_mlp* flow_adv = nullptr;  // learned advection and tension columns (hybrid mode), borrowed
  struct vs_mlp* flow_ten = nullptr;
  int flow_kf = 0, flow_kout = 0;
  struct vs_mlp* near_net[NEAR_LAYERS] = {};  // learned near-field layers (hybrid mode), borrowed
  int near_kf = 0, near_kout = 0;
  int cur = 0;
  int64_t steps = 0;
  int64_t launches = 0;
  Prof prof;
  // one captured step per (operator-slot parity, relaxation kind: learned 0 / exact 1)
  cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t graph_launches[4] = {0, 0, 0, 0};
  int ff_variant = 0;                              // FP32 far-field launch shape (FF_VARIANTS)
  FfSymState ffs;                                  // symmetric FP32 far field, used when ffs.on
  GmresState gm;                                   // fully implicit step (mode 2)
  std::string msg;
};

struct vs_farfield_plan {
  Layout L;
  DevLayout D;
  SourceBufs B;
  FfSymState ffs;
  double mu = 1.0;
  int near_mask = 0, precision = 0;
  cudaStream_t stream = nullptr;
  unsigned* err = nullptr;
  std::string msg;
};

namespace {

vs_status cuda_fail(std::string& msg, cudaError_t e, const char* where) {
  msg = std::string(where) + ": " + cudaGetErrorString(e);
  return (e == cudaErrorMemoryAllocation) ? VS_ERR_NOMEM : VS_ERR_CUDA;
}

#define VS_CK(h, x, where)                          \
  do {                                              \
    cudaError_t e_ = (x);                           \
    if (e_ != cudaSuccess) return cuda_fail((h)->msg, e_, where); \
  } while (0)

// Record a CUDA event before a launch when profiling; returns the pool slot or -1.
int prof_begin(vs_suspension* h, const char* name) {
  h->launches += 1;
  Prof& P = h->prof;
  if (!P.on) return -1;
  const size_t k = P.rec_id.size();
  while (P.pool.size() < 2 * (k + 1)) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    P.pool.push_back(e);
  }
  P.rec_id.push_back(P.id(name));
  cudaEventRecord(P.pool[2 * k], h->stream);
  return (int)k;
}

void prof_end(vs_suspension* h, int k) {
  if (k < 0) return;
  cudaEventRecord(h->prof.pool[2 * k + 1], h->stream);
}

// Fold recorded event pairs into per-kernel totals (synchronises the stream).
void prof_collect(vs_suspension* h) {
  Prof& P = h->prof;
  if (P.rec_id.empty()) return;
  cudaStreamSynchronize(h->stream);
  for (size_t k = 0; k < P.rec_id.size(); ++k) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, P.pool[2 * k], P.pool[2 * k + 1]);
    P.total_ms[P.rec_id[k]] += ms;
    P.count[P.rec_id[k]] += 1;
  }
  P.rec_id.clear();
}

#define VS_LAUNCH(h, name, ...)              \
  do {                                      \
    const int pk_ = prof_begin((h), (name)); \
    __VA_ARGS__;                            \
    prof_end((h), pk_);                     \
  } while (0)

constexpr size_t LU_SMEM_MAX = 200 * 1024;  // dynamic shared memory granted to k_lu_smem

// Batched LU: staged through shared memory when the largest matrix fits, else in global memory.
template <class Geo>
void launch_lu(vs_suspension* h, const char* name, const Geo& geo, int nmax_dim, const int* active) {
  const size_t bytes = (size_t)nmax_dim * nmax_dim * sizeof(typename Geo::T);
  if (bytes <= LU_SMEM_MAX) {
    VS_LAUNCH(h, name, k_lu_smem<Geo><<<h->L.M, 256, bytes, h->stream>>>(geo, h->err, active));
  } else {
    VS_LAUNCH(h, name, k_lu<Geo><<<h->L.M, 256, 0, h->stream>>>(geo, h->err, active));
  }
}

// In-place FP32 inverses by Gauss-Jordan in registers (k_gj_inverse) for matrices up to 128 x 128;
// false when nmax_dim is larger (nothing launched).
// The FP32 Gauss-Jordan inverse shape for matrices of order <= nmax_dim, on M matrices of geo.
template <class Geo>
cudaError_t gj32_launch(const Geo& geo, int nmax_dim, int M, cudaStream_t st, unsigned* err, const int* active,
                        int* fallbacks) {
  if (nmax_dim <= 32) {
    k_gj_inverse<2, 2, 16><<<M, 256, 0, st>>>(geo, err, active, fallbacks);
  } else if (nmax_dim <= 64) {
    k_gj_inverse<4, 8, 8><<<M, 128, 0, st>>>(geo, err, active, fallbacks);
  } else if (nmax_dim <= 128) {
    k_gj_inverse<8, 8, 16><<<M, 256, 0, st>>>(geo, err, active, fallbacks);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaSuccess;  // launch errors stay pending for the caller's check
}

bool launch_gj32(vs_suspension* h, const char* name, const LuGeo32& geo, int nmax_dim, const int* active) {
  if (nmax_dim > 128) return false;
  VS_LAUNCH(h, name, gj32_launch(geo, nmax_dim, h->L.M, h->stream, h->err, active, nullptr));
  return true;
}

// k_self_matrix: one CTA per 16 x 16 tile of the upper triangle of the largest vesicle
inline dim3 self_grid(int nmax, int M) {
  const int nt = (nmax + SM_TILE - 1) / SM_TILE;
  return dim3(nt * (nt + 1) / 2, M);
}

inline dim3 gemm_grid(int m, int n, int M) { return dim3((n + GT - 1) / GT, (m + GT - 1) / GT, M); }

// FP32 operator product C = A B of every vesicle (Op: operand functors, m x n output): with FP32 FMAs
// (k_bgemm), or on the tensor cores with the three-part BF16 split (k_bgemm_tc) under VS_FLAG_TC_GEMM.
template <class Op>
void gemm32(vs_suspension* h, const char* name, const Op& op, int m, int n, const int* active) {
  if (h->p.flags & VS_FLAG_TC_GEMM) {
    const dim3 grid((n + TC_BN - 1) / TC_BN, (m + TC_BM - 1) / TC_BM, h->L.M);
    VS_LAUNCH(h, name, k_bgemm_tc<Op><<<grid, TC_THREADS, TC_SMEM, h->stream>>>(op, active, h->err));
  } else {
    VS_LAUNCH(h, name, k_bgemm<Op><<<gemm_grid(m, n, h->L.M), 256, 0, h->stream>>>(op, active));
  }
}

FlowDev flow_dev(const vs_flow& f) { return FlowDev{f.kind, f.p[0], f.p[1]}; }

// Refinement kernels: 256 threads per vesicle when the vesicles are large or too few to give every SM
// several, else 128.
inline bool mp_wide(const vs_suspension* h) { return h->L.nmax > 64 || h->L.M < 4 * 148; }

// Launch a refinement kernel with the CTA size of mp_wide and the mat-vec column capacity (128 or 256)
// that covers 2 nmax.
#define MP_DISPATCH(h, name, kern, grid, args)                                                              \
  do {                                                                                                      \
    const bool wide_ = mp_wide(h), small_ = 2 * (h)->L.nmax <= 128;                                          \
    if (wide_ && small_)                                                                                     \
      VS_LAUNCH(h, name, kern<MP_THREADS_WIDE, 128><<<grid, MP_THREADS_WIDE, 0, (h)->stream>>> args);         \
    else if (wide_)                                                                                          \
      VS_LAUNCH(h, name, kern<MP_THREADS_WIDE, 256><<<grid, MP_THREADS_WIDE, 0, (h)->stream>>> args);         \
    else if (small_)                                                                                         \
      VS_LAUNCH(h, name, kern<MP_THREADS, 128><<<grid, MP_THREADS, 0, (h)->stream>>> args);                   \
    else                                                                                                     \
      VS_LAUNCH(h, name, kern<MP_THREADS, 256><<<grid, MP_THREADS, 0, (h)->stream>>> args);                   \
  } while (0)

// Mixed precision (default): FP32 operator products and factorisations refined in FP64.
// FP32 factorisations (refined in FP64, or preconditioning the implicit step's FP64 GMRES) unless FP64
// operators are asked for
inline bool mixed(const vs_suspension* h) { return !(h->p.flags & VS_FLAG_DIRECT_FP64); }
// FP32 operator products by the fused per-vesicle kernels (k_fused.cuh; vesicles of at most 64 points) instead
// of one batched GEMM launch per product
inline bool fused(const vs_suspension* h) {
  return mixed(h) && h->L.nmax <= FZ && !(h->p.flags & (VS_FLAG_TC_GEMM | VS_FLAG_OPS_BATCHED));
}

// S, T, L at slot s for the geometry currently in the SourceBufs, then LU of L.
vs_status build_operators(vs_suspension* h, const double* xy, int s, const int* active) {
  const Layout& L = h->L;
  const int M = L.M, n = L.nmax;
  const VesIndex vi = h->D.vi();
  if (mixed(h)) {
    VS_LAUNCH(h, "k_self_matrix_df", k_self_matrix_df<<<self_grid(n, M), 256, 0, h->stream>>>(vi, h->B.sdf, h->D.tabdf,
                                                                      h->D.logtab, h->scratch32, s, active));
  } else {
    VS_LAUNCH(h, "k_self_matrix", k_self_matrix<<<self_grid(n, M), 256, 0, h->stream>>>(vi, xy, h->B.sa, h->B.tx, h->B.ty,
                                                                      h->D.tab, h->p.mu, h->scratch, s, active));
  }
  OpCtx c{vi, h->D.tab, h->B.sa, h->B.tx, h->B.ty, h->scratch, h->scratch32, h->D.tab32, h->B.g32};
  if (fused(h)) {
    VS_LAUNCH(h, "k_fused_tl", k_fused_tl<<<M, FUSED_THREADS, fz_tl_smem(), h->stream>>>(c, s, active));
    launch_gj32(h, "k_gj_inverse<L>", LuGeo32{vi, h->scratch32, MatLayout::slot(s) + MatLayout::L, 1, 0, h->piv32, s}, n, active);
  } else if (mixed(h)) {
    gemm32(h, "k_bgemm<OpT32>", OpT32{c, s}, 2 * n, n, active);
    gemm32(h, "k_bgemm<OpL32>", OpL32{c, s}, n, n, active);
    static_assert(NMAX <= 128, "the FP32 inverse of L is formed in registers");
    launch_gj32(h, "k_gj_inverse<L>", LuGeo32{vi, h->scratch32, MatLayout::slot(s) + MatLayout::L, 1, 0, h->piv32, s}, n, active);
  } else {
    VS_LAUNCH(h, "k_bgemm<OpT>", k_bgemm<OpT><<<gemm_grid(2 * n, n, M), 256, 0, h->stream>>>(OpT{c, s}, active));
    VS_LAUNCH(h, "k_bgemm<OpL>", k_bgemm<OpL><<<gemm_grid(n, n, M), 256, 0, h->stream>>>(OpL{c, s}, active));
    launch_lu(h, "k_lu<L>", LuGeo{vi, h->scratch, MatLayout::slot(s) + MatLayout::L, 1, 0, h->piv, s}, n, active);
  }
  VS_CK(h, cudaGetLastError(), "operator build");
  return VS_OK;
}

inline GeomOut geom_active(GeomOut g, const int* active, const float4* logtab) {
  g.active = active;
  g.logtab = logtab;
  return g;
}

vs_status geometry(vs_suspension* h, const double* xy, bool with_force, const int* active = nullptr) {
  ForceOut fo{};
  if (with_force)
    fo = ForceOut{h->B.f, h->u, h->B.src, h->B.centre, h->B.centre32, h->B.h2, h->B.g64, h->B.gsum};
  VS_LAUNCH(h, "k_geometry", launch_geometry(h->L.M, h->L.nmax, h->stream, h->D.vi(), xy, h->sigma, h->D.tab, h->p.kappa_b,
                                             h->p.mu, flow_dev(h->flow), geom_active(h->B.geom(), active, h->D.logtab),
                                             fo, nullptr));
  VS_CK(h, cudaGetLastError(), "geometry");
  return VS_OK;
}

// Launch shapes of the FP32 far field (threads per CTA, source points staged per chunk). All give the
// same result bit for bit; the fastest for a suspension is picked by tune_far_field.
struct FfVariant {
  int threads, chunk;
};
constexpr FfVariant FF_VARIANTS[] = {{128, 2048}, {64, 2048}, {256, 2048}, {128, 1024}, {64, 1024}, {32, 1024}};
constexpr int FF_NVARIANTS = (int)(sizeof(FF_VARIANTS) / sizeof(FF_VARIANTS[0]));

void launch_far_field_f32(const vs_suspension* h, int var, FarFieldArgs a) {
  const FfVariant fv = FF_VARIANTS[var];
  const bool big = fv.chunk == 2048;
  a.chunk = big ? h->D.chunk : h->D.chunk1k;
  a.nchunk = (int)(big ? h->L.chunk.size() : h->L.chunk1k.size()) - 1;
  const int grid = (int)((h->L.P + fv.threads - 1) / fv.threads);
  const float4* src = h->B.src;
  const float4* c32 = h->B.centre32;
  const float2* h2 = h->B.h2;
  const float2* gs = h->B.gsum;
  cudaStream_t st = h->stream;
  switch (var) {
    case 0: k_farfield_f32<128, 2048><<<grid, 128, 0, st>>>(a, src, c32, h2, gs); break;
    case 1: k_farfield_f32<64, 2048><<<grid, 64, 0, st>>>(a, src, c32, h2, gs); break;
    case 2: k_farfield_f32<256, 2048><<<grid, 256, 0, st>>>(a, src, c32, h2, gs); break;
    case 3: k_farfield_f32<128, 1024><<<grid, 128, 0, st>>>(a, src, c32, h2, gs); break;
    case 4: k_farfield_f32<64, 1024><<<grid, 64, 0, st>>>(a, src, c32, h2, gs); break;
    default: k_farfield_f32<32, 1024><<<grid, 32, 0, st>>>(a, src, c32, h2, gs); break;
  }
}

// k_ff_moments: one thread per point of the largest vesicle, whole warps
inline int ff_moment_threads(const Layout& L) { return (L.nmax + 31) / 32 * 32; }
// k_tree_moments: CTAs striding over the boxes of a level (a level holds fewer than M boxes)
inline int tree_moment_grid(int M) { return std::min(M, 4 * 148); }

FarFieldArgs far_field_args(vs_suspension* h) {
  const Layout& L = h->L;
  return FarFieldArgs{L.P, L.M, h->D.owner, h->D.off, h->D.chunk, (int)L.chunk.size() - 1,
                      h->p.near_field ? 1 : 0, h->u, h->B.near_cnt, h->B.near_v, h->err};
}

// Symmetric FP32 far field: eligible when M >= 2 and the chunk slots (one float4 per point and chunk of at
// most FFS_V vesicles) fit in an eighth of the device's memory; otherwise, and with
// VS_FLAG_FARFIELD_PER_TARGET, the per-target kernel runs.
FfSymArgs ffs_args(const FfSymState& f, const Layout& L, int near_mask, const SourceBufs& B, unsigned* err) {
  return FfSymArgs{L.P, L.M, f.nchunk, near_mask, f.part, f.slots, B.near_cnt, B.near_v, err,
                   f.vid, f.poff, f.roff, f.nreal, f.chunk, f.padded ? f.psrc : B.src};
}

// Persistent grid of one instantiation: CTAs per SM as many as fit, or per_sm when smaller.
template <int RR, int RC, bool EQ, int V>
cudaError_t ffs_prepare(int per_sm_want, int* grid) {
  const size_t smem = ffs_smem_bytes(RC, V);
  cudaError_t e = cudaFuncSetAttribute(k_farfield_sym<RR, RC, EQ, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_farfield_sym<RR, RC, EQ, V>, 32 * FFS_W, smem)) !=
      cudaSuccess)
    return e;
  per_sm = std::max(per_sm, 1);
  if (per_sm_want > 0) per_sm = std::min(per_sm, per_sm_want);
  *grid = sms * per_sm;
  return cudaSuccess;
}

template <int RR, int RC, bool EQ>
cudaError_t ffs_prepare_v(int V, int per_sm, int* grid) {
  return V == 8 ? ffs_prepare<RR, RC, EQ, 8>(per_sm, grid)
                : V == 32 ? ffs_prepare<RR, RC, EQ, 32>(per_sm, grid) : ffs_prepare<RR, RC, EQ, 16>(per_sm, grid);
}

// The instantiated pairs of classes (row segments >= column segments); eq: equal N of 32, 64 or 128 in index
// order (no padding, identity order), chunks of V = 8, 16 or 32 vesicles; otherwise V = 16.
cudaError_t ffs_prepare(int rr, int rc, bool eq, int V, int per_sm, int* grid) {
  if (eq) {
    switch (rr) {
      case 4: return ffs_prepare_v<4, 4, true>(V, per_sm, grid);
      case 2: return ffs_prepare_v<2, 2, true>(V, per_sm, grid);
      default: return ffs_prepare_v<1, 1, true>(V, per_sm, grid);
    }
  }
  switch (rr * 8 + rc) {
    case 4 * 8 + 4: return ffs_prepare<4, 4, false, FFS_V>(per_sm, grid);
    case 4 * 8 + 2: return ffs_prepare<4, 2, false, FFS_V>(per_sm, grid);
    case 4 * 8 + 1: return ffs_prepare<4, 1, false, FFS_V>(per_sm, grid);
    case 2 * 8 + 2: return ffs_prepare<2, 2, false, FFS_V>(per_sm, grid);
    case 2 * 8 + 1: return ffs_prepare<2, 1, false, FFS_V>(per_sm, grid);
    default: return ffs_prepare<1, 1, false, FFS_V>(per_sm, grid);
  }
}

// Sets f up for the layout when `wanted` and the layout is eligible; leaves f.on false otherwise. V: vesicles
// per chunk (equal N only; 16 otherwise), per_sm: persistent CTAs per SM (0: as many as fit).
cudaError_t ffs_setup(FfSymState& f, const Layout& L, bool wanted, cudaStream_t st, int V = FFS_V, int per_sm = 0) {
  f.release();
  if (!wanted || L.M < 2) return cudaSuccess;
  // symmetric order: classes of 4, 2, 1 segments, vesicle index ascending inside a class
  std::vector<int> vid;
  for (int R : {4, 2, 1})
    for (int v = 0; v < L.M; ++v)
      if (ffs_segments(L.N[v]) == R) vid.push_back(v);
  std::vector<int64_t> poff(L.M), roff(L.M);
  std::vector<int> nreal(L.M), cls(L.M);
  int64_t pp = 0;
  bool padded = false;
  for (int s = 0; s < L.M; ++s) {
    const int v = vid[s];
    cls[s] = ffs_segments(L.N[v]);
    poff[s] = pp;
    roff[s] = L.off[v];
    nreal[s] = L.N[v];
    pp += 32 * cls[s];
    if (v != s || L.N[v] != 32 * cls[s]) padded = true;
  }
  if (padded) V = FFS_V;
  std::vector<int2> chunk;
  std::vector<int> ccls;
  for (int s = 0; s < L.M;) {
    int n = 0;
    while (s + n < L.M && n < V && cls[s + n] == cls[s]) ++n;
    chunk.push_back(make_int2(s, n));
    ccls.push_back(cls[s]);
    s += n;
  }
  const int nchunk = (int)chunk.size();
  size_t free_b = 0, total_b = 0;
  cudaError_t e;
  if ((e = cudaMemGetInfo(&free_b, &total_b)) != cudaSuccess) return e;
  // partial-sum memory: one slot (16 bytes a point) per chunk within the budget (1/8 of the device memory, or
  // VS_FFS_SLOT_BYTES), else the phased evaluation with groups of S chunks; fewer than 4 slots: none
  size_t budget = total_b / 8;
  if (const char* sb = std::getenv("VS_FFS_SLOT_BYTES")) budget = (size_t)std::strtoull(sb, nullptr, 10);
  const size_t per_slot = (size_t)L.P * sizeof(float4);
  int S = nchunk;
  if ((size_t)nchunk * per_slot > budget) {
    S = (int)std::min<size_t>(budget / per_slot, (size_t)nchunk);
    if (S < 4) return cudaSuccess;
  }
  const int G = (nchunk + S - 1) / S;
  // tiles per (phase, pair of classes): whole tiles first, the half-empty diagonal ones last
  std::vector<int2> tiles;
  const int pairs[FFS_NPAIR][2] = {{4, 4}, {4, 2}, {4, 1}, {2, 2}, {2, 1}, {1, 1}};
  int grid_of[FFS_NPAIR] = {};
  for (int k = 0; k < FFS_NPAIR; ++k)
    if ((e = ffs_prepare(pairs[k][0], pairs[k][1], !padded, V, per_sm, &grid_of[k])) != cudaSuccess) return e;
  for (int ga = 0; ga < G; ++ga)
    for (int gb = ga; gb < G; ++gb) {
      const int a0 = ga * S, a1 = std::min(nchunk, a0 + S), b0 = gb * S, b1 = std::min(nchunk, b0 + S);
      FfSymState::Phase ph{(int)f.launch.size(), 0, ga, gb, a1 - a0, b1 - b0};
      for (int k = 0; k < FFS_NPAIR; ++k) {
        const size_t t0 = tiles.size();
        for (int i = a0; i < a1; ++i)
          for (int j = std::max(b0, i + 1); j < b1; ++j)
            if (ccls[i] == pairs[k][0] && ccls[j] == pairs[k][1]) tiles.push_back(make_int2(i, j));
        if (ga == gb && pairs[k][0] == pairs[k][1])
          for (int i = a0; i < a1; ++i)
            if (ccls[i] == pairs[k][0]) tiles.push_back(make_int2(i, i));
        if (tiles.size() == t0) continue;
        const int nt = (int)(tiles.size() - t0);
        f.launch.push_back(FfSymState::Launch{pairs[k][0], pairs[k][1], nt, std::min(grid_of[k], nt), (int64_t)t0});
        ++ph.count;
      }
      f.phase.push_back(ph);
    }
#define VS_TRY(x) do { if ((e = (x)) != cudaSuccess) return e; } while (0)
  VS_TRY(dalloc(&f.tiles, (int64_t)tiles.size()));
  VS_TRY(upload(f.tiles, tiles.data(), (int64_t)tiles.size(), st));
  VS_TRY(dalloc(&f.part, (int64_t)S * L.P));
  VS_TRY(dalloc(&f.ctr, (int64_t)f.launch.size()));
  if (S < nchunk) {  // the chunk of every point, for the phased reduction
    std::vector<int> pchunk(L.P);
    for (int c = 0; c < nchunk; ++c)
      for (int q = chunk[c].x; q < chunk[c].x + chunk[c].y; ++q)
        for (int i = 0; i < nreal[q]; ++i) pchunk[roff[q] + i] = c;
    VS_TRY(dalloc(&f.pchunk, L.P));
    VS_TRY(upload(f.pchunk, pchunk.data(), L.P, st));
  }
  VS_TRY(dalloc(&f.vid, L.M)); VS_TRY(upload(f.vid, vid.data(), L.M, st));
  VS_TRY(dalloc(&f.poff, L.M)); VS_TRY(upload(f.poff, poff.data(), L.M, st));
  VS_TRY(dalloc(&f.roff, L.M)); VS_TRY(upload(f.roff, roff.data(), L.M, st));
  VS_TRY(dalloc(&f.nreal, L.M)); VS_TRY(upload(f.nreal, nreal.data(), L.M, st));
  VS_TRY(dalloc(&f.chunk, nchunk)); VS_TRY(upload(f.chunk, chunk.data(), nchunk, st));
  if (padded) VS_TRY(dalloc(&f.psrc, pp));
#undef VS_TRY
  f.padded = padded;
  f.V = V;
  f.per_sm = per_sm;
  f.nchunk = nchunk;
  f.slots = S;
  f.phased = S < nchunk;
  f.on = true;
  return cudaStreamSynchronize(st);
}

// The pair kernels of one phase: one persistent launch per pair of classes with tiles in it.
void ffs_launch_phase(const FfSymState& f, const FfSymArgs& a, const SourceBufs& B, int ph, cudaStream_t st) {
  const FfSymState::Phase& P = f.phase[ph];
  for (int k = P.first; k < P.first + P.count; ++k) {
    const FfSymState::Launch& l = f.launch[k];
    const FfSymTiles t{f.tiles + l.tile_off, l.ntile, f.ctr + k};
    const size_t smem = ffs_smem_bytes(l.rc, f.V);
    const int g = l.grid, nt = 32 * FFS_W;
    const float4* c32 = B.centre32;
    const float2 *h2 = B.h2, *gs = B.gsum;
    if (!f.padded) {  // equal N of 32, 64 or 128: a single pair of classes
#define VS_FFS_EQ(R)                                                                                          \
  (f.V == 8 ? k_farfield_sym<R, R, true, 8><<<g, nt, smem, st>>>(a, t, c32, h2, gs)                           \
            : f.V == 32 ? k_farfield_sym<R, R, true, 32><<<g, nt, smem, st>>>(a, t, c32, h2, gs)              \
                        : k_farfield_sym<R, R, true, 16><<<g, nt, smem, st>>>(a, t, c32, h2, gs))
      switch (l.rr) {
        case 4: VS_FFS_EQ(4); break;
        case 2: VS_FFS_EQ(2); break;
        default: VS_FFS_EQ(1); break;
      }
#undef VS_FFS_EQ
      continue;
    }
    switch (l.rr * 8 + l.rc) {
      case 4 * 8 + 4: k_farfield_sym<4, 4, false, FFS_V><<<g, nt, smem, st>>>(a, t, c32, h2, gs); break;
      case 4 * 8 + 2: k_farfield_sym<4, 2, false, FFS_V><<<g, nt, smem, st>>>(a, t, c32, h2, gs); break;
      case 4 * 8 + 1: k_farfield_sym<4, 1, false, FFS_V><<<g, nt, smem, st>>>(a, t, c32, h2, gs); break;
      case 2 * 8 + 2: k_farfield_sym<2, 2, false, FFS_V><<<g, nt, smem, st>>>(a, t, c32, h2, gs); break;
      case 2 * 8 + 1: k_farfield_sym<2, 1, false, FFS_V><<<g, nt, smem, st>>>(a, t, c32, h2, gs); break;
      default: k_farfield_sym<1, 1, false, FFS_V><<<g, nt, smem, st>>>(a, t, c32, h2, gs); break;
    }
  }
}

// Zero the tile counters (and the near counts), pad the sources if needed, then the pair kernels; u is added to
// by ffs_reduce (one pass), or here phase by phase (phased: each phase's slots are reduced before the next
// phase writes them), the near lists sorted after the last phase.
void ffs_launch(const FfSymState& f, const FfSymArgs& a, const SourceBufs& B, const DevLayout& D, double* u,
                cudaStream_t st) {
  cudaMemsetAsync(f.ctr, 0, f.launch.size() * sizeof(unsigned), st);
  if (a.near_mask) cudaMemsetAsync(B.near_cnt, 0, a.P * sizeof(int), st);
  if (f.padded) k_ffs_pad<<<a.M, 128, 0, st>>>(a, B.src, f.psrc);
  const int rg = (int)((a.P + 255) / 256);
  for (int ph = 0; ph < (int)f.phase.size(); ++ph) {
    ffs_launch_phase(f, a, B, ph, st);
    if (f.phased) {
      const FfSymState::Phase& P = f.phase[ph];
      k_ffs_reduce_phase<<<rg, 256, 0, st>>>(a, D.owner, D.off, f.pchunk, P.ga, P.gb, P.na, P.nb, u);
    }
  }
  if (f.phased && a.near_mask) k_ffs_near_sort<<<rg, 256, 0, st>>>(a);
}

void ffs_reduce(const FfSymState& f, const FfSymArgs& a, const DevLayout& D, double* u, cudaStream_t st) {
  if (!f.phased) k_farfield_sym_reduce<<<(int)((a.P + 255) / 256), 256, 0, st>>>(a, D.owner, D.off, u);
}

vs_status far_field(vs_suspension* h) {
  const Layout& L = h->L;
  if (L.M < 2) return VS_OK;
  const FarFieldArgs a = far_field_args(h);
  if (h->p.flags & VS_FLAG_FARFIELD_FP64) {
    const int grid = (int)((L.P + FF_THREADS - 1) / FF_THREADS);
    VS_LAUNCH(h, "k_farfield_f64", k_farfield_f64<<<grid, FF_THREADS, 0, h->stream>>>(a, h->xy, h->B.g64, h->B.length, h->D.N));
  } else if (h->p.flags & VS_FLAG_FARFIELD_TREE) {
    const int mt = ff_moment_threads(L);
    const FfTreeArgs t = h->B.tree(L.M);
    VS_LAUNCH(h, "k_ff_moments", k_ff_moments<FF_MP_P><<<L.M, mt, ffm_smem(FF_MP_P, mt), h->stream>>>(
                                     h->D.off, h->B.src, h->B.mpcoef, h->B.mpa0, h->B.vraw));
    VS_LAUNCH(h, "k_tree_build", k_tree_build<<<1, TREE_THREADS, tree_build_smem(L.M), h->stream>>>(t));
    VS_LAUNCH(h, "k_tree_moments", k_tree_moments<<<tree_moment_grid(L.M), TM_THREADS, 0, h->stream>>>(t, 0, 1));
    for (int l = TREE_LMAX - 1; l >= 0; --l)
      VS_LAUNCH(h, "k_tree_moments", k_tree_moments<<<tree_moment_grid(L.M), TM_THREADS, 0, h->stream>>>(t, l, 0));
    const FfLocArgs la = h->B.loc(L.M);
    VS_LAUNCH(h, "k_ff_local_tree", k_ff_local_tree<FF_MP_P><<<L.M, 128, 0, h->stream>>>(la, t));
    VS_LAUNCH(h, "k_farfield_loc", k_farfield_loc<FF_MP_P><<<L.M, 128, 0, h->stream>>>(a, la, h->B.src));
  } else if (h->p.flags & VS_FLAG_FARFIELD_MULTIPOLE) {
    const int mt = ff_moment_threads(L);
    VS_LAUNCH(h, "k_ff_moments", k_ff_moments<FF_MP_P><<<L.M, mt, ffm_smem(FF_MP_P, mt), h->stream>>>(
                                     h->D.off, h->B.src, h->B.mpcoef, h->B.mpa0));
    const FfLocArgs la = h->B.loc(L.M);
    VS_LAUNCH(h, "k_ff_local", k_ff_local<FF_MP_P><<<L.M, 128, 0, h->stream>>>(la));
    VS_LAUNCH(h, "k_farfield_loc", k_farfield_loc<FF_MP_P><<<L.M, 128, 0, h->stream>>>(a, la, h->B.src));
  } else if (h->ffs.on) {
    const FfSymArgs fa = ffs_args(h->ffs, L, h->p.near_field ? 1 : 0, h->B, h->err);
    VS_LAUNCH(h, "k_farfield_sym", ffs_launch(h->ffs, fa, h->B, h->D, h->u, h->stream));
    VS_LAUNCH(h, "k_farfield_sym_reduce", ffs_reduce(h->ffs, fa, h->D, h->u, h->stream));
  } else {
    VS_LAUNCH(h, "k_farfield_f32", launch_far_field_f32(h, h->ff_variant, a));
  }
  VS_CK(h, cudaGetLastError(), "far field");
  return VS_OK;
}

// Autotuner of the FP32 far-field launch shape: every variant timed on the suspension's own sources
// (CUDA events, best of two launches after one warm-up), the fastest kept. Results are cached per
// (device name, M, points, near mask) for the process, and in the text file named by VS_TUNE_CACHE
// when that variable is set (one "key variant" line per entry). The far field writes only the
// velocity accumulator and near lists, which every step rebuilds; the caller refreshes them.
std::map<std::string, int>& tune_cache() {
  static std::map<std::string, int> c;
  return c;
}

// Autotuner of the symmetric far field (equal point counts): chunk size V (8, 16, 32 vesicles) and persistent
// CTAs per SM (as many as fit, or 2), each timed on the suspension's own sources (best of two launches after
// one warm-up); cached as the per-target kernel's shapes are, under a key of its own.
vs_status tune_symmetric(vs_suspension* h, const char* devname) {
  const Layout& L = h->L;
  char key[512];
  snprintf(key, sizeof key, "sym|%s|M=%d|P=%lld|near=%d", devname, L.M, (long long)L.P, h->p.near_field ? 1 : 0);
  for (char* c = key; *c; ++c)
    if (*c == ' ') *c = '_';
  auto& cache = tune_cache();
  const char* path = std::getenv("VS_TUNE_CACHE");
  if (!cache.count(key) && path) {
    if (FILE* f = std::fopen(path, "r")) {
      char k[512];
      int var = 0;
      while (std::fscanf(f, "%511s %d", k, &var) == 2)
        if (var >= 0) cache[k] = var;
      std::fclose(f);
    }
  }
  const bool want = true;
  auto it = cache.find(key);
  if (it != cache.end()) {
    VS_CK(h, ffs_setup(h->ffs, L, want, h->stream, it->second / 10, it->second % 10), "autotune");
    return VS_OK;
  }
  cudaEvent_t e0, e1;
  VS_CK(h, cudaEventCreate(&e0), "autotune");
  VS_CK(h, cudaEventCreate(&e1), "autotune");
  int best = FFS_V * 10;
  float best_ms = 1e30f;
  for (int V : {8, 16, 32})
    for (int per_sm : {0, 2}) {
      VS_CK(h, ffs_setup(h->ffs, L, want, h->stream, V, per_sm), "autotune");
      const FfSymArgs fa = ffs_args(h->ffs, L, h->p.near_field ? 1 : 0, h->B, h->err);
      ffs_launch(h->ffs, fa, h->B, h->D, h->u, h->stream);
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, h->stream);
        ffs_launch(h->ffs, fa, h->B, h->D, h->u, h->stream);
        cudaEventRecord(e1, h->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; best = V * 10 + per_sm; }
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  VS_CK(h, cudaGetLastError(), "autotune");
  VS_CK(h, ffs_setup(h->ffs, L, want, h->stream, best / 10, best % 10), "autotune");
  cache[key] = best;
  if (path)
    if (FILE* f = std::fopen(path, "a")) {
      std::fprintf(f, "%s %d\n", key, best);
      std::fclose(f);
    }
  return VS_OK;
}

vs_status tune_far_field(vs_suspension* h) {
  const Layout& L = h->L;
  if (L.M < 2 || (h->p.flags & (VS_FLAG_FARFIELD_FP64 | VS_FLAG_NO_AUTOTUNE | VS_FLAG_FARFIELD_MULTIPOLE |
                                VS_FLAG_FARFIELD_TREE)))
    return VS_OK;
  int dev = 0;
  VS_CK(h, cudaGetDevice(&dev), "autotune");
  cudaDeviceProp prop;
  VS_CK(h, cudaGetDeviceProperties(&prop, dev), "autotune");
  if (h->ffs.on) return h->ffs.padded ? VS_OK : tune_symmetric(h, prop.name);
  char key[512];
  snprintf(key, sizeof key, "%s|M=%d|P=%lld|near=%d", prop.name, L.M, (long long)L.P, h->p.near_field ? 1 : 0);
  for (char* c = key; *c; ++c)
    if (*c == ' ') *c = '_';
  auto& cache = tune_cache();
  const char* path = std::getenv("VS_TUNE_CACHE");
  if (!cache.count(key) && path) {
    if (FILE* f = std::fopen(path, "r")) {
      char k[512];
      int var = 0;
      while (std::fscanf(f, "%511s %d", k, &var) == 2)
        if (var >= 0 && var < FF_NVARIANTS) cache[k] = var;
      std::fclose(f);
    }
  }
  auto it = cache.find(key);
  if (it != cache.end()) {
    h->ff_variant = it->second;
    return VS_OK;
  }
  const FarFieldArgs a = far_field_args(h);
  cudaEvent_t e0, e1;
  VS_CK(h, cudaEventCreate(&e0), "autotune");
  VS_CK(h, cudaEventCreate(&e1), "autotune");
  int best = 0;
  float best_ms = 1e30f;
  for (int var = 0; var < FF_NVARIANTS; ++var) {
    launch_far_field_f32(h, var, a);
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, h->stream);
      launch_far_field_f32(h, var, a);
      cudaEventRecord(e1, h->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) { best_ms = ms; best = var; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  VS_CK(h, cudaGetLastError(), "autotune");
  h->ff_variant = best;
  cache[key] = best;
  if (path)
    if (FILE* f = std::fopen(path, "a")) {
      std::fprintf(f, "%s %d\n", key, best);
      std::fclose(f);
    }
  return VS_OK;
}

vs_status mlp_forward(vs_mlp* h, const float* x, int batch, bool out_map);
const float* mlp_output(const vs_mlp* h);

// FP64 relaxation matrices with the operators of slot s and the geometry in the SourceBufs: D4, B,
// W = L^{-1} P B and the LU of A = I - dt (B - T W) (Eq. relaxation_disc).
vs_status relax_matrix_fp64(vs_suspension* h, int s) {
  const int M = h->L.M, n = h->L.nmax;
  const VesIndex vi = h->D.vi();
  OpCtx c{vi, h->D.tab, h->B.sa, h->B.tx, h->B.ty, h->scratch, h->scratch32, h->D.tab32, h->B.g32};
  VS_LAUNCH(h, "k_bgemm<OpD2>", k_bgemm<OpD2><<<gemm_grid(n, n, M), 256, 0, h->stream>>>(OpD2{c}, nullptr));
  VS_LAUNCH(h, "k_bgemm<OpD4>", k_bgemm<OpD4><<<gemm_grid(n, n, M), 256, 0, h->stream>>>(OpD4{c}, nullptr));
  VS_LAUNCH(h, "k_bgemm<OpB>", k_bgemm<OpB><<<gemm_grid(2 * n, n, M), 256, 0, h->stream>>>(OpB{c, s, 0, h->p.kappa_b}, nullptr));
  VS_LAUNCH(h, "k_bgemm<OpB>", k_bgemm<OpB><<<gemm_grid(2 * n, n, M), 256, 0, h->stream>>>(OpB{c, s, 1, h->p.kappa_b}, nullptr));
  VS_LAUNCH(h, "k_bgemm<OpPB>", k_bgemm<OpPB><<<gemm_grid(n, 2 * n, M), 256, 0, h->stream>>>(OpPB{c}, nullptr));
  VS_LAUNCH(h, "k_lu_solve_cols", k_lu_solve_cols<double><<<M, 2 * NMAX, 0, h->stream>>>(vi, h->scratch, s, h->piv, nullptr));
  VS_LAUNCH(h, "k_bgemm<OpA>", k_bgemm<OpA><<<gemm_grid(2 * n, 2 * n, M), 256, 0, h->stream>>>(OpA{c, s, h->p.dt}, nullptr));
  launch_lu(h, "k_lu<A>", LuGeo{vi, h->scratch, MatLayout::A, 2, 0, h->piv, 2}, 2 * n, nullptr);
  VS_CK(h, cudaGetLastError(), "relaxation matrix");
  return VS_OK;
}

// FP32 relaxation matrices with the operators of slot s (FP32 copies) and the geometry in the SourceBufs:
// D4, B, W = Li32 P B and the explicit FP32 inverse of A = I - dt (B - T W) (Eq. relaxation_disc); returns
// where the inverse sits in the FP32 scratch (units of N^2), -1 on a launch error. With active non-null only
// the flagged vesicles' matrices are formed (the 2 x 2 block path forms all).
int64_t relax_matrix_32(vs_suspension* h, int s, const int* active) {
  const int M = h->L.M, n = h->L.nmax;
  const VesIndex vi = h->D.vi();
  OpCtx c{vi, h->D.tab, h->B.sa, h->B.tx, h->B.ty, h->scratch, h->scratch32, h->D.tab32, h->B.g32};
  if (fused(h)) {
    VS_LAUNCH(h, "k_fused_relax", k_fused_relax<<<M, FUSED_THREADS, fz_relax_smem(), h->stream>>>(
                                      c, s, (float)h->p.kappa_b, (float)h->p.dt, active));
    launch_gj32(h, "k_gj_inverse<A>", LuGeo32{vi, h->scratch32, MatLayout::A, 2, 0, h->piv32, 2}, 2 * n, active);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      cuda_fail(h->msg, e, "relaxation matrix");
      return -1;
    }
    return MatLayout::A;
  }
  gemm32(h, "k_bgemm<OpD2_32>", OpD2_32{c}, n, n, active);
  gemm32(h, "k_bgemm<OpD4_32>", OpD4_32{c}, n, n, active);
  gemm32(h, "k_bgemm<OpB32>", OpB32{c, s, 0, h->p.kappa_b}, 2 * n, n, active);
  gemm32(h, "k_bgemm<OpB32>", OpB32{c, s, 1, h->p.kappa_b}, 2 * n, n, active);
  gemm32(h, "k_bgemm<OpPB32>", OpPB32{c}, n, 2 * n, active);
  gemm32(h, "k_bgemm<OpW32>", OpW32{c, s}, n, 2 * n, active);
  gemm32(h, "k_bgemm<OpA32>", OpA32{c, s, h->p.dt}, 2 * n, 2 * n, active);
  const LuGeo32 ga{vi, h->scratch32, MatLayout::A, 2, 0, h->piv32, 2};
  const int64_t ainv = MatLayout::A;
  if (!launch_gj32(h, "k_gj_inverse<A>", ga, 2 * n, active)) {
    // 2N beyond the register Gauss-Jordan: the 2 x 2 block (Schur complement) inverse in place,
    // A = [A11 A12; A21 A22], X1 = A11^{-1}, Y = X1 A12, Z = A21 X1, S = A22 - A21 Y,
    // A^{-1} = [X1 - C12 Z, C12; -S^{-1} Z, S^{-1}] with C12 = -Y S^{-1}; X1, Y, Z, S^{-1} in the free B block
    const int64_t Bq = MatLayout::B;
    const BlkView A11{MatLayout::A, 2, 0, 0}, A12{MatLayout::A, 2, 0, 1}, A21{MatLayout::A, 2, 1, 0},
        A22{MatLayout::A, 2, 1, 1}, X1{Bq, 1, 0, 0}, Y{Bq + 1, 1, 0, 0}, Z{Bq + 2, 1, 0, 0}, Si{Bq + 3, 1, 0, 0};
    const dim3 gcopy((n * n + 255) / 256, M);
    VS_LAUNCH(h, "k_blk_copy", k_blk_copy<<<gcopy, 256, 0, h->stream>>>(c, A11, X1));
    launch_gj32(h, "k_gj_inverse<A11>", LuGeo32{vi, h->scratch32, Bq, 1, 0, h->piv32, 2}, n, nullptr);
    gemm32(h, "k_bgemm<OpBlk32>", OpBlk32{c, X1, A12, Y, Y, 1.f, 0}, n, n, nullptr);
    gemm32(h, "k_bgemm<OpBlk32>", OpBlk32{c, A21, X1, Z, Z, 1.f, 0}, n, n, nullptr);
    gemm32(h, "k_bgemm<OpBlk32>", OpBlk32{c, A21, Y, Si, A22, -1.f, 1}, n, n, nullptr);
    launch_gj32(h, "k_gj_inverse<S>", LuGeo32{vi, h->scratch32, Bq + 3, 1, 0, h->piv32, 2}, n, nullptr);
    gemm32(h, "k_bgemm<OpBlk32>", OpBlk32{c, Y, Si, A12, A12, -1.f, 0}, n, n, nullptr);
    gemm32(h, "k_bgemm<OpBlk32>", OpBlk32{c, Si, Z, A21, A21, -1.f, 0}, n, n, nullptr);
    gemm32(h, "k_bgemm<OpBlk32>", OpBlk32{c, A12, Z, A11, X1, -1.f, 1}, n, n, nullptr);
    VS_LAUNCH(h, "k_blk_copy", k_blk_copy<<<gcopy, 256, 0, h->stream>>>(c, Si, A22));
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    cuda_fail(h->msg, e, "relaxation matrix");
    return -1;
  }
  return ainv;
}

// Exact relaxation (Eq. relaxation_disc) of xs into xo with the operators at slot s; with active non-null
// only the vesicles with active[v] != 0 are processed and written.
vs_status relax_exact(vs_suspension* h, const double* xs, double* xo, int s, const int* active = nullptr) {
  const Layout& L = h->L;
  const int M = L.M;
  const VesIndex vi = h->D.vi();
  vs_status st;
  if ((st = geometry(h, xs, false, active)) != VS_OK) return st;
  if ((st = build_operators(h, xs, s, active)) != VS_OK) return st;
  if (mixed(h)) {
    const int64_t ainv = relax_matrix_32(h, s, active);
    if (ainv < 0) return VS_ERR_CUDA;
    MP_DISPATCH(h, "k_relax_mp", k_relax_mp, M, (vi, xs, h->B.sa, h->B.tx, h->B.ty, h->D.tab, h->scratch32, s, ainv,
                                                    h->p.kappa_b, h->p.dt, xo, h->err, active));
    VS_CK(h, cudaGetLastError(), "relaxation");
    return VS_OK;
  }
  vs_status st2 = relax_matrix_fp64(h, s);
  if (st2 != VS_OK) return st2;
  VS_LAUNCH(h, "k_relax_solve", k_relax_solve<<<M, 256, 0, h->stream>>>(vi, xs, h->scratch, h->piv, xo, active));
  VS_CK(h, cudaGetLastError(), "relaxation");
  return VS_OK;
}

// sigma at the points whose operators sit in slot s (geometry in the SourceBufs), velocity u.
vs_status tension(vs_suspension* h, const double* u, int s) {
  const VesIndex vi = h->D.vi();
  const int M = h->L.M;
  if (mixed(h)) {
    MP_DISPATCH(h, "k_tension_mp", k_tension_mp, M, (vi, h->B.bx, h->B.by, u, h->B.sa, h->B.tx, h->B.ty, h->D.tab,
                                                        h->scratch32, s, h->p.kappa_b, h->sigma, h->err));
  } else {
    VS_LAUNCH(h, "k_tension", k_tension<<<M, 256, 0, h->stream>>>(vi, h->B.bx, h->B.by, u, h->B.pg(), h->D.tab, h->scratch, s,
                                                                 h->piv, h->p.kappa_b, h->sigma));
  }
  VS_CK(h, cudaGetLastError(), "tension");
  return VS_OK;
}

// sigma_out = -L^{-1} P (B X + u) with the operators of slot s and the geometry in the SourceBufs.
vs_status tension_into(vs_suspension* h, const double* u, int s, double* sigma_out, const int* active = nullptr) {
  const VesIndex vi = h->D.vi();
  const int M = h->L.M;
  if (mixed(h)) {
    MP_DISPATCH(h, "k_tension_mp", k_tension_mp, M, (vi, h->B.bx, h->B.by, u, h->B.sa, h->B.tx, h->B.ty, h->D.tab,
                                                        h->scratch32, s, h->p.kappa_b, sigma_out, h->err, active));
  } else {
    VS_LAUNCH(h, "k_tension", k_tension<<<M, 256, 0, h->stream>>>(vi, h->B.bx, h->B.by, u, h->B.pg(), h->D.tab, h->scratch, s,
                                                                 h->piv, h->p.kappa_b, sigma_out, active));
  }
  VS_CK(h, cudaGetLastError(), "tension");
  return VS_OK;
}

// xo = xy + dt (I - M) u with the operators of slot s (Eq. advection_disc).
vs_status advect_into(vs_suspension* h, const double* xy, const double* u, int s, double dt, double* xo,
                      const int* active = nullptr) {
  const VesIndex vi = h->D.vi();
  const int M = h->L.M;
  if (mixed(h)) {
    MP_DISPATCH(h, "k_advect_mp", k_advect_mp, M, (vi, xy, u, h->B.sa, h->B.tx, h->B.ty, h->D.tab, h->scratch32, s,
                                                      dt, xo, h->err, active));
  } else {
    VS_LAUNCH(h, "k_advect", k_advect<<<M, 256, 0, h->stream>>>(vi, xy, u, h->B.pg(), h->D.tab, h->scratch, s, h->piv, dt,
                                                               xo, active));
  }
  VS_CK(h, cudaGetLastError(), "advection");
  return VS_OK;
}

// Learned advection (Eq. advectionMap): X* = X^n + dt (I - M) u with the network's columns at the
// standardised X^n; or learned tension (Eq. advTenMap and S_sigma): sigma = -L^{-1} P (B X + u) at X.
vs_status flow_learned(vs_suspension* h, bool ten, const double* xy, const double* u, double* out) {
  const Layout& L = h->L;
  const VesIndex vi = h->D.vi();
  const int W = feat_width(feat_kmax(h->net_kmax, L.nmax));
  VS_LAUNCH(h, "k_standardize", k_standardize<<<L.M, NMAX, 0, h->stream>>>(vi, xy, h->D.tab, h->xin, W, h->frames,
                                                                           h->net_kmax, true));
  VS_CK(h, cudaGetLastError(), "standardise");
  vs_mlp* net = ten ? h->flow_ten : h->flow_adv;
  vs_status st = mlp_forward(net, h->xin, L.M, true);
  if (st != VS_OK) { h->msg = "flow network forward failed"; return st; }
  const int ld = net->dims.back();
  if (ten) {
    VS_LAUNCH(h, "k_flow_apply<tension>", k_flow_apply<true><<<L.M, NMAX, 0, h->stream>>>(
                                              vi, u, h->frames, mlp_output(net), ld, h->flow_kf, h->flow_kout, h->D.tab,
                                              0.0, nullptr, nullptr, out));
  } else {
    VS_LAUNCH(h, "k_flow_apply<advection>", k_flow_apply<false><<<L.M, NMAX, 0, h->stream>>>(
                                                vi, u, h->frames, mlp_output(net), ld, h->flow_kf, h->flow_kout, h->D.tab,
                                                h->p.dt, xy, out, nullptr));
  }
  VS_CK(h, cudaGetLastError(), "learned flow");
  return VS_OK;
}

// Learned relaxation (VesNet's X_X map): X*_r = redistribute(X*),
// X^{n+1} = lowpass_kmax(X*_r + destandardise(net(standardise(X*_r)))).
vs_status relax_learned(vs_suspension* h, const double* xs, double* xo) {
  const Layout& L = h->L;
  const VesIndex vi = h->D.vi();
  if (!h->net) { h->msg = "hybrid mode needs a relaxation network (vs_set_network)"; return VS_ERR_NO_NETWORK; }
  const int W = feat_width(feat_kmax(h->net_kmax, L.nmax));
  VS_LAUNCH(h, "k_redistribute", k_redistribute<<<L.M, 256, 0, h->stream>>>(vi, xs, h->u, h->D.tab, xo, h->u_r));
  VS_LAUNCH(h, "k_standardize", k_standardize<<<L.M, NMAX, 0, h->stream>>>(vi, xo, h->D.tab, h->xin, W, h->frames,
                                                                           h->net_kmax, true));
  VS_CK(h, cudaGetLastError(), "standardise");
  vs_status st = mlp_forward(h->net, h->xin, L.M, true);
  if (st != VS_OK) { h->msg = "network forward failed"; return st; }
  VS_LAUNCH(h, "k_destandardize_add", k_destandardize_add<<<L.M, NMAX, 0, h->stream>>>(vi, mlp_output(h->net), W,
                                                                                       h->net_scale, h->net_kmax,
                                                                                       h->D.tab, h->frames, xo));
  VS_LAUNCH(h, "k_lowpass", k_lowpass<<<L.M, NMAX, 0, h->stream>>>(vi, h->D.tab, h->net_kmax, xo));
  VS_CK(h, cudaGetLastError(), "destandardise");
  return VS_OK;
}

// Hybrid suspension with the near-field networks set (vs_set_near_networks).
inline bool near_learned_on(const vs_suspension* h) { return h->p.mode == 1 && h->near_net[0] != nullptr; }

// u += near-field correction of every (target, vesicle) pair the far field masked (Sec. 3.3). With
// build_sources the operators of slot s are first built for the source vesicles that have near targets (a
// step with learned advection and tension keeps no operators at X^n otherwise). With the near-field networks
// set (hybrid mode) the layer velocities come from them, and no operators are needed.
vs_status near_field(vs_suspension* h, int s, bool build_sources = false) {
  const Layout& L = h->L;
  const VesIndex vi = h->D.vi();
  VS_CK(h, cudaMemsetAsync(h->has_near, 0, L.M * sizeof(int), h->stream), "near field");
  const int tgrid = (int)((L.P + 127) / 128);
  VS_LAUNCH(h, "k_near_mark", k_near_mark<<<tgrid, 128, 0, h->stream>>>(L.P, h->B.near_cnt, h->B.near_v, h->has_near));
  const size_t smem = near_layers_smem(L.nmax);
  if (near_learned_on(h)) {
    // learned layer velocities (Sec. 3.3, Eq. NearFieldMap): the networks take the relaxation network's input
    const int W = feat_width(feat_kmax(h->net_kmax, L.nmax));
    VS_LAUNCH(h, "k_standardize", k_standardize<<<L.M, NMAX, 0, h->stream>>>(vi, h->xy, h->D.tab, h->xin, W,
                                                                             h->frames, h->net_kmax, true));
    NearNets nn{};
    for (int d = 0; d < NEAR_LAYERS; ++d) {
      vs_status st = mlp_forward(h->near_net[d], h->xin, L.M, true);
      if (st != VS_OK) { h->msg = "near-field network forward failed"; return st; }
      nn.rows[d] = mlp_output(h->near_net[d]);
    }
    nn.ld = h->near_net[0]->dims.back();
    nn.Kf = h->near_kf;
    nn.Kout = h->near_kout;
    nn.frames = h->frames;
    VS_LAUNCH(h, "k_near_layers<learned>", k_near_layers<NEAR_LEARNED><<<L.M, 256, smem, h->stream>>>(
                                               vi, h->has_near, h->xy, h->B.f, h->B.pg(), h->B.length, h->D.tab,
                                               h->scratch, nullptr, s, h->p.mu, h->nb, nn));
  } else if (h->p.flags & VS_FLAG_NEAR_YZ) {
    // Ying-Zorin evaluation at each near target (Sec. 2.2.2) instead of the layers and the RBF
    if (build_sources) {
      vs_status st = build_operators(h, h->xy, s, h->has_near);
      if (st != VS_OK) return st;
    }
    VS_LAUNCH(h, "k_near_layers<yz>", k_near_layers<NEAR_YZ><<<L.M, 256, smem, h->stream>>>(
                                          vi, h->has_near, h->xy, h->B.f, h->B.pg(), h->B.length, h->D.tab,
                                          h->scratch, mixed(h) ? h->scratch32 : nullptr, s, h->p.mu, h->nb,
                                          NearNets{}));
    const int yg = (int)std::min<int64_t>((L.P + 3) / 4, 148 * 32);
    VS_LAUNCH(h, "k_near_yz", k_near_yz<<<yg, 128, 0, h->stream>>>(L.P, h->D.owner, h->D.off, h->D.N, h->B.near_cnt,
                                                                   h->B.near_v, h->xy, h->B.length, h->nb.layer,
                                                                   h->u));
    VS_CK(h, cudaGetLastError(), "near field");
    return VS_OK;
  } else {
    if (build_sources) {
      vs_status st = build_operators(h, h->xy, s, h->has_near);
      if (st != VS_OK) return st;
    }
    VS_LAUNCH(h, "k_near_layers", k_near_layers<NEAR_EXACT><<<L.M, 256, smem, h->stream>>>(
                                      vi, h->has_near, h->xy, h->B.f, h->B.pg(), h->B.length, h->D.tab, h->scratch,
                                      mixed(h) ? h->scratch32 : nullptr, s, h->p.mu, h->nb, NearNets{}));
  }
  if (5 * L.nmax <= NEAR_RBF_SMEM_N) {
    VS_LAUNCH(h, "k_near_rbf", k_near_rbf_smem<<<L.M, 512, near_rbf_smem(5 * L.nmax), h->stream>>>(
                                   vi, h->has_near, h->B.length, h->nb, h->err));
  } else {
    VS_LAUNCH(h, "k_near_rbf", k_near_rbf<<<L.M, 256, 0, h->stream>>>(vi, h->has_near, h->B.length, h->nb, h->err));
  }
  VS_LAUNCH(h, "k_near_apply", k_near_apply<<<tgrid, 128, 0, h->stream>>>(L.P, h->D.owner, h->D.off, h->D.N,
                                                                        h->B.near_cnt, h->B.near_v, h->xy,
                                                                        h->B.length, h->nb, h->u));
  VS_CK(h, cudaGetLastError(), "near field");
  return VS_OK;
}

// Area/length correction of every vesicle whose relative error exceeds corr_tol (Sec. 4.3).
vs_status correction(vs_suspension* h) {
  const Layout& L = h->L;
  const VesIndex vi = h->D.vi();
  VS_LAUNCH(h, "k_corr_init", k_corr_init<<<L.M, NMAX, 0, h->stream>>>(vi, h->xy, h->A0, h->L0, h->p.corr_tol, h->D.tab,
                                                                       h->corr, h->cactive, h->dirty, h->err));
  const int n = 2 * L.nmax + 2;
  const size_t bytes = (size_t)n * n * sizeof(double);
  const size_t bytes32 = (size_t)4 * L.nmax * L.nmax * sizeof(float);
  if (2 * L.nmax <= 32) {
    VS_LAUNCH(h, "k_corr_newton32", k_corr_newton32<2><<<L.M, 256, bytes32, h->stream>>>(vi, h->D.tab, h->A0, h->L0,
                                                                                     h->corr, h->cactive, h->dirty,
                                                                                     CORR_NEWTON_ITERS, h->xy,
                                                                                     h->fired, h->err));
  } else if (2 * L.nmax <= 64) {
    VS_LAUNCH(h, "k_corr_newton32", k_corr_newton32<4><<<L.M, 256, bytes32, h->stream>>>(vi, h->D.tab, h->A0, h->L0,
                                                                                     h->corr, h->cactive, h->dirty,
                                                                                     CORR_NEWTON_ITERS, h->xy,
                                                                                     h->fired, h->err));
  } else if (2 * L.nmax <= 128) {
    VS_LAUNCH(h, "k_corr_newton32", k_corr_newton32<8><<<L.M, 256, bytes32, h->stream>>>(vi, h->D.tab, h->A0, h->L0,
                                                                                     h->corr, h->cactive, h->dirty,
                                                                                     CORR_NEWTON_ITERS, h->xy,
                                                                                     h->fired, h->err));
  } else if (bytes <= LU_SMEM_MAX) {
    VS_LAUNCH(h, "k_corr_newton", k_corr_newton<true><<<L.M, 256, bytes, h->stream>>>(vi, h->D.tab, h->A0, h->L0, h->corr,
                                                                                    h->scratch, h->cpiv, h->cactive,
                                                                                    h->dirty, CORR_NEWTON_ITERS, h->xy,
                                                                                    h->fired, h->err));
  } else {
    VS_LAUNCH(h, "k_corr_newton", k_corr_newton<false><<<L.M, 256, 0, h->stream>>>(vi, h->D.tab, h->A0, h->L0, h->corr,
                                                                                  h->scratch, h->cpiv, h->cactive,
                                                                                  h->dirty, CORR_NEWTON_ITERS, h->xy,
                                                                                  h->fired, h->err));
  }
  VS_CK(h, cudaGetLastError(), "correction");
  return VS_OK;
}

// Hybrid suspension with the advection and tension networks set (vs_set_flow_networks).
inline bool flow_learned_on(const vs_suspension* h) { return h->p.mode == 1 && h->flow_adv && h->flow_ten; }

double exact_gap(const vs_suspension* h) { return h->p.exact_gap > 0.0 ? h->p.exact_gap : HYBRID_EXACT_GAP; }

// Hybrid steps use the learned relaxation except every exact_every-th step (counting from 1), which takes
// the exact one.
inline bool learned_step(const vs_suspension* h) {
  if (h->p.mode != 1) return false;
  return !(h->p.exact_every > 0 && (h->steps + 1) % h->p.exact_every == 0);
}

vs_status step_once(vs_suspension* h) {
  const Layout& L = h->L;
  const int M = L.M;
  const VesIndex vi = h->D.vi();
  vs_status st;
  const int cur = h->cur, nxt = 1 - h->cur;
  // hybrid with flow networks: advection and tension learned in every step (Sec. 3.2), no operators at X^n
  // or X^{n+1}
  const bool lf = flow_learned_on(h);
  // (1) geometry + force at X^n, u = u_inf(X^n)
  if ((st = geometry(h, h->xy, true)) != VS_OK) return st;
  // (2) operators at X^n where the cache is stale (first step, or after a correction)
  if (!lf && (st = build_operators(h, h->xy, cur, h->dirty)) != VS_OK) return st;
  // (3) u += far field (near pairs masked) + near-field correction
  if ((st = far_field(h)) != VS_OK) return st;
  if (h->p.near_field && L.M > 1 && (st = near_field(h, cur, lf)) != VS_OK) return st;
  // the plain step is the fallback of the learned one: vesicles in a near pair this step, or closer to another
  // vesicle than exact_gap (default HYBRID_EXACT_GAP) spacings h, relax exactly in a learned step and, with
  // the flow networks, take the exact advection and tension in every step
  const bool fallback = M > 1 && (learned_step(h) || lf);
  if (fallback) {
    VS_CK(h, cudaMemsetAsync(h->involved, 0, M * sizeof(int), h->stream), "hybrid fallback");
    const int tgrid = (int)((L.P + 127) / 128);
    if (h->p.near_field)
      VS_LAUNCH(h, "k_near_involved", k_near_involved<<<tgrid, 128, 0, h->stream>>>(L.P, h->D.owner, h->B.near_cnt,
                                                                                     h->B.near_v, h->involved));
    VS_LAUNCH(h, "k_proximity", k_proximity<<<M, 128, 0, h->stream>>>(vi, h->xy, h->B.centre, h->B.h2, M,
                                                                       exact_gap(h), h->involved));
    VS_LAUNCH(h, "k_count_flags", k_count_flags<<<1, 256, 0, h->stream>>>(M, h->involved, h->fb_acc));
  }
  // (4) advection
  if (lf) {
    if ((st = flow_learned(h, false, h->xy, h->u, h->xy_star)) != VS_OK) return st;
    if (M > 1) {
      if ((st = build_operators(h, h->xy, cur, h->involved)) != VS_OK) return st;
      if ((st = advect_into(h, h->xy, h->u, cur, h->p.dt, h->xy_star, h->involved)) != VS_OK) return st;
    }
  } else if (mixed(h)) {
    MP_DISPATCH(h, "k_advect_mp", k_advect_mp, M, (vi, h->xy, h->u, h->B.sa, h->B.tx, h->B.ty, h->D.tab, h->scratch32,
                                                      cur, h->p.dt, h->xy_star, h->err));
  } else {
    VS_LAUNCH(h, "k_advect", k_advect<<<M, 256, 0, h->stream>>>(vi, h->xy, h->u, h->B.pg(), h->D.tab, h->scratch, cur, h->piv, h->p.dt,
                                                               h->xy_star));
  }
  VS_CK(h, cudaGetLastError(), "advection");
  // (5) relaxation at X*: exact (plain) or the learned map (hybrid)
  if (learned_step(h)) {
    if ((st = relax_learned(h, h->xy_star, h->xy_next)) != VS_OK) return st;
    if (M > 1 && (st = relax_exact(h, h->xy_star, h->xy_next, nxt, h->involved)) != VS_OK) return st;
  } else {
    if ((st = relax_exact(h, h->xy_star, h->xy_next, nxt)) != VS_OK) return st;
  }
  // (6) redistribution of X^{n+1}; u carried to the new parameters
  VS_LAUNCH(h, "k_redistribute", k_redistribute<<<M, 256, 0, h->stream>>>(vi, h->xy_next, h->u, h->D.tab, h->xy, h->u_r));
  VS_CK(h, cudaGetLastError(), "redistribution");
  // (7) tension at the redistributed X^{n+1}; operators cached in slot nxt for the next step
  if (lf) {
    if ((st = flow_learned(h, true, h->xy, h->u_r, h->sigma)) != VS_OK) return st;
    if (M > 1) {
      if ((st = geometry(h, h->xy, false, h->involved)) != VS_OK) return st;
      if ((st = build_operators(h, h->xy, nxt, h->involved)) != VS_OK) return st;
      if ((st = tension_into(h, h->u_r, nxt, h->sigma, h->involved)) != VS_OK) return st;
    }
  } else {
    if ((st = geometry(h, h->xy, false)) != VS_OK) return st;
    if ((st = build_operators(h, h->xy, nxt, nullptr)) != VS_OK) return st;
    if ((st = tension(h, h->u_r, nxt)) != VS_OK) return st;
  }
  // (8) area/length correction (Newton on the KKT system); marks the cached operators stale where it fires
  if ((st = correction(h)) != VS_OK) return st;
  h->cur = nxt;
  h->steps += 1;
  return VS_OK;
}

// ---- Fully implicit step (mode 2; Sec. 2.2.3, Eq. time_step_sc1), solved by restarted flexible GMRES
// with the block-diagonal (per-vesicle) preconditioner of k_implicit.cuh applied on the right: the Arnoldi
// process runs on A M^{-1}, the preconditioned vectors z_j = M^{-1} v_j are kept and the solution is
// z = z0 + Z y, so an approximate (FP32) M^{-1} costs iterations but no accuracy. Gram-Schmidt is
// classical, applied twice (CGS2) with batched dot products; the small Hessenberg least-squares problem
// (Givens rotations) runs on the host, which reads one column per iteration.

vs_status gmres_alloc(vs_suspension* h) {
  GmresState& g = h->gm;
  const int64_t n = 3 * h->L.P;
  if (g.V && g.alloc_restart == g.restart && g.n == n) return VS_OK;
  g.release();
  g.n = n;
  g.G = (int)std::min<int64_t>((n + GM_THREADS - 1) / GM_THREADS, 4 * 148);
  const int m = g.restart;
  VS_CK(h, dalloc(&g.V, (int64_t)(m + 1) * n), "GMRES buffers");
  VS_CK(h, dalloc(&g.Z, (int64_t)m * n), "GMRES buffers");
  VS_CK(h, dalloc(&g.w, n), "GMRES buffers");
  VS_CK(h, dalloc(&g.z, n), "GMRES buffers");
  VS_CK(h, dalloc(&g.b, n), "GMRES buffers");
  VS_CK(h, dalloc(&g.t1, n), "GMRES buffers");
  VS_CK(h, dalloc(&g.part, (int64_t)(m + 2) * g.G), "GMRES buffers");
  VS_CK(h, dalloc(&g.hd, m + 2), "GMRES buffers");
  VS_CK(h, dalloc(&g.hd2, m + 2), "GMRES buffers");
  VS_CK(h, cudaMallocHost(&g.hh, (m + 2) * sizeof(double)), "GMRES buffers");
  g.alloc_restart = m;
  return VS_OK;
}

// q = A p: the density of p, its far field (and near-field correction) from the other vesicles, the self
// single layer, then both lines of the system (operators of slot s at X^n).
vs_status imp_matvec(vs_suspension* h, int s, const double* p, double* q) {
  const Layout& L = h->L;
  const VesIndex vi = h->D.vi();
  VS_LAUNCH(h, "k_imp_density", k_imp_density<<<L.M, NMAX, 0, h->stream>>>(vi, p, h->B.pg(), h->D.tab, h->p.kappa_b,
                                                                           h->p.mu, h->B.f, h->B.g64, h->B.src,
                                                                           h->B.gsum, h->u));
  vs_status st;
  if ((st = far_field(h)) != VS_OK) return st;
  if (h->p.near_field && L.M > 1 && (st = near_field(h, s)) != VS_OK) return st;
  VS_LAUNCH(h, "k_imp_apply", k_imp_apply<<<L.M, 256, 0, h->stream>>>(vi, p, h->B.f, h->u, h->B.pg(), h->D.tab,
                                                                       h->scratch, s, h->p.dt, q));
  VS_CK(h, cudaGetLastError(), "implicit matrix-vector product");
  return VS_OK;
}

vs_status imp_precond(vs_suspension* h, int s, const double* r, double* out) {
  const VesIndex vi = h->D.vi();
  if (mixed(h)) {
    MP_DISPATCH(h, "k_imp_precond32", k_imp_precond32, h->L.M, (vi, r, h->scratch32, s, h->gm.ainv, h->p.dt, out));
  } else {
    VS_LAUNCH(h, "k_imp_precond", k_imp_precond<<<h->L.M, 256, 0, h->stream>>>(vi, r, h->scratch, h->piv, s, h->p.dt,
                                                                               out));
  }
  VS_CK(h, cudaGetLastError(), "implicit preconditioner");
  return VS_OK;
}

// out[0..J) = <V_j, x> (norm_slot < 0), or out[norm_slot] = ||x|| (J = 1, V = x); with acc non-null the
// results are also added to acc.
vs_status gm_dots(vs_suspension* h, const double* V, int J, const double* x, double* out, double* acc,
                  int norm_slot) {
  GmresState& g = h->gm;
  VS_LAUNCH(h, "k_gm_dots", k_gm_dots<<<g.G, GM_THREADS, 0, h->stream>>>(V, g.n, J, x, g.part));
  VS_LAUNCH(h, "k_gm_reduce", k_gm_reduce<<<J, 32, 0, h->stream>>>(g.part, g.G, J, out, acc, norm_slot));
  VS_CK(h, cudaGetLastError(), "GMRES dot products");
  return VS_OK;
}

vs_status read_doubles(vs_suspension* h, const double* d, int n) {
  VS_CK(h, cudaMemcpyAsync(h->gm.hh, d, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "GMRES readback");
  VS_CK(h, cudaStreamSynchronize(h->stream), "GMRES readback");
  return VS_OK;
}

// Solves A z = b for z (starting from the z in the state) to gm.tol; operators at slot s.
vs_status gmres_solve(vs_suspension* h, int s) {
  GmresState& g = h->gm;
  const int m = g.restart;
  const int64_t n = g.n;
  vs_status st;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
  // ||b||
  if ((st = gm_dots(h, g.b, 1, g.b, g.hd, nullptr, 0)) != VS_OK) return st;
  if ((st = read_doubles(h, g.hd, 1)) != VS_OK) return st;
  const double bnorm = g.hh[0];
  const double target = g.tol * (bnorm > 0.0 ? bnorm : 1.0);
  int iters = 0;
  double res = 0.0;
  for (;;) {
    // r = b - A z into V_0 (unnormalised), beta = ||r||
    if ((st = imp_matvec(h, s, g.z, g.t1)) != VS_OK) return st;
    VS_LAUNCH(h, "k_gm_sub", k_gm_sub<<<g.G, GM_THREADS, 0, h->stream>>>(g.b, g.t1, n, g.w));
    if ((st = gm_dots(h, g.w, 1, g.w, g.hd, nullptr, 0)) != VS_OK) return st;
    if ((st = read_doubles(h, g.hd, 1)) != VS_OK) return st;
    const double beta = g.hh[0];
    res = beta;
    if (!std::isfinite(beta)) { h->msg = "non-finite GMRES residual"; return VS_ERR_UNSTABLE; }
    if (beta <= target) break;
    if (iters >= g.max_iter) break;
    VS_LAUNCH(h, "k_gm_scale", k_gm_scale<<<g.G, GM_THREADS, 0, h->stream>>>(g.w, n, g.hd, g.V));
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int k = 0;
    bool done = false;
    for (int j = 0; j < m && iters < g.max_iter; ++j) {
      double* vj = g.V + (int64_t)j * n;
      double* vn = g.V + (int64_t)(j + 1) * n;
      double* zj = g.Z + (int64_t)j * n;
      if ((st = imp_precond(h, s, vj, zj)) != VS_OK) return st;
      if ((st = imp_matvec(h, s, zj, g.w)) != VS_OK) return st;
      // CGS2: h = V^T w, w -= V h, h2 = V^T w, w -= V h2, h += h2
      if ((st = gm_dots(h, g.V, j + 1, g.w, g.hd, nullptr, -1)) != VS_OK) return st;
      VS_LAUNCH(h, "k_gm_combine", k_gm_combine<<<g.G, GM_THREADS, 0, h->stream>>>(g.V, n, j + 1, g.hd, -1.0, g.w));
      if ((st = gm_dots(h, g.V, j + 1, g.w, g.hd2, g.hd, -1)) != VS_OK) return st;
      VS_LAUNCH(h, "k_gm_combine", k_gm_combine<<<g.G, GM_THREADS, 0, h->stream>>>(g.V, n, j + 1, g.hd2, -1.0, g.w));
      if ((st = gm_dots(h, g.w, 1, g.w, g.hd, nullptr, j + 1)) != VS_OK) return st;
      VS_LAUNCH(h, "k_gm_scale", k_gm_scale<<<g.G, GM_THREADS, 0, h->stream>>>(g.w, n, g.hd + j + 1, vn));
      if ((st = read_doubles(h, g.hd, j + 2)) != VS_OK) return st;
      ++iters;
      k = j + 1;
      // Givens rotations on column j
      double* col = H.data() + (size_t)j * (m + 1);
      for (int i = 0; i <= j + 1; ++i) col[i] = g.hh[i];
      for (int i = 0; i < j; ++i) {
        const double a = col[i], b = col[i + 1];
        col[i] = cs[i] * a + sn[i] * b;
        col[i + 1] = -sn[i] * a + cs[i] * b;
      }
      const double a = col[j], b = col[j + 1];
      const double r = std::hypot(a, b);
      cs[j] = r > 0.0 ? a / r : 1.0;
      sn[j] = r > 0.0 ? b / r : 0.0;
      col[j] = r;
      col[j + 1] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      res = std::fabs(gv[j + 1]);
      if (!std::isfinite(res)) { h->msg = "non-finite GMRES residual"; return VS_ERR_UNSTABLE; }
      if (res <= target || g.hh[j + 1] == 0.0) { done = true; break; }
    }
    // y = R^{-1} g (upper triangular k x k), z += Z y
    for (int i = k - 1; i >= 0; --i) {
      double acc = gv[i];
      for (int c = i + 1; c < k; ++c) acc -= H[(size_t)c * (m + 1) + i] * y[c];
      const double d = H[(size_t)i * (m + 1) + i];
      y[i] = d != 0.0 ? acc / d : 0.0;
    }
    for (int i = 0; i < k; ++i) g.hh[i] = y[i];
    VS_CK(h, cudaMemcpyAsync(g.hd2, g.hh, k * sizeof(double), cudaMemcpyHostToDevice, h->stream), "GMRES update");
    VS_LAUNCH(h, "k_gm_combine", k_gm_combine<<<g.G, GM_THREADS, 0, h->stream>>>(g.Z, n, k, g.hd2, 1.0, g.z));
    VS_CK(h, cudaGetLastError(), "GMRES update");
    // the host buffer is reused by the next readback only after this copy has run
    VS_CK(h, cudaStreamSynchronize(h->stream), "GMRES update");
    if (done) break;
  }
  g.last_iters = iters;
  g.last_res = res / (bnorm > 0.0 ? bnorm : 1.0);
  g.total_iters += iters;
  if (res > target) {
    h->msg = "GMRES did not reach its tolerance within max_iter iterations";
    return VS_ERR_NOT_CONVERGED;
  }
  return VS_OK;
}

vs_status step_implicit(vs_suspension* h) {
  const Layout& L = h->L;
  const VesIndex vi = h->D.vi();
  const int s = 0;
  vs_status st;
  if ((st = gmres_alloc(h)) != VS_OK) return st;
  GmresState& g = h->gm;
  // geometry, centres and sources at X^n; every operator at X^n (Eq. time_step_sc1 discretises them there):
  // the FP64 self matrix for the products, and the preconditioner's factors (FP64 LU or FP32 inverses)
  if ((st = geometry(h, h->xy, true)) != VS_OK) return st;
  if ((st = build_operators(h, h->xy, s, nullptr)) != VS_OK) return st;
  if (mixed(h)) {
    VS_LAUNCH(h, "k_self_matrix", k_self_matrix<<<self_grid(L.nmax, L.M), 256, 0, h->stream>>>(
                                      vi, h->xy, h->B.sa, h->B.tx, h->B.ty, h->D.tab, h->p.mu, h->scratch, s, nullptr));
    if ((g.ainv = relax_matrix_32(h, s, nullptr)) < 0) return VS_ERR_CUDA;
  } else if ((st = relax_matrix_fp64(h, s)) != VS_OK) {
    return st;
  }
  VS_LAUNCH(h, "k_imp_rhs", k_imp_rhs<<<L.M, NMAX, 0, h->stream>>>(vi, h->xy, h->B.pg(), h->D.tab, flow_dev(h->flow),
                                                                   h->p.dt, g.b));
  VS_LAUNCH(h, "k_imp_pack", k_imp_pack<<<L.M, NMAX, 0, h->stream>>>(vi, h->xy, h->sigma, g.z));
  VS_CK(h, cudaGetLastError(), "implicit step");
  if ((st = gmres_solve(h, s)) != VS_OK) return st;
  // X^{n+1}, sigma^{n+1}; redistribution (sigma carried by the interpolant) and area/length correction
  VS_LAUNCH(h, "k_imp_unpack", k_imp_unpack<<<L.M, NMAX, 0, h->stream>>>(vi, g.z, h->xy_next, h->u));
  VS_LAUNCH(h, "k_redistribute", k_redistribute<<<L.M, 256, 0, h->stream>>>(vi, h->xy_next, h->u, h->D.tab, h->xy, h->u_r));
  VS_LAUNCH(h, "k_imp_sigma", k_imp_sigma<<<L.M, NMAX, 0, h->stream>>>(vi, h->u_r, h->sigma));
  VS_CK(h, cudaGetLastError(), "implicit step");
  if ((st = correction(h)) != VS_OK) return st;
  h->cur = 0;
  h->steps += 1;
  return VS_OK;
}

vs_status read_err(vs_suspension* h) {
  VS_CK(h, cudaStreamSynchronize(h->stream), "synchronize");
  unsigned e = 0;
  VS_CK(h, cudaMemcpy(&e, h->err, sizeof e, cudaMemcpyDeviceToHost), "error word");
  if (e & ERR_NONFINITE) { h->msg = "non-finite vesicle state"; return VS_ERR_UNSTABLE; }
  if (e & ERR_PIVOT) { h->msg = "singular per-vesicle system (zero pivot)"; return VS_ERR_UNSTABLE; }
  if (e & ERR_CORRECTION) { h->msg = "area/length correction did not converge"; return VS_ERR_NOT_CONVERGED; }
  if (e & ERR_REFINE) { h->msg = "mixed-precision refinement did not converge"; return VS_ERR_NOT_CONVERGED; }
  if (e & ERR_NEAR_OVERFLOW) { h->msg = "more near vesicles per target than recorded"; return VS_ERR_UNSTABLE; }
  return VS_OK;
}

void drop_graphs(vs_suspension* h) {
  for (int c = 0; c < 4; ++c)
    if (h->graph[c]) {
      cudaGraphExecDestroy(h->graph[c]);
      h->graph[c] = nullptr;
    }
}

// One step replayed from a CUDA graph captured on first use (per slot parity). The step's kernels
// read every per-step decision (dirty operator slots, near lists, correction triggers) from device
// flags, so the captured sequence is valid for every later step with the same parity.
vs_status step_graph(vs_suspension* h) {
  const int c = h->cur + (learned_step(h) ? 0 : 2);
  if (!h->graph[c]) {
    cudaGraph_t g = nullptr;
    VS_CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "graph capture");
    const int64_t l0 = h->launches, s0 = h->steps;
    const vs_status st = step_once(h);
    const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    h->graph_launches[c] = h->launches - l0;
    h->launches = l0;
    h->steps = s0;
    h->cur = c & 1;
    if (st != VS_OK) { if (g) cudaGraphDestroy(g); return st; }
    VS_CK(h, e, "graph capture");
    const cudaError_t ei = cudaGraphInstantiate(&h->graph[c], g, 0);
    cudaGraphDestroy(g);
    VS_CK(h, ei, "graph instantiate");
  }
  VS_CK(h, cudaGraphLaunch(h->graph[c], h->stream), "graph launch");
  h->cur = 1 - (c & 1);
  h->steps += 1;
  h->launches += h->graph_launches[c];
  return VS_OK;
}

bool params_ok(const vs_params* p, const vs_flow* f, std::string& msg) {
  if (!p || !f) { msg = "null params or flow"; return false; }
  if (!(p->kappa_b > 0) || !(p->mu > 0) || !(p->dt > 0) || !(p->corr_tol >= 0) || !std::isfinite(p->dt)) {
    msg = "kappa_b, mu, dt must be positive and corr_tol non-negative";
    return false;
  }
  if (p->mode < 0 || p->mode > 2) { msg = "mode must be 0 (plain), 1 (hybrid) or 2 (fully implicit)"; return false; }
  if (p->exact_every < 0) { msg = "exact_every must be >= 0"; return false; }
  if (!(p->exact_gap >= 0.0) || !std::isfinite(p->exact_gap)) { msg = "exact_gap must be finite and >= 0"; return false; }
  if (f->kind < 0 || f->kind > 3) { msg = "unknown flow kind"; return false; }
  if ((f->kind == 2 || f->kind == 3) && !(f->p[1] != 0.0)) { msg = "flow length scale p[1] must be non-zero"; return false; }
  return true;
}

void free_suspension(vs_suspension* h) {
  if (!h) return;
  h->D.release();
  h->B.release();
  cudaFree(h->xy); cudaFree(h->xy_star); cudaFree(h->xy_next); cudaFree(h->sigma); cudaFree(h->u);
  cudaFree(h->u_r); cudaFree(h->A0); cudaFree(h->L0); cudaFree(h->scratch); cudaFree(h->piv);
  cudaFree(h->scratch32); cudaFree(h->piv32);
  cudaFree(h->dirty); cudaFree(h->fired); cudaFree(h->err); cudaFree(h->has_near); cudaFree(h->involved); cudaFree(h->fb_acc);
  cudaFree(h->nb.layer); cudaFree(h->nb.phi); cudaFree(h->xin); cudaFree(h->frames);
  cudaFree(h->corr); cudaFree(h->cactive); cudaFree(h->cpiv);
  h->ffs.release();
  h->gm.release();
}

thread_local std::string g_create_msg;

}  // namespace

extern "C" {

vs_status vs_create(const double* xy, const int64_t* offsets, int32_t M, const vs_params* params,
                    const vs_flow* flow, void* cuda_stream, vs_suspension** out) {
  if (!out) return VS_ERR_INVALID_ARG;
  *out = nullptr;
  vs_suspension* h = new (std::nothrow) vs_suspension();
  if (!h) return VS_ERR_NOMEM;
  auto fail = [&](vs_status s) {
    g_create_msg = h->msg;
    free_suspension(h);
    delete h;
    return s;
  };
  if (!xy) { h->msg = "null xy"; return fail(VS_ERR_INVALID_ARG); }
  if (!params_ok(params, flow, h->msg)) return fail(VS_ERR_INVALID_ARG);
  if (!build_layout(offsets, M, h->L, h->msg)) return fail(VS_ERR_INVALID_ARG);
  if ((params->flags & VS_FLAG_FARFIELD_TREE) && M > TREE_MAX_M) {
    h->msg = "the cluster tree takes at most 16384 vesicles";
    return fail(VS_ERR_INVALID_ARG);
  }
  for (int64_t i = 0; i < 2 * h->L.P; ++i)
    if (!std::isfinite(xy[i])) { h->msg = "non-finite input point"; return fail(VS_ERR_INVALID_ARG); }
  h->p = *params;
  h->flow = *flow;
  h->stream = (cudaStream_t)cuda_stream;
  const Layout& L = h->L;
  cudaError_t e;
#define VS_A(x) do { e = (x); if (e != cudaSuccess) { cuda_fail(h->msg, e, "vs_create"); return fail(e == cudaErrorMemoryAllocation ? VS_ERR_NOMEM : VS_ERR_CUDA); } } while (0)
  VS_A(upload_layout(L, h->D, h->stream));
  VS_A(h->B.alloc(L.P, L.M));
  VS_A(dalloc(&h->xy, 2 * L.P)); VS_A(dalloc(&h->xy_star, 2 * L.P)); VS_A(dalloc(&h->xy_next, 2 * L.P));
  VS_A(dalloc(&h->sigma, L.P)); VS_A(dalloc(&h->u, 2 * L.P)); VS_A(dalloc(&h->u_r, 2 * L.P));
  VS_A(dalloc(&h->A0, L.M)); VS_A(dalloc(&h->L0, L.M));
  VS_A(dalloc(&h->scratch, L.moff[L.M])); VS_A(dalloc(&h->piv, 4 * L.P));
  VS_A(dalloc(&h->scratch32, L.moff[L.M])); VS_A(dalloc(&h->piv32, 4 * L.P));
  VS_A(dalloc(&h->dirty, L.M)); VS_A(dalloc(&h->fired, 1)); VS_A(dalloc(&h->err, 1));
  VS_A(dalloc(&h->has_near, L.M));
  VS_A(dalloc(&h->involved, L.M));
  VS_A(dalloc(&h->fb_acc, 2));
  VS_A(cudaFuncSetAttribute(k_lu_smem<LuGeo>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LU_SMEM_MAX));
  VS_A(cudaFuncSetAttribute(k_corr_newton<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LU_SMEM_MAX));
  VS_A(cudaFuncSetAttribute(k_corr_newton32<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 128 * 4));
  VS_A(cudaFuncSetAttribute(k_fused_tl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fz_tl_smem()));
  VS_A(cudaFuncSetAttribute(k_fused_relax, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fz_relax_smem()));
  VS_A(cudaFuncSetAttribute(k_bgemm_tc<OpT32>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  VS_A(cudaFuncSetAttribute(k_bgemm_tc<OpL32>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  VS_A(cudaFuncSetAttribute(k_bgemm_tc<OpD2_32>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  VS_A(cudaFuncSetAttribute(k_bgemm_tc<OpD4_32>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  VS_A(cudaFuncSetAttribute(k_bgemm_tc<OpB32>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  VS_A(cudaFuncSetAttribute(k_bgemm_tc<OpPB32>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  VS_A(cudaFuncSetAttribute(k_bgemm_tc<OpW32>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  VS_A(cudaFuncSetAttribute(k_bgemm_tc<OpA32>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  VS_A(cudaFuncSetAttribute(k_bgemm_tc<OpBlk32>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  VS_A(cudaFuncSetAttribute(k_ff_moments<FF_MP_P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)ffm_smem(FF_MP_P, NMAX)));
  if (h->p.flags & VS_FLAG_FARFIELD_TREE) {
    VS_A(h->B.alloc_tree(L.M));
    VS_A(cudaFuncSetAttribute(k_tree_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tree_build_smem(TREE_MAX_M)));
  }
  VS_A(dalloc(&h->corr, 6 * L.P + 16 * (int64_t)L.M));
  VS_A(dalloc(&h->cactive, L.M));
  VS_A(dalloc(&h->cpiv, 2 * L.P + 2 * (int64_t)L.M));
  VS_A(dalloc(&h->xin, (int64_t)std::max(2 * L.nmax, feat_width(feat_kmax(L.nmax, L.nmax))) * L.M));
  VS_A(dalloc(&h->frames, L.M));
  if (h->p.near_field) {
    VS_A(dalloc(&h->nb.layer, 30 * L.P));
    VS_A(dalloc(&h->nb.phi, L.moff[L.M]));
    VS_A(cudaFuncSetAttribute(k_near_layers<NEAR_EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)near_layers_smem(L.nmax)));
    VS_A(cudaFuncSetAttribute(k_near_layers<NEAR_LEARNED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)near_layers_smem(L.nmax)));
    VS_A(cudaFuncSetAttribute(k_near_layers<NEAR_YZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)near_layers_smem(L.nmax)));
    if (5 * L.nmax <= NEAR_RBF_SMEM_N)
      VS_A(cudaFuncSetAttribute(k_near_rbf_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)near_rbf_smem(5 * L.nmax)));
  }
  VS_A(cudaMemsetAsync(h->fired, 0, sizeof(int), h->stream));
  VS_A(cudaMemsetAsync(h->fb_acc, 0, 2 * sizeof(unsigned long long), h->stream));
  VS_A(cudaMemsetAsync(h->err, 0, sizeof(unsigned), h->stream));
  VS_A(cudaMemsetAsync(h->sigma, 0, L.P * sizeof(double), h->stream));
  VS_A(cudaMemsetAsync(h->u, 0, 2 * L.P * sizeof(double), h->stream));
  VS_A(cudaMemsetAsync(h->B.near_cnt, 0, L.P * sizeof(int), h->stream));
  VS_A(upload(h->xy_next, xy, 2 * L.P, h->stream));
  {
    std::vector<int> ones(L.M, 0);
    VS_A(upload(h->dirty, ones.data(), L.M, h->stream));
    VS_A(cudaStreamSynchronize(h->stream));
  }
  const VesIndex vi = h->D.vi();
  // redistribute X^0, record A_0 and L_0, initial tension from self + background terms
  VS_LAUNCH(h, "k_redistribute", k_redistribute<<<L.M, 256, 0, h->stream>>>(vi, h->xy_next, h->u, h->D.tab, h->xy, h->u_r));
  VS_A(cudaGetLastError());
  if (geometry(h, h->xy, true) != VS_OK) return fail(VS_ERR_CUDA);
  VS_A(cudaMemcpyAsync(h->A0, h->B.area, L.M * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  VS_A(cudaMemcpyAsync(h->L0, h->B.length, L.M * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  if (build_operators(h, h->xy, 0, nullptr) != VS_OK) return fail(VS_ERR_CUDA);
  if (tension(h, h->u, 0) != VS_OK) return fail(VS_ERR_CUDA);
  VS_A(cudaGetLastError());
  VS_A(ffs_setup(h->ffs, L, !(h->p.flags & (VS_FLAG_FARFIELD_FP64 | VS_FLAG_FARFIELD_MULTIPOLE |
                                            VS_FLAG_FARFIELD_PER_TARGET)), h->stream));
  if (tune_far_field(h) != VS_OK) return fail(VS_ERR_CUDA);
  if (geometry(h, h->xy, true) != VS_OK) return fail(VS_ERR_CUDA);  // u back to u_inf after tuning
  h->cur = 0;
  VS_A(cudaStreamSynchronize(h->stream));
#undef VS_A
  const vs_status st = read_err(h);
  if (st != VS_OK) return fail(st);
  *out = h;
  return VS_OK;
}

vs_status vs_step(vs_suspension* h, int32_t nsteps) {
  if (!h || nsteps < 0) return VS_ERR_INVALID_ARG;
  // the implicit step reads GMRES's residual on the host every iteration: never captured in a graph
  const bool implicit = h->p.mode == 2;
  const bool graphs = !implicit && h->p.use_graph && h->stream != nullptr && !h->prof.on;
  for (int32_t k = 0; k < nsteps; ++k) {
    const bool learned = learned_step(h);
    const vs_status st = implicit ? step_implicit(h) : graphs ? step_graph(h) : step_once(h);
    if (st != VS_OK) return st;
    h->learned_steps += learned;
  }
  return VS_OK;
}

vs_status vs_set_gmres(vs_suspension* h, double tol, int32_t restart, int32_t max_iter) {
  if (!h) return VS_ERR_INVALID_ARG;
  if (!(tol > 0.0) || !std::isfinite(tol) || restart < 1 || restart > VS_GMRES_MAX_RESTART || max_iter < 1) {
    h->msg = "GMRES needs tol > 0, 1 <= restart <= VS_GMRES_MAX_RESTART and max_iter >= 1";
    return VS_ERR_INVALID_ARG;
  }
  h->gm.tol = tol;
  h->gm.restart = restart;
  h->gm.max_iter = max_iter;
  return VS_OK;
}

vs_status vs_gmres_stats(const vs_suspension* h, int32_t* last_iters, double* last_residual, int64_t* total_iters) {
  if (!h) return VS_ERR_INVALID_ARG;
  if (last_iters) *last_iters = h->gm.last_iters;
  if (last_residual) *last_residual = h->gm.last_res;
  if (total_iters) *total_iters = h->gm.total_iters;
  return VS_OK;
}

vs_status vs_sync(vs_suspension* h) {
  if (!h) return VS_ERR_INVALID_ARG;
  return read_err(h);
}

vs_status vs_set_state(vs_suspension* h, const double* xy, const double* sigma) {
  if (!h || !xy || !sigma) return VS_ERR_INVALID_ARG;
  const Layout& L = h->L;
  // staged in xy_star (free between steps); only vesicles whose points changed lose their cached operators
  VS_CK(h, upload(h->xy_star, xy, 2 * L.P, h->stream), "set_state");
  VS_CK(h, upload(h->sigma, sigma, L.P, h->stream), "set_state");
  VS_LAUNCH(h, "k_state_update", k_state_update<<<L.M, NMAX, 0, h->stream>>>(h->D.vi(), h->xy_star, h->xy, h->dirty));
  VS_CK(h, cudaGetLastError(), "set_state");
  VS_CK(h, cudaStreamSynchronize(h->stream), "set_state");
  return VS_OK;
}

static vs_status copy_out(vs_suspension* h, const double* src, int64_t n, double* dst, int64_t cap) {
  if (!h || !dst) return VS_ERR_INVALID_ARG;
  if (cap < n) { h->msg = "output buffer too small"; return VS_ERR_INVALID_ARG; }
  const vs_status st = read_err(h);
  VS_CK(h, cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy out");
  VS_CK(h, cudaStreamSynchronize(h->stream), "copy out");
  return st;
}

vs_status vs_get_positions(vs_suspension* h, double* xy, int64_t cap) {
  return h ? copy_out(h, h->xy, 2 * h->L.P, xy, cap) : VS_ERR_INVALID_ARG;
}
vs_status vs_get_tension(vs_suspension* h, double* sigma, int64_t cap) {
  return h ? copy_out(h, h->sigma, h->L.P, sigma, cap) : VS_ERR_INVALID_ARG;
}
vs_status vs_get_velocity(vs_suspension* h, double* u, int64_t cap) {
  return h ? copy_out(h, h->u, 2 * h->L.P, u, cap) : VS_ERR_INVALID_ARG;
}
vs_status vs_get_reference(vs_suspension* h, double* a0l0, int64_t cap) {
  if (!h || !a0l0) return VS_ERR_INVALID_ARG;
  if (cap < 2 * h->L.M) { h->msg = "output buffer too small"; return VS_ERR_INVALID_ARG; }
  VS_CK(h, cudaStreamSynchronize(h->stream), "reference");
  VS_CK(h, cudaMemcpy(a0l0, h->A0, h->L.M * sizeof(double), cudaMemcpyDeviceToHost), "reference");
  VS_CK(h, cudaMemcpy(a0l0 + h->L.M, h->L0, h->L.M * sizeof(double), cudaMemcpyDeviceToHost), "reference");
  return VS_OK;
}

vs_status vs_get_device_ptrs(const vs_suspension* h, const double** xy, const double** sigma) {
  if (!h || !xy || !sigma) return VS_ERR_INVALID_ARG;
  *xy = h->xy;
  *sigma = h->sigma;
  return VS_OK;
}

// Checkpoint format (little-endian host memory): CkptHeader, then xy (2P), sigma (P), A_0 (M), L_0 (M)
// as doubles.
struct CkptHeader {
  char magic[8];       // "VSCKPT\0\1"
  int64_t M, P;
  uint64_t layout;     // FNV-1a hash of the point counts
  int64_t steps;
  int32_t fired, mode;
  double kappa_b, mu, dt;
};
constexpr char CKPT_MAGIC[8] = {'V', 'S', 'C', 'K', 'P', 'T', 0, 1};

uint64_t layout_hash(const Layout& L) {
  uint64_t x = 1469598103934665603ull;
  for (int32_t n : L.N) {
    x ^= (uint64_t)(uint32_t)n;
    x *= 1099511628211ull;
  }
  return x;
}

int64_t ckpt_bytes(const Layout& L) { return (int64_t)sizeof(CkptHeader) + (3 * L.P + 2 * (int64_t)L.M) * 8; }

vs_status vs_get_counters(vs_suspension* h, int64_t* out4) {
  if (!h || !out4) return VS_ERR_INVALID_ARG;
  prof_collect(h);
  VS_CK(h, cudaStreamSynchronize(h->stream), "counters");
  int fired = 0;
  unsigned e = 0;
  VS_CK(h, cudaMemcpy(&fired, h->fired, sizeof fired, cudaMemcpyDeviceToHost), "counters");
  VS_CK(h, cudaMemcpy(&e, h->err, sizeof e, cudaMemcpyDeviceToHost), "counters");
  std::vector<int> nc(h->L.P);
  VS_CK(h, cudaMemcpy(nc.data(), h->B.near_cnt, h->L.P * sizeof(int), cudaMemcpyDeviceToHost), "counters");
  int64_t pairs = 0;
  for (int c : nc) pairs += c;
  out4[0] = h->steps;
  out4[1] = fired;
  out4[2] = pairs;
  out4[3] = e;
  out4[4] = h->launches;
  return VS_OK;
}

vs_status vs_get_hybrid_counters(vs_suspension* h, int64_t* out3) {
  if (!h || !out3) return VS_ERR_INVALID_ARG;
  VS_CK(h, cudaStreamSynchronize(h->stream), "hybrid counters");
  unsigned long long acc[2] = {0ull, 0ull};
  VS_CK(h, cudaMemcpy(acc, h->fb_acc, sizeof acc, cudaMemcpyDeviceToHost), "hybrid counters");
  out3[0] = h->learned_steps;
  out3[1] = (int64_t)acc[1];
  out3[2] = (int64_t)acc[0];
  return VS_OK;
}

vs_status vs_farfield_variant(vs_suspension* h, int32_t set, int32_t* index, int32_t* threads, int32_t* chunk) {
  if (!h || set >= FF_NVARIANTS) return VS_ERR_INVALID_ARG;
  if (set >= 0 && (set != h->ff_variant || h->ffs.on)) {
    h->ff_variant = set;
    h->ffs.on = false;  // an explicit per-target launch shape leaves the symmetric kernel
    drop_graphs(h);
  }
  if (h->ffs.on) {
    if (index) *index = -1;
    if (threads) *threads = 32 * FFS_W;
    if (chunk) *chunk = h->ffs.V * h->L.nmax;
    return VS_OK;
  }
  if (index) *index = h->ff_variant;
  if (threads) *threads = FF_VARIANTS[h->ff_variant].threads;
  if (chunk) *chunk = FF_VARIANTS[h->ff_variant].chunk;
  return VS_OK;
}

vs_status vs_profile(vs_suspension* h, int32_t enable) {
  if (!h) return VS_ERR_INVALID_ARG;
  prof_collect(h);
  h->prof.on = enable != 0;
  std::fill(h->prof.total_ms.begin(), h->prof.total_ms.end(), 0.0);
  std::fill(h->prof.count.begin(), h->prof.count.end(), 0);
  return VS_OK;
}

vs_status vs_profile_read(vs_suspension* h, int32_t idx, char* name, int32_t name_cap, double* total_ms,
                          int64_t* launches) {
  if (!h || !name || name_cap < 1 || !total_ms || !launches) return VS_ERR_INVALID_ARG;
  prof_collect(h);
  if (idx < 0 || idx >= (int32_t)h->prof.names.size()) return VS_ERR_INVALID_ARG;
  snprintf(name, (size_t)name_cap, "%s", h->prof.names[idx].c_str());
  *total_ms = h->prof.total_ms[idx];
  *launches = h->prof.count[idx];
  return VS_OK;
}


vs_status vs_set_network(vs_suspension* h, int32_t which, vs_mlp* net, double out_scale, int32_t filter_kmax) {
  if (!h || which != 0) return VS_ERR_INVALID_ARG;
  if (!net) { drop_graphs(h); h->net = nullptr; return VS_OK; }
  const Layout& L = h->L;
  for (int v = 0; v < L.M; ++v)
    if (L.N[v] != L.nmax) { h->msg = "the learned relaxation needs one point count for all vesicles"; return VS_ERR_INVALID_ARG; }
  if (!(out_scale > 0) || filter_kmax < 0) return VS_ERR_INVALID_ARG;
  const int W = feat_width(feat_kmax(filter_kmax, L.nmax));
  if (net->dims.front() != W || net->dims.back() != W || net->Bcap < L.M) {
    h->msg = "network widths must be the feature width 16 ceil((4K + 2)/16), K = min(filter_kmax, N/2 - 1), in "
             "and out, and its batch capacity at least M";
    return VS_ERR_INVALID_ARG;
  }
  if (net->stream != h->stream) { h->msg = "network and suspension must share one stream"; return VS_ERR_INVALID_ARG; }
  drop_graphs(h);
  h->net = net;
  h->net_scale = out_scale;
  h->net_kmax = filter_kmax;
  return VS_OK;
}

vs_status vs_set_flow_networks(vs_suspension* h, vs_mlp* adv, vs_mlp* ten, int32_t Kf, int32_t Kout) {
  if (!h || (!adv) != (!ten)) return VS_ERR_INVALID_ARG;
  const Layout& L = h->L;
  if (!adv) {
    drop_graphs(h);
    h->flow_adv = h->flow_ten = nullptr;
    std::vector<int> ones(L.M, 1);  // the operator cache at X^n was not kept while the networks were in use
    VS_CK(h, cudaMemcpy(h->dirty, ones.data(), L.M * sizeof(int), cudaMemcpyHostToDevice), "flow networks");
    return VS_OK;
  }
  if (!h->net) { h->msg = "set the relaxation network (vs_set_network) first: the flow networks share its input"; return VS_ERR_INVALID_ARG; }
  if (Kf < 0 || Kout < 0 || Kf > L.nmax / 2 - 1 || Kout > L.nmax / 2 - 1) {
    h->msg = "Kf and Kout must be in [0, N/2 - 1]";
    return VS_ERR_INVALID_ARG;
  }
  const int W = feat_width(feat_kmax(h->net_kmax, L.nmax));
  if (adv->dims.front() != W || ten->dims.front() != W || adv->dims.back() != flow_adv_width(Kf, Kout) ||
      ten->dims.back() != flow_ten_width(Kf, Kout) || adv->Bcap < L.M || ten->Bcap < L.M) {
    h->msg = "flow networks: input width that of the relaxation network, outputs flow_adv_width(Kf, Kout) and "
             "flow_ten_width(Kf, Kout), batch capacity at least M";
    return VS_ERR_INVALID_ARG;
  }
  if (adv->stream != h->stream || ten->stream != h->stream) {
    h->msg = "networks and suspension must share one stream";
    return VS_ERR_INVALID_ARG;
  }
  drop_graphs(h);
  h->flow_adv = adv;
  h->flow_ten = ten;
  h->flow_kf = Kf;
  h->flow_kout = Kout;
  return VS_OK;
}

vs_status vs_flow_maps(vs_suspension* h, int32_t Kf, int32_t Kout, int32_t filter_kmax, float* xin, float* adv,
                       float* ten) {
  if (!h || !xin || !adv || !ten || filter_kmax < 0) return VS_ERR_INVALID_ARG;
  const Layout& L = h->L;
  for (int v = 0; v < L.M; ++v)
    if (L.N[v] != L.nmax) { h->msg = "vs_flow_maps needs one point count for all vesicles"; return VS_ERR_INVALID_ARG; }
  if (Kf < 0 || Kout < 0 || Kf > L.nmax / 2 - 1 || Kout > L.nmax / 2 - 1) return VS_ERR_INVALID_ARG;
  const VesIndex vi = h->D.vi();
  const int M = L.M, nxt = 1 - h->cur;
  const int W = feat_width(feat_kmax(filter_kmax, L.nmax));
  const int la = flow_adv_width(Kf, Kout), lt = flow_ten_width(Kf, Kout);
  const int ca = flow_col_adv(Kout), ct = flow_col_ten(Kout);
  // inputs and frames at the current points, the standardised points into xy_next
  VS_LAUNCH(h, "k_standardize", k_standardize<<<M, NMAX, 0, h->stream>>>(vi, h->xy, h->D.tab, xin, W, h->frames,
                                                                         filter_kmax, true));
  VS_LAUNCH(h, "k_standard_points", k_standard_points<<<M, NMAX, 0, h->stream>>>(vi, h->xy, h->frames, h->xy_next));
  VS_CK(h, cudaMemsetAsync(adv, 0, (size_t)M * la * sizeof(float), h->stream), "flow maps");
  VS_CK(h, cudaMemsetAsync(ten, 0, (size_t)M * lt * sizeof(float), h->stream), "flow maps");
  // the exact operators at the standardised shapes in slot nxt (the cache of slot cur is left alone)
  vs_status st;
  if ((st = geometry(h, h->xy_next, false)) != VS_OK) return st;
  if ((st = build_operators(h, h->xy_next, nxt, nullptr)) != VS_OK) return st;
  double *zero = nullptr, *ub = nullptr, *out = nullptr, *s0 = nullptr, *sb = nullptr;
  cudaError_t e = dalloc(&zero, 2 * L.P);
  if (e == cudaSuccess) e = dalloc(&ub, 2 * L.P);
  if (e == cudaSuccess) e = dalloc(&out, 2 * L.P);
  if (e == cudaSuccess) e = dalloc(&s0, L.P);
  if (e == cudaSuccess) e = dalloc(&sb, L.P);
  if (e == cudaSuccess) e = cudaMemsetAsync(zero, 0, 2 * L.P * sizeof(double), h->stream);
  auto done = [&](vs_status r) {
    cudaStreamSynchronize(h->stream);
    cudaFree(zero); cudaFree(ub); cudaFree(out); cudaFree(s0); cudaFree(sb);
    return r;
  };
  if (e != cudaSuccess) { cuda_fail(h->msg, e, "vs_flow_maps"); return done(VS_ERR_NOMEM); }
  // S_sigma = L^{-1} P B X = -sigma(u = 0)
  if ((st = tension_into(h, zero, nxt, s0)) != VS_OK) return done(st);
  k_field_features<<<M, NMAX, 0, h->stream>>>(vi, s0, 1, h->D.tab, Kout, -1.0, false, ten, lt, 0);
  for (int b = 0; b < flow_basis(Kf); ++b) {
    k_basis_velocity<<<M, NMAX, 0, h->stream>>>(vi, h->D.tab, b, Kf, ub);
    // (I - M) psi_b
    if ((st = advect_into(h, zero, ub, nxt, 1.0, out)) != VS_OK) return done(st);
    k_field_features<<<M, NMAX, 0, h->stream>>>(vi, out, 2, h->D.tab, Kout, 1.0, false, adv, la, b * ca);
    // L^{-1} P psi_b = sigma(0) - sigma(psi_b)
    if ((st = tension_into(h, ub, nxt, sb)) != VS_OK) return done(st);
    k_field_features<<<M, NMAX, 0, h->stream>>>(vi, s0, 1, h->D.tab, Kout, 1.0, false, ten, lt, (b + 1) * ct);
    k_field_features<<<M, NMAX, 0, h->stream>>>(vi, sb, 1, h->D.tab, Kout, -1.0, true, ten, lt, (b + 1) * ct);
  }
  VS_CK(h, cudaGetLastError(), "flow maps");
  return done(VS_OK);
}

vs_status vs_set_near_networks(vs_suspension* h, vs_mlp* const* nets, int32_t n, int32_t Kf, int32_t Kout) {
  if (!h) return VS_ERR_INVALID_ARG;
  const Layout& L = h->L;
  if (!nets) {
    drop_graphs(h);
    for (auto& p : h->near_net) p = nullptr;
    return VS_OK;
  }
  if (n != NEAR_LAYERS) { h->msg = "the near field takes one network per layer (5)"; return VS_ERR_INVALID_ARG; }
  if (!h->p.near_field || !h->nb.layer) {
    h->msg = "near-field networks need a suspension created with near_field = 1";
    return VS_ERR_INVALID_ARG;
  }
  if (!h->net) { h->msg = "set the relaxation network (vs_set_network) first: the near-field networks share its input"; return VS_ERR_INVALID_ARG; }
  if (Kf < 0 || Kout < 0 || Kf > L.nmax / 2 - 1 || Kout > L.nmax / 2 - 1) {
    h->msg = "Kf and Kout must be in [0, N/2 - 1]";
    return VS_ERR_INVALID_ARG;
  }
  const int W = feat_width(feat_kmax(h->net_kmax, L.nmax));
  for (int d = 0; d < NEAR_LAYERS; ++d) {
    const vs_mlp* m = nets[d];
    if (!m || m->dims.front() != W || m->dims.back() != flow_adv_width(Kf, Kout) || m->Bcap < L.M) {
      h->msg = "near-field networks: input width that of the relaxation network, output flow_adv_width(Kf, Kout), "
               "batch capacity at least M";
      return VS_ERR_INVALID_ARG;
    }
    if (m->stream != h->stream) { h->msg = "networks and suspension must share one stream"; return VS_ERR_INVALID_ARG; }
  }
  drop_graphs(h);
  for (int d = 0; d < NEAR_LAYERS; ++d) h->near_net[d] = nets[d];
  h->near_kf = Kf;
  h->near_kout = Kout;
  return VS_OK;
}

vs_status vs_near_maps(vs_suspension* h, int32_t Kf, int32_t Kout, int32_t filter_kmax, float* xin, float* out) {
  if (!h || !xin || !out || filter_kmax < 0) return VS_ERR_INVALID_ARG;
  const Layout& L = h->L;
  for (int v = 0; v < L.M; ++v)
    if (L.N[v] != L.nmax) { h->msg = "vs_near_maps needs one point count for all vesicles"; return VS_ERR_INVALID_ARG; }
  if (Kf < 0 || Kout < 0 || Kf > L.nmax / 2 - 1 || Kout > L.nmax / 2 - 1) return VS_ERR_INVALID_ARG;
  const VesIndex vi = h->D.vi();
  const int M = L.M, nxt = 1 - h->cur;
  const int W = feat_width(feat_kmax(filter_kmax, L.nmax));
  const int width = flow_adv_width(Kf, Kout), cw = flow_col_adv(Kout);
  // inputs and frames at the current points, the standardised points into xy_next
  VS_LAUNCH(h, "k_standardize", k_standardize<<<M, NMAX, 0, h->stream>>>(vi, h->xy, h->D.tab, xin, W, h->frames,
                                                                         filter_kmax, true));
  VS_LAUNCH(h, "k_standard_points", k_standard_points<<<M, NMAX, 0, h->stream>>>(vi, h->xy, h->frames, h->xy_next));
  VS_CK(h, cudaMemsetAsync(out, 0, (size_t)NEAR_LAYERS * M * width * sizeof(float), h->stream), "near maps");
  // the self matrix at the standardised shapes in slot nxt (the cache of slot cur is left alone), with mu = 1
  // as the columns are defined
  vs_status st;
  const double mu = h->p.mu;
  h->p.mu = 1.0;
  st = geometry(h, h->xy_next, false);
  if (st == VS_OK) st = build_operators(h, h->xy_next, nxt, nullptr);
  h->p.mu = mu;
  if (st != VS_OK) return st;
  double *psi = nullptr, *layer = nullptr;
  int* ones = nullptr;
  cudaError_t e = dalloc(&psi, 2 * L.P);
  if (e == cudaSuccess) e = dalloc(&layer, 30 * L.P);
  if (e == cudaSuccess) e = dalloc(&ones, M);
  if (e == cudaSuccess) {
    std::vector<int> one(M, 1);
    e = cudaMemcpyAsync(ones, one.data(), M * sizeof(int), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  const size_t smem = near_layers_smem(L.nmax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_near_layers<NEAR_EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  auto done = [&](vs_status r) {
    cudaStreamSynchronize(h->stream);
    cudaFree(psi); cudaFree(layer); cudaFree(ones);
    return r;
  };
  if (e != cudaSuccess) { cuda_fail(h->msg, e, "vs_near_maps"); return done(VS_ERR_NOMEM); }
  const NearBufs nbuf{layer, nullptr};
  for (int b = 0; b < flow_basis(Kf); ++b) {
    k_basis_velocity<<<M, NMAX, 0, h->stream>>>(vi, h->D.tab, b, Kf, psi);
    // the layer velocities of psi_b at the standardised shape, mu = 1
    k_near_layers<NEAR_EXACT><<<M, 256, smem, h->stream>>>(vi, ones, h->xy_next, psi, h->B.pg(), h->B.length, h->D.tab,
                                                      h->scratch, mixed(h) ? h->scratch32 : nullptr, nxt, 1.0, nbuf,
                                                      NearNets{});
    for (int d = 0; d < NEAR_LAYERS; ++d)
      k_layer_features<<<M, NMAX, 0, h->stream>>>(vi, ones, layer, d, h->D.tab, Kout, out + (int64_t)d * M * width,
                                                  width, b * cw);
  }
  VS_CK(h, cudaGetLastError(), "near maps");
  return done(VS_OK);
}

vs_status vs_relax(vs_suspension* h, const double* xy_in, double* xy_out) {
  if (!h || !xy_in || !xy_out || xy_in == xy_out) return VS_ERR_INVALID_ARG;
  return relax_exact(h, xy_in, xy_out, 1 - h->cur);
}


vs_status vs_training_pairs(vs_suspension* h, const double* xy_in, float* xin, float* yout, double out_scale,
                            int32_t kmax) {
  if (!h || !xy_in || !xin || !yout || !(out_scale > 0) || kmax < 0) return VS_ERR_INVALID_ARG;
  const Layout& L = h->L;
  for (int v = 0; v < L.M; ++v)
    if (L.N[v] != L.nmax) { h->msg = "training pairs need one point count for all vesicles"; return VS_ERR_INVALID_ARG; }
  const VesIndex vi = h->D.vi();
  vs_status st = relax_exact(h, xy_in, h->xy_next, 1 - h->cur);
  if (st != VS_OK) return st;
  const int W = feat_width(feat_kmax(kmax, L.nmax));
  VS_LAUNCH(h, "k_standardize", k_standardize<<<L.M, NMAX, 0, h->stream>>>(vi, xy_in, h->D.tab, xin, W, h->frames, kmax,
                                                                           true));
  VS_LAUNCH(h, "k_to_frame_rows", k_to_frame_rows<<<L.M, NMAX, 0, h->stream>>>(vi, xy_in, h->xy_next, h->frames,
                                                                             1.0 / out_scale, h->D.tab, kmax, yout, W));
  VS_CK(h, cudaGetLastError(), "training pairs");
  return VS_OK;
}

vs_status vs_checkpoint_size(vs_suspension* h, int64_t* bytes) {
  if (!h || !bytes) return VS_ERR_INVALID_ARG;
  *bytes = ckpt_bytes(h->L);
  return VS_OK;
}

vs_status vs_checkpoint(vs_suspension* h, void* buf, int64_t cap) {
  if (!h || !buf) return VS_ERR_INVALID_ARG;
  const Layout& L = h->L;
  if (cap < ckpt_bytes(L)) { h->msg = "checkpoint buffer too small"; return VS_ERR_INVALID_ARG; }
  const vs_status st = read_err(h);
  if (st != VS_OK) return st;
  int fired = 0;
  VS_CK(h, cudaMemcpy(&fired, h->fired, sizeof fired, cudaMemcpyDeviceToHost), "checkpoint");
  CkptHeader hd{};
  std::memcpy(hd.magic, CKPT_MAGIC, 8);
  hd.M = L.M;
  hd.P = L.P;
  hd.layout = layout_hash(L);
  hd.steps = h->steps;
  hd.fired = fired;
  hd.mode = h->p.mode;
  hd.kappa_b = h->p.kappa_b;
  hd.mu = h->p.mu;
  hd.dt = h->p.dt;
  unsigned char* b = static_cast<unsigned char*>(buf);
  std::memcpy(b, &hd, sizeof hd);
  double* d = reinterpret_cast<double*>(b + sizeof hd);
  VS_CK(h, cudaMemcpy(d, h->xy, 2 * L.P * sizeof(double), cudaMemcpyDeviceToHost), "checkpoint");
  VS_CK(h, cudaMemcpy(d + 2 * L.P, h->sigma, L.P * sizeof(double), cudaMemcpyDeviceToHost), "checkpoint");
  VS_CK(h, cudaMemcpy(d + 3 * L.P, h->A0, L.M * sizeof(double), cudaMemcpyDeviceToHost), "checkpoint");
  VS_CK(h, cudaMemcpy(d + 3 * L.P + L.M, h->L0, L.M * sizeof(double), cudaMemcpyDeviceToHost), "checkpoint");
  return VS_OK;
}

vs_status vs_restore(vs_suspension* h, const void* buf, int64_t size) {
  if (!h || !buf) return VS_ERR_INVALID_ARG;
  const Layout& L = h->L;
  CkptHeader hd;
  if (size < (int64_t)sizeof hd) { h->msg = "checkpoint too short"; return VS_ERR_INVALID_ARG; }
  std::memcpy(&hd, buf, sizeof hd);
  if (std::memcmp(hd.magic, CKPT_MAGIC, 8) != 0) { h->msg = "not a checkpoint of this format"; return VS_ERR_INVALID_ARG; }
  if (hd.M != L.M || hd.P != L.P || hd.layout != layout_hash(L) || size < ckpt_bytes(L)) {
    h->msg = "checkpoint of a suspension with other point counts";
    return VS_ERR_INVALID_ARG;
  }
  if (hd.kappa_b != h->p.kappa_b || hd.mu != h->p.mu || hd.dt != h->p.dt || hd.mode != h->p.mode) {
    h->msg = "checkpoint of a suspension with other parameters (kappa_b, mu, dt, mode)";
    return VS_ERR_INVALID_ARG;
  }
  const double* d = reinterpret_cast<const double*>(static_cast<const unsigned char*>(buf) + sizeof hd);
  VS_CK(h, cudaStreamSynchronize(h->stream), "restore");
  VS_CK(h, cudaMemcpy(h->xy, d, 2 * L.P * sizeof(double), cudaMemcpyHostToDevice), "restore");
  VS_CK(h, cudaMemcpy(h->sigma, d + 2 * L.P, L.P * sizeof(double), cudaMemcpyHostToDevice), "restore");
  VS_CK(h, cudaMemcpy(h->A0, d + 3 * L.P, L.M * sizeof(double), cudaMemcpyHostToDevice), "restore");
  VS_CK(h, cudaMemcpy(h->L0, d + 3 * L.P + L.M, L.M * sizeof(double), cudaMemcpyHostToDevice), "restore");
  VS_CK(h, cudaMemcpy(h->fired, &hd.fired, sizeof hd.fired, cudaMemcpyHostToDevice), "restore");
  std::vector<int> ones(L.M, 1);  // every cached operator is rebuilt from the restored points
  VS_CK(h, cudaMemcpy(h->dirty, ones.data(), L.M * sizeof(int), cudaMemcpyHostToDevice), "restore");
  h->steps = hd.steps;
  return VS_OK;
}

const char* vs_last_error(const vs_suspension* h) { return h ? h->msg.c_str() : g_create_msg.c_str(); }

void vs_destroy(vs_suspension* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  for (cudaEvent_t e : h->prof.pool) cudaEventDestroy(e);
  free_suspension(h);
  delete h;
}

// ---------------------------------------------------------------------------------------------
vs_status vs_farfield_plan_create(const int64_t* offsets, int32_t M, double mu, int32_t near_mask,
                                  int32_t precision, void* cuda_stream, vs_farfield_plan** out) {
  if (!out) return VS_ERR_INVALID_ARG;
  *out = nullptr;
  vs_farfield_plan* h = new (std::nothrow) vs_farfield_plan();
  if (!h) return VS_ERR_NOMEM;
  auto fail = [&](vs_status s) {
    g_create_msg = h->msg;
    h->D.release();
    h->B.release();
    h->ffs.release();
    cudaFree(h->err);
    delete h;
    return s;
  };
  if (!(mu > 0) || precision < 0 || precision > 4) { h->msg = "mu must be > 0, precision 0 to 4"; return fail(VS_ERR_INVALID_ARG); }
  if (precision == 4 && M > TREE_MAX_M) { h->msg = "the cluster tree takes at most 16384 vesicles"; return fail(VS_ERR_INVALID_ARG); }
  if (!build_layout(offsets, M, h->L, h->msg)) return fail(VS_ERR_INVALID_ARG);
  h->mu = mu;
  h->near_mask = near_mask ? 1 : 0;
  h->precision = precision;
  h->stream = (cudaStream_t)cuda_stream;
  cudaError_t e;
  if ((e = upload_layout(h->L, h->D, h->stream)) != cudaSuccess ||
      (e = h->B.alloc(h->L.P, h->L.M)) != cudaSuccess || (e = dalloc(&h->err, 1)) != cudaSuccess ||
      (e = cudaMemset(h->err, 0, sizeof(unsigned))) != cudaSuccess ||
      (e = cudaMemset(h->B.near_cnt, 0, h->L.P * sizeof(int))) != cudaSuccess ||
      (e = ffs_setup(h->ffs, h->L, precision == 0, h->stream)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_ff_moments<FF_MP_P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ffm_smem(FF_MP_P, NMAX))) != cudaSuccess ||
      (precision == 4 && (e = h->B.alloc_tree(h->L.M)) != cudaSuccess) ||
      (precision == 4 && (e = cudaFuncSetAttribute(k_tree_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)tree_build_smem(TREE_MAX_M))) != cudaSuccess)) {
    cuda_fail(h->msg, e, "vs_farfield_plan_create");
    return fail(e == cudaErrorMemoryAllocation ? VS_ERR_NOMEM : VS_ERR_CUDA);
  }
  *out = h;
  return VS_OK;
}

vs_status vs_farfield_eval(vs_farfield_plan* h, const double* xy, const double* f, double* u) {
  if (!h || !xy || !f || !u) return VS_ERR_INVALID_ARG;
  const Layout& L = h->L;
  ForceOut fo{h->B.f, u, h->B.src, h->B.centre, h->B.centre32, h->B.h2, h->B.g64, h->B.gsum};
  FlowDev none{0, 0.0, 0.0};
  launch_geometry(L.M, L.nmax, h->stream, h->D.vi(), xy, nullptr, h->D.tab, 1.0, h->mu, none, h->B.geom(), fo, f);
  VS_CK(h, cudaGetLastError(), "far-field sources");
  if (L.M < 2) return VS_OK;
  FarFieldArgs a{L.P, L.M, h->D.owner, h->D.off, h->D.chunk, (int)L.chunk.size() - 1, h->near_mask, u,
                 h->B.near_cnt, h->B.near_v, h->err};
  const int grid = (int)((L.P + FF_THREADS - 1) / FF_THREADS);
  if (h->precision == 1) {
    k_farfield_f64<<<grid, FF_THREADS, 0, h->stream>>>(a, xy, h->B.g64, h->B.length, h->D.N);
  } else if (h->precision == 4) {
    const int mt = ff_moment_threads(L);
    const FfTreeArgs t = h->B.tree(L.M);
    k_ff_moments<FF_MP_P><<<L.M, mt, ffm_smem(FF_MP_P, mt), h->stream>>>(h->D.off, h->B.src, h->B.mpcoef, h->B.mpa0,
                                                                        h->B.vraw);
    k_tree_build<<<1, TREE_THREADS, tree_build_smem(L.M), h->stream>>>(t);
    k_tree_moments<<<tree_moment_grid(L.M), TM_THREADS, 0, h->stream>>>(t, 0, 1);
    for (int l = TREE_LMAX - 1; l >= 0; --l) k_tree_moments<<<tree_moment_grid(L.M), TM_THREADS, 0, h->stream>>>(t, l, 0);
    const FfLocArgs la = h->B.loc(L.M);
    k_ff_local_tree<FF_MP_P><<<L.M, 128, 0, h->stream>>>(la, t);
    k_farfield_loc<FF_MP_P><<<L.M, 128, 0, h->stream>>>(a, la, h->B.src);
  } else if (h->precision == 2) {
    const int mt = ff_moment_threads(L);
    k_ff_moments<FF_MP_P><<<L.M, mt, ffm_smem(FF_MP_P, mt), h->stream>>>(h->D.off, h->B.src, h->B.mpcoef, h->B.mpa0);
    const FfLocArgs la = h->B.loc(L.M);
    k_ff_local<FF_MP_P><<<L.M, 128, 0, h->stream>>>(la);
    k_farfield_loc<FF_MP_P><<<L.M, 128, 0, h->stream>>>(a, la, h->B.src);
  } else if (h->ffs.on) {
    const FfSymArgs fa = ffs_args(h->ffs, L, h->near_mask, h->B, h->err);
    ffs_launch(h->ffs, fa, h->B, h->D, u, h->stream);
    ffs_reduce(h->ffs, fa, h->D, u, h->stream);
  } else {
    k_farfield_f32<FF_THREADS, FF_CHUNK><<<grid, FF_THREADS, 0, h->stream>>>(a, h->B.src, h->B.centre32, h->B.h2,
                                                                        h->B.gsum);
  }
  VS_CK(h, cudaGetLastError(), "far field");
  return VS_OK;
}

vs_status vs_farfield_counters(vs_farfield_plan* h, int64_t* out2) {
  if (!h || !out2) return VS_ERR_INVALID_ARG;
  VS_CK(h, cudaStreamSynchronize(h->stream), "counters");
  unsigned e = 0;
  VS_CK(h, cudaMemcpy(&e, h->err, sizeof e, cudaMemcpyDeviceToHost), "counters");
  std::vector<int> nc(h->L.P);
  VS_CK(h, cudaMemcpy(nc.data(), h->B.near_cnt, h->L.P * sizeof(int), cudaMemcpyDeviceToHost), "counters");
  int64_t pairs = 0;
  for (int c : nc) pairs += c;
  out2[0] = e;
  out2[1] = pairs;
  return VS_OK;
}

const char* vs_farfield_last_error(const vs_farfield_plan* h) { return h ? h->msg.c_str() : g_create_msg.c_str(); }

void vs_farfield_plan_destroy(vs_farfield_plan* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  h->D.release();
  h->B.release();
  h->ffs.release();
  cudaFree(h->err);
  delete h;
}

// ---------------------------------------------------------------------------------------------

vs_status vs_batched_inverse32(const float* a, float* a_inv, int32_t n, int32_t batch, int32_t* fallbacks,
                               void* cuda_stream) {
  if (!a || !a_inv || n < 1 || n > 128 || batch < 1) return VS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned* err = nullptr;
  int* fb = nullptr;
  cudaError_t e = dalloc(&err, 1);
  if (e == cudaSuccess) e = dalloc(&fb, 1);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(fb, 0, sizeof(int), s);
  const size_t bytes = (size_t)batch * n * n * sizeof(float);
  if (e == cudaSuccess && a != a_inv) e = cudaMemcpyAsync(a_inv, a, bytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = gj32_launch(DenseGeo32{a_inv, n}, n, batch, s, err, nullptr, fb);
  if (e == cudaSuccess) e = cudaGetLastError();
  unsigned he = 0;
  int hf = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&he, err, sizeof he, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hf, fb, sizeof hf, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(err);
  cudaFree(fb);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? VS_ERR_NOMEM : VS_ERR_CUDA;
  if (fallbacks) *fallbacks = hf;
  return (he & ERR_PIVOT) ? VS_ERR_UNSTABLE : VS_OK;
}

vs_status vs_fp32_rate(int32_t mix, int32_t iters, double* tera_lane_ops, double* ms, void* cuda_stream) {
  if ((mix != 0 && mix != 1) || iters < 1 || iters > (1 << 20) || !tera_lane_ops) return VS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = 2 * sms;  // 16 warps per SM, the symmetric far field's residency
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = dalloc(&out, (int64_t)blocks * threads);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // mix 0: 8 chains of 2 lanes per step; mix 1: PROBE_ROWS pair-pairs of 18 paired instructions per step
  const int steps = mix == 0 ? 4 * iters : iters;
  float t = 0.f;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
    cudaEventRecord(e0, s);
    if (mix == 0) k_probe_ffma2<<<blocks, threads, 0, s>>>(out, steps);
    else k_probe_pair<<<blocks, threads, 0, s>>>(out, steps);
    cudaEventRecord(e1, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? VS_ERR_NOMEM : VS_ERR_CUDA;
  const double lanes = (double)blocks * threads * steps * (mix == 0 ? 16.0 : PROBE_ROWS * 36.0);
  *tera_lane_ops = lanes / (t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return VS_OK;
}

vs_status vs_standardize(const double* xy, const int64_t* offsets, int32_t M, int32_t kmax, float* xin,
                         double* frames, void* cuda_stream) {
  if (!xy || !xin || !frames || kmax < 0) return VS_ERR_INVALID_ARG;
  Layout L;
  std::string msg;
  if (!build_layout(offsets, M, L, msg)) return VS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  DevLayout D;
  StdFrame* fr = nullptr;
  cudaError_t e = upload_layout(L, D, s);
  if (e == cudaSuccess) e = dalloc(&fr, L.M);
  if (e == cudaSuccess) {
    k_standardize<<<M, NMAX, 0, s>>>(D.vi(), xy, D.tab, xin, 2 * L.nmax, fr, kmax, false);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) {
    std::vector<StdFrame> hf(M);
    e = cudaMemcpy(hf.data(), fr, M * sizeof(StdFrame), cudaMemcpyDeviceToHost);
    std::vector<double> out(6 * (size_t)M);
    for (int v = 0; v < M; ++v) {
      out[6 * v + 0] = hf[v].cx; out[6 * v + 1] = hf[v].cy; out[6 * v + 2] = hf[v].ct;
      out[6 * v + 3] = hf[v].st; out[6 * v + 4] = hf[v].s; out[6 * v + 5] = hf[v].j0;
    }
    if (e == cudaSuccess) e = cudaMemcpy(frames, out.data(), out.size() * sizeof(double), cudaMemcpyHostToDevice);
  }
  cudaFree(fr);
  D.release();
  return e == cudaSuccess ? VS_OK : (e == cudaErrorMemoryAllocation ? VS_ERR_NOMEM : VS_ERR_CUDA);
}

vs_status vs_self_matrices(const double* xy, const int64_t* offsets, int32_t M, double mu, double* S_out,
                           void* cuda_stream) {
  if (!xy || !S_out || !(mu > 0)) return VS_ERR_INVALID_ARG;
  Layout L;
  std::string msg;
  if (!build_layout(offsets, M, L, msg)) return VS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // a private layout whose matrix offsets are 4 N^2 apart (the output's packing)
  std::vector<int64_t> moff(M + 1);
  int64_t acc = 0;
  for (int v = 0; v < M; ++v) { moff[v] = acc; acc += 4 * (int64_t)L.N[v] * L.N[v]; }
  moff[M] = acc;
  DevLayout D;
  SourceBufs B;
  cudaError_t e = upload_layout(L, D, s);
  if (e == cudaSuccess) e = upload(D.moff, moff.data(), M + 1, s);
  if (e == cudaSuccess) e = B.alloc(L.P, L.M);
  if (e == cudaSuccess) {
    FlowDev none{0, 0.0, 0.0};
    launch_geometry(M, L.nmax, s, D.vi(), xy, nullptr, D.tab, 1.0, mu, none, B.geom(), ForceOut{}, nullptr);
    const int n = L.nmax;
    k_self_matrix<<<self_grid(n, M), 256, 0, s>>>(D.vi(), xy, B.sa, B.tx, B.ty, D.tab, mu, S_out, 0, nullptr);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  D.release();
  B.release();
  return e == cudaSuccess ? VS_OK : (e == cudaErrorMemoryAllocation ? VS_ERR_NOMEM : VS_ERR_CUDA);
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Learned part: MLP forward / backward / AdamW on the tensor cores.


namespace {

inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

vs_status mlp_gemm(vs_mlp* h, const GemmArgs& a) {
  const dim3 grid((a.N + MM_BN - 1) / MM_BN, (a.M + MM_BM - 1) / MM_BM);
  k_gemm_bf16<<<grid, MM_THREADS, MM_SMEM, h->stream>>>(a);
  h->launches += 1;
  VS_CK(h, cudaGetLastError(), "mlp gemm");
  return VS_OK;
}

GemmArgs gemm_args(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, int M, int N, int K,
                   unsigned* err) {
  GemmArgs a{};
  a.A = A; a.lda = lda; a.B = B; a.ldb = ldb; a.M = M; a.N = N; a.K = K; a.act = EPI_NONE; a.err = err;
  return a;
}

vs_status mlp_refresh_bf16(vs_mlp* h) {
  for (int l = 0; l < h->L; ++l) {
    const int rows = h->dims[l + 1], cols = h->dims[l];
    const int64_t n = (int64_t)rows * cols;
    k_weights_bf16<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(h->w + h->woff[l], rows, cols, h->Wb[l],
                                                                        h->WbT[l]);
    h->launches += 1;
  }
  VS_CK(h, cudaGetLastError(), "mlp weights");
  return VS_OK;
}

// out_map: apply the output map (inference); training compares the output before it with the mapped
// targets.
vs_status mlp_forward(vs_mlp* h, const float* x, int batch, bool out_map) {
  const int Bp = round_up(batch, MM_BM);
  const int d0 = h->dims[0], dL = h->dims[h->L];
  const int64_t n0 = (int64_t)Bp * d0;
  k_rows_to_bf16<<<(unsigned)((n0 + 255) / 256), 256, 0, h->stream>>>(x, batch, Bp, d0, h->has_in ? h->aff : nullptr,
                                                                      h->aff + d0, h->H[0], h->HT[0]);
  h->launches += 1;
  VS_CK(h, cudaGetLastError(), "mlp input");
  for (int l = 0; l < h->L; ++l) {
    GemmArgs a = gemm_args(h->H[l], h->dims[l], h->Wb[l], h->dims[l], Bp, h->dims[l + 1], h->dims[l], h->err);
    a.bias = h->w + h->boff[l];
    if (l + 1 < h->L) {
      a.act = EPI_RELU;
      a.out_bf = h->H[l + 1];
      a.ld_bf = h->dims[l + 1];
      a.out_bfT = h->HT[l + 1];
      a.ld_bfT = Bp;
    } else {
      a.out_f32 = h->yhat;
      a.ld_f32 = h->dims[l + 1];
      if (out_map && h->has_out) {
        a.oshift = h->aff + 2 * d0;
        a.oscale = h->aff + 2 * d0 + dL;
      }
    }
    vs_status st = mlp_gemm(h, a);
    if (st != VS_OK) return st;
  }
  return VS_OK;
}

// gradient of the loss into h->g (flat, same layout as the parameters); loss into h->loss
vs_status mlp_backward(vs_mlp* h, const float* y, int batch) {
  const int Bp = round_up(batch, MM_BM);
  const int dL = h->dims[h->L];
  const int d0 = h->dims[0];
  const float* ysh = h->has_out ? h->aff + 2 * d0 : nullptr;
  k_mlp_loss<<<Bp, 128, 0, h->stream>>>(h->yhat, y, ysh, h->aff + 2 * d0 + 2 * dL, h->ynorm, batch, dL, h->ncomp, h->beta,
                                        h->g32[0], h->gbf[0], h->gbfT[0], Bp,
                                        h->loss_b);
  k_mean<<<1, 32, 0, h->stream>>>(h->loss_b, batch, h->loss);
  h->launches += 2;
  VS_CK(h, cudaGetLastError(), "mlp loss");
  int cur = 0;
  for (int l = h->L - 1; l >= 0; --l) {
    const int dout = h->dims[l + 1], din = h->dims[l];
    // dW_l = G^T H_l  (d_out x d_in), reduction over the padded batch
    GemmArgs a = gemm_args(h->gbfT[cur], Bp, h->HT[l], Bp, dout, din, Bp, h->err);
    a.out_f32 = h->g + h->woff[l];
    a.ld_f32 = din;
    vs_status st = mlp_gemm(h, a);
    if (st != VS_OK) return st;
    k_colsum<<<(dout + 127) / 128, 128, 0, h->stream>>>(h->g32[cur], Bp, dout, h->g + h->boff[l]);
    h->launches += 1;
    if (l > 0) {
      // dH_l = (G W_l) * (H_l > 0)
      GemmArgs b = gemm_args(h->gbf[cur], dout, h->WbT[l], dout, Bp, din, dout, h->err);
      b.act = EPI_MASK;
      b.mask = h->H[l];
      b.ld_mask = din;
      b.out_f32 = h->g32[1 - cur];
      b.ld_f32 = din;
      b.out_bf = h->gbf[1 - cur];
      b.ld_bf = din;
      b.out_bfT = h->gbfT[1 - cur];
      b.ld_bfT = Bp;
      if ((st = mlp_gemm(h, b)) != VS_OK) return st;
      cur = 1 - cur;
    }
  }
  VS_CK(h, cudaGetLastError(), "mlp backward");
  return VS_OK;
}

const float* mlp_output(const vs_mlp* h) { return h->yhat; }

vs_status mlp_check_err(vs_mlp* h) {
  unsigned e = 0;
  VS_CK(h, cudaStreamSynchronize(h->stream), "mlp sync");
  VS_CK(h, cudaMemcpy(&e, h->err, sizeof e, cudaMemcpyDeviceToHost), "mlp error word");
  if (e & ERR_MMA_TIMEOUT) { h->msg = "tensor-core GEMM wait timed out"; return VS_ERR_TIMEOUT; }
  return VS_OK;
}

void mlp_free(vs_mlp* h) {
  cudaFree(h->w); cudaFree(h->g); cudaFree(h->m); cudaFree(h->v); cudaFree(h->yhat);
  for (auto* p : h->Wb) cudaFree(p);
  for (auto* p : h->WbT) cudaFree(p);
  for (auto* p : h->H) cudaFree(p);
  for (auto* p : h->HT) cudaFree(p);
  for (int i = 0; i < 2; ++i) { cudaFree(h->g32[i]); cudaFree(h->gbf[i]); cudaFree(h->gbfT[i]); }
  cudaFree(h->loss_b); cudaFree(h->loss); cudaFree(h->err);
  cudaFree(h->aff); cudaFree(h->ynorm); cudaFree(h->stats);
}

}  // namespace

extern "C" {

vs_status vs_mlp_create(const int32_t* dims, int32_t nlayers, int32_t max_batch, int32_t ncomp, float beta,
                        void* cuda_stream, vs_mlp** out) {
  if (!out) return VS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!dims || nlayers < 1 || max_batch < 1 || ncomp < 1 || !(beta >= 0.f)) {
    g_create_msg = "bad MLP arguments";
    return VS_ERR_INVALID_ARG;
  }
  for (int l = 0; l <= nlayers; ++l)
    if (dims[l] < 16 || dims[l] % 16 != 0 || dims[l] > MLP_MAX_OUT) {
      g_create_msg = "MLP widths must be multiples of 16 in [16, 16384]";
      return VS_ERR_INVALID_ARG;
    }
  if (dims[nlayers] % ncomp != 0) {
    g_create_msg = "output width must be divisible by ncomp";
    return VS_ERR_INVALID_ARG;
  }
  vs_mlp* h = new (std::nothrow) vs_mlp();
  if (!h) return VS_ERR_NOMEM;
  h->dims.assign(dims, dims + nlayers + 1);
  h->L = nlayers;
  h->Bcap = round_up(max_batch, MM_BM);
  h->ncomp = ncomp;
  h->beta = beta;
  h->stream = (cudaStream_t)cuda_stream;
  int64_t o = 0;
  for (int l = 0; l < h->L; ++l) { h->woff.push_back(o); o += (int64_t)h->dims[l] * h->dims[l + 1]; }
  for (int l = 0; l < h->L; ++l) { h->boff.push_back(o); o += h->dims[l + 1]; }
  h->nparam = o;
  int dmax = 0;
  for (int d : h->dims) dmax = std::max(dmax, d);
  cudaError_t e;
  auto fail = [&](cudaError_t ee) {
    cuda_fail(g_create_msg, ee, "vs_mlp_create");
    mlp_free(h);
    delete h;
    return ee == cudaErrorMemoryAllocation ? VS_ERR_NOMEM : VS_ERR_CUDA;
  };
#define VS_M(x) do { e = (x); if (e != cudaSuccess) return fail(e); } while (0)
  VS_M(dalloc(&h->w, h->nparam)); VS_M(dalloc(&h->g, h->nparam));
  VS_M(dalloc(&h->m, h->nparam)); VS_M(dalloc(&h->v, h->nparam));
  h->Wb.assign(h->L, nullptr); h->WbT.assign(h->L, nullptr);
  for (int l = 0; l < h->L; ++l) {
    VS_M(dalloc(&h->Wb[l], (int64_t)h->dims[l] * h->dims[l + 1]));
    VS_M(dalloc(&h->WbT[l], (int64_t)h->dims[l] * h->dims[l + 1]));
  }
  h->H.assign(h->L, nullptr); h->HT.assign(h->L, nullptr);
  for (int l = 0; l < h->L; ++l) {
    VS_M(dalloc(&h->H[l], (int64_t)h->Bcap * h->dims[l]));
    VS_M(dalloc(&h->HT[l], (int64_t)h->Bcap * h->dims[l]));
  }
  VS_M(dalloc(&h->yhat, (int64_t)h->Bcap * h->dims[h->L]));
  for (int i = 0; i < 2; ++i) {
    VS_M(dalloc(&h->g32[i], (int64_t)h->Bcap * dmax));
    VS_M(dalloc(&h->gbf[i], (int64_t)h->Bcap * dmax));
    VS_M(dalloc(&h->gbfT[i], (int64_t)h->Bcap * dmax));
  }
  VS_M(dalloc(&h->loss_b, h->Bcap)); VS_M(dalloc(&h->loss, 1)); VS_M(dalloc(&h->err, 1));
  VS_M(dalloc(&h->aff, 2 * (int64_t)h->dims[0] + 3 * (int64_t)h->dims[h->L]));
  VS_M(dalloc(&h->ynorm, (int64_t)h->Bcap * h->dims[h->L]));
  VS_M(dalloc(&h->stats, 2 * (int64_t)std::max(h->dims[0], h->dims[h->L])));
  VS_M(cudaMemset(h->err, 0, sizeof(unsigned)));
  VS_M(cudaMemset(h->w, 0, h->nparam * sizeof(float)));
  VS_M(cudaMemset(h->m, 0, h->nparam * sizeof(float)));
  VS_M(cudaMemset(h->v, 0, h->nparam * sizeof(float)));
  VS_M(cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, MM_SMEM));
#undef VS_M
  if (mlp_refresh_bf16(h) != VS_OK) return fail(cudaErrorUnknown);
  *out = h;
  return VS_OK;
}

vs_status vs_mlp_num_params(const vs_mlp* h, int64_t* n) {
  if (!h || !n) return VS_ERR_INVALID_ARG;
  *n = h->nparam;
  return VS_OK;
}

vs_status vs_mlp_set_params(vs_mlp* h, const float* params, int64_t n) {
  if (!h || !params || n != h->nparam) return VS_ERR_INVALID_ARG;
  VS_CK(h, cudaMemcpyAsync(h->w, params, n * sizeof(float), cudaMemcpyHostToDevice, h->stream), "set params");
  VS_CK(h, cudaMemsetAsync(h->m, 0, n * sizeof(float), h->stream), "set params");
  VS_CK(h, cudaMemsetAsync(h->v, 0, n * sizeof(float), h->stream), "set params");
  h->t = 0;
  vs_status st = mlp_refresh_bf16(h);
  if (st != VS_OK) return st;
  VS_CK(h, cudaStreamSynchronize(h->stream), "set params");
  return VS_OK;
}

vs_status vs_mlp_get_params(vs_mlp* h, float* params, int64_t n) {
  if (!h || !params || n != h->nparam) return VS_ERR_INVALID_ARG;
  VS_CK(h, cudaMemcpyAsync(params, h->w, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream), "get params");
  VS_CK(h, cudaStreamSynchronize(h->stream), "get params");
  return VS_OK;
}

vs_status vs_mlp_set_affine(vs_mlp* h, const float* in_shift, const float* in_scale, const float* out_shift,
                            const float* out_scale) {
  if (!h) return VS_ERR_INVALID_ARG;
  const int d0 = h->dims[0], dL = h->dims[h->L];
  std::vector<float> a(2 * d0 + 3 * dL);
  for (int j = 0; j < d0; ++j) {
    a[j] = in_shift ? in_shift[j] : 0.f;
    a[d0 + j] = in_scale ? in_scale[j] : 1.f;
  }
  for (int j = 0; j < dL; ++j) {
    a[2 * d0 + j] = out_shift ? out_shift[j] : 0.f;
    const float t = out_scale ? out_scale[j] : 1.f;
    if (!(t != 0.f) || !std::isfinite(t)) return VS_ERR_INVALID_ARG;
    a[2 * d0 + dL + j] = t;
    a[2 * d0 + 2 * dL + j] = 1.f / t;
  }
  for (float x : a)
    if (!std::isfinite(x)) return VS_ERR_INVALID_ARG;
  VS_CK(h, cudaMemcpyAsync(h->aff, a.data(), a.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream), "set affine");
  VS_CK(h, cudaStreamSynchronize(h->stream), "set affine");
  h->has_in = in_shift || in_scale;
  h->has_out = out_shift || out_scale;
  return VS_OK;
}

vs_status vs_mlp_get_affine(vs_mlp* h, float* in_shift, float* in_scale, float* out_shift, float* out_scale) {
  if (!h) return VS_ERR_INVALID_ARG;
  const int d0 = h->dims[0], dL = h->dims[h->L];
  std::vector<float> a(2 * d0 + 3 * dL);
  VS_CK(h, cudaMemcpyAsync(a.data(), h->aff, a.size() * sizeof(float), cudaMemcpyDeviceToHost, h->stream), "get affine");
  VS_CK(h, cudaStreamSynchronize(h->stream), "get affine");
  for (int j = 0; j < d0; ++j) {
    if (in_shift) in_shift[j] = h->has_in ? a[j] : 0.f;
    if (in_scale) in_scale[j] = h->has_in ? a[d0 + j] : 1.f;
  }
  for (int j = 0; j < dL; ++j) {
    if (out_shift) out_shift[j] = h->has_out ? a[2 * d0 + j] : 0.f;
    if (out_scale) out_scale[j] = h->has_out ? a[2 * d0 + dL + j] : 1.f;
  }
  return VS_OK;
}

vs_status vs_mlp_fit_affine(vs_mlp* h, const float* x, const float* y, int32_t rows, double rel_floor) {
  if (!h || !x || !y || rows < 1 || !(rel_floor >= 0.0)) return VS_ERR_INVALID_ARG;
  const int d0 = h->dims[0], dL = h->dims[h->L];
  std::vector<double> st(2 * (size_t)std::max(d0, dL));
  std::vector<float> sh_in(d0), sc_in(d0), sh_out(dL), sc_out(dL);
  const int dmx = std::max(d0, dL);
  for (int pass = 0; pass < 2; ++pass) {
    const int d = pass ? dL : d0;
    k_colstats<<<(d + 127) / 128, 128, 0, h->stream>>>(pass ? y : x, rows, d, h->stats, h->stats + dmx);
    h->launches += 1;
    VS_CK(h, cudaGetLastError(), "fit affine");
    VS_CK(h, cudaMemcpyAsync(st.data(), h->stats, 2 * dmx * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
          "fit affine");
    VS_CK(h, cudaStreamSynchronize(h->stream), "fit affine");
    double sdmax = 0.0;
    for (int j = 0; j < d; ++j)
      if (std::isfinite(st[dmx + j])) sdmax = std::max(sdmax, st[dmx + j]);
    for (int j = 0; j < d; ++j) {
      const double m = st[j], sd = std::max(st[dmx + j], rel_floor * sdmax);
      const bool flat = !(sd > 0.0) || !std::isfinite(sd);
      if (pass) {
        sh_out[j] = (float)m;
        sc_out[j] = flat ? 1.f : (float)sd;
      } else {
        sh_in[j] = (float)m;
        sc_in[j] = flat ? 1.f : (float)(1.0 / sd);
      }
    }
  }
  return vs_mlp_set_affine(h, sh_in.data(), sc_in.data(), sh_out.data(), sc_out.data());
}

vs_status vs_mlp_forward(vs_mlp* h, const float* x, int32_t batch, float* y) {
  if (!h || !x || !y || batch < 1 || batch > h->Bcap) return VS_ERR_INVALID_ARG;
  vs_status st = mlp_forward(h, x, batch, true);
  if (st != VS_OK) return st;
  const int dL = h->dims[h->L];
  VS_CK(h, cudaMemcpyAsync(y, h->yhat, (size_t)batch * dL * sizeof(float), cudaMemcpyDeviceToDevice, h->stream),
        "forward out");
  return VS_OK;
}

vs_status vs_mlp_loss_grad(vs_mlp* h, const float* x, const float* y, int32_t batch, float* loss, float* grad,
                           int64_t n) {
  if (!h || !x || !y || !loss || batch < 1 || batch > h->Bcap) return VS_ERR_INVALID_ARG;
  if (grad && n != h->nparam) return VS_ERR_INVALID_ARG;
  vs_status st = mlp_forward(h, x, batch, false);
  if (st == VS_OK) st = mlp_backward(h, y, batch);
  if (st != VS_OK) return st;
  VS_CK(h, cudaMemcpyAsync(loss, h->loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream), "loss");
  if (grad) VS_CK(h, cudaMemcpyAsync(grad, h->g, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream), "grad");
  return mlp_check_err(h);
}

vs_status vs_mlp_train_step(vs_mlp* h, const float* x, const float* y, int32_t batch, const vs_adamw* opt, float* loss) {
  if (!h || !x || !y || !opt || batch < 1 || batch > h->Bcap) return VS_ERR_INVALID_ARG;
  vs_status st = mlp_forward(h, x, batch, false);
  if (st == VS_OK) st = mlp_backward(h, y, batch);
  if (st != VS_OK) return st;
  h->t += 1;
  const float c1 = 1.f - powf(opt->beta1, (float)h->t), c2 = 1.f - powf(opt->beta2, (float)h->t);
  k_adamw<<<(unsigned)((h->nparam + 255) / 256), 256, 0, h->stream>>>(h->w, h->g, h->m, h->v, h->nparam, opt->lr,
                                                                      opt->beta1, opt->beta2, opt->eps,
                                                                      opt->weight_decay, c1, c2);
  h->launches += 1;
  VS_CK(h, cudaGetLastError(), "adamw");
  if ((st = mlp_refresh_bf16(h)) != VS_OK) return st;
  if (loss) {
    VS_CK(h, cudaMemcpyAsync(loss, h->loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream), "loss");
    return mlp_check_err(h);
  }
  return VS_OK;
}

vs_status vs_mlp_sync(vs_mlp* h) {
  if (!h) return VS_ERR_INVALID_ARG;
  return mlp_check_err(h);
}

const char* vs_mlp_last_error(const vs_mlp* h) { return h ? h->msg.c_str() : g_create_msg.c_str(); }

void vs_mlp_destroy(vs_mlp* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  mlp_free(h);
  delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Far field with file-scope scratch: for callers that must not allocate device memory.
//
// Scratch lives in one static __device__ array (every GPU that loads this library holds it until
// the process exits). Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress (with that device current)
// and fills the differentiation tables there; later calls reuse the address.
namespace {

constexpr int SF_MAX_M = VS_STATIC_MAX_VESICLES;
constexpr int64_t SF_MAX_P = VS_STATIC_MAX_POINTS;
constexpr int SF_NSLOTS = (NMAX - 8) / 2 + 1;            // even N in [8, NMAX]
constexpr int64_t SF_TAB = (int64_t)TAB_STRIDE * (NMAX + 2 + 6) * (NMAX + 2 - 8) / 4;  // all N slots

// byte offsets inside the scratch array (each region 256-byte aligned)
constexpr int64_t sf_align(int64_t b) { return (b + 255) / 256 * 256; }
constexpr int64_t SF_N = 0;
constexpr int64_t SF_OFF = SF_N + sf_align(4 * SF_MAX_M);
constexpr int64_t SF_TOFF = SF_OFF + sf_align(8 * (SF_MAX_M + 1));
constexpr int64_t SF_OWNER = SF_TOFF + sf_align(8 * SF_MAX_M);
constexpr int64_t SF_CHUNK = SF_OWNER + sf_align(4 * SF_MAX_P);
constexpr int64_t SF_ERR = SF_CHUNK + sf_align(4 * (SF_MAX_M + 1));
constexpr int64_t SF_TABLE = SF_ERR + 256;
constexpr int64_t SF_GEOM = SF_TABLE + sf_align(8 * SF_TAB);        // sa, tx, ty, bx, by
constexpr int64_t SF_AREA = SF_GEOM + sf_align(5 * 8 * SF_MAX_P);   // area, length
constexpr int64_t SF_F = SF_AREA + sf_align(2 * 8 * SF_MAX_M);
constexpr int64_t SF_G64 = SF_F + sf_align(16 * SF_MAX_P);
constexpr int64_t SF_SRC = SF_G64 + sf_align(16 * SF_MAX_P);
constexpr int64_t SF_CENTRE = SF_SRC + sf_align(16 * SF_MAX_P);
constexpr int64_t SF_CENTRE32 = SF_CENTRE + sf_align(16 * SF_MAX_M);
constexpr int64_t SF_H2 = SF_CENTRE32 + sf_align(16 * SF_MAX_M);
constexpr int64_t SF_GSUM = SF_H2 + sf_align(8 * SF_MAX_M);
constexpr int64_t SF_BYTES = SF_GSUM + sf_align(8 * SF_MAX_M);

__device__ __align__(256) static unsigned char g_ff_scratch[SF_BYTES];

__host__ __device__ inline int64_t sf_tab_slot(int N) { return (int64_t)TAB_STRIDE * (N + 6) * (N - 8) / 4; }

// Differentiation circulant d(m) = (-1)^m cot(pi m / N) / 2 of every even N (the only table
// entries the source-preparation kernel reads).
__global__ void k_static_tables(unsigned char* base) {
  double* tab = (double*)(base + SF_TABLE);
  for (int s = blockIdx.x; s < SF_NSLOTS; s += gridDim.x) {
    const int N = 8 + 2 * s;
    double* t = tab + sf_tab_slot(N);
    for (int m = threadIdx.x; m < N; m += blockDim.x)
      t[m] = (m == 0) ? 0.0 : 0.5 * ((m & 1) ? -1.0 : 1.0) / tan(VS_PI * m / N);
  }
}

// Per-call layout from the offsets already copied into the scratch: N, table slots, owners,
// and the same greedy source chunks the allocating path builds on the host.
__global__ void k_static_layout(unsigned char* base, int M) {
  const int64_t* off = (const int64_t*)(base + SF_OFF);
  int32_t* N = (int32_t*)(base + SF_N);
  int64_t* toff = (int64_t*)(base + SF_TOFF);
  int32_t* owner = (int32_t*)(base + SF_OWNER);
  for (int v = threadIdx.x; v < M; v += blockDim.x) {
    const int n = (int)(off[v + 1] - off[v]);
    N[v] = n;
    toff[v] = sf_tab_slot(n);
    for (int64_t p = off[v]; p < off[v + 1]; ++p) owner[p] = v;
  }
  if (threadIdx.x == 0) {
    int32_t* chunk = (int32_t*)(base + SF_CHUNK);
    int c = 0;
    int64_t acc = 0;
    chunk[c++] = 0;
    for (int v = 0; v < M; ++v) {
      const int n = (int)(off[v + 1] - off[v]);
      if (acc + n > FF_CHUNK) { chunk[c++] = v; acc = 0; }
      acc += n;
    }
    chunk[c] = M;
    *(unsigned*)(base + SF_ERR) = 0u;
  }
}

std::mutex g_sf_mutex;
unsigned char* g_sf_ptr[256] = {};

}  // namespace

extern "C" vs_status vs_farfield_eval_static(const int64_t* offsets, int32_t M, double mu, int32_t precision,
                                             const double* xy, const double* f, double* u, void* cuda_stream) {
  if (!offsets || !xy || !f || !u || !(mu > 0) || (precision != 0 && precision != 1)) return VS_ERR_INVALID_ARG;
  if (M < 1 || M > SF_MAX_M || offsets[0] != 0) return VS_ERR_INVALID_ARG;
  int nchunk = 1;
  int64_t acc = 0;
  for (int v = 0; v < M; ++v) {
    const int64_t n = offsets[v + 1] - offsets[v];
    if (n < 8 || n > NMAX || (n & 1)) return VS_ERR_INVALID_ARG;
    if (acc + n > FF_CHUNK) { ++nchunk; acc = 0; }
    acc += n;
  }
  const int64_t P = offsets[M];
  if (P > SF_MAX_P) return VS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return VS_ERR_CUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_sf_mutex);
    if (!g_sf_ptr[dev]) {  // one-time set-up on this device
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_ff_scratch) != cudaSuccess || p == nullptr) return VS_ERR_CUDA;
      k_static_tables<<<SF_NSLOTS, 128, 0, st>>>((unsigned char*)p);
      if (cudaGetLastError() != cudaSuccess) return VS_ERR_CUDA;
      g_sf_ptr[dev] = (unsigned char*)p;
    }
    base = g_sf_ptr[dev];
  }
  if (cudaMemcpyAsync(base + SF_OFF, offsets, (M + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return VS_ERR_CUDA;
  k_static_layout<<<1, 256, 0, st>>>(base, M);
  const int64_t* off = (const int64_t*)(base + SF_OFF);
  const VesIndex vi{(const int32_t*)(base + SF_N), off, off, (const int64_t*)(base + SF_TOFF)};
  double* geo = (double*)(base + SF_GEOM);
  double* al = (double*)(base + SF_AREA);
  const GeomOut g{geo, geo + SF_MAX_P, geo + 2 * SF_MAX_P, geo + 3 * SF_MAX_P, geo + 4 * SF_MAX_P, al, al + SF_MAX_M};
  const ForceOut fo{(double*)(base + SF_F), u, (float4*)(base + SF_SRC), (double2*)(base + SF_CENTRE),
                    (float4*)(base + SF_CENTRE32), (float2*)(base + SF_H2), (double*)(base + SF_G64),
                    (float2*)(base + SF_GSUM)};
  const FlowDev none{0, 0.0, 0.0};
  k_geometry<1><<<M, NMAX, 0, st>>>(vi, xy, nullptr, (const double*)(base + SF_TABLE), 1.0, mu, none, g, fo, f);
  if (M >= 2) {
    FarFieldArgs a{P, M, (const int32_t*)(base + SF_OWNER), off, (const int32_t*)(base + SF_CHUNK), nchunk, 0, u,
                   nullptr, nullptr, (unsigned*)(base + SF_ERR)};
    const int grid = (int)((P + FF_THREADS - 1) / FF_THREADS);
    if (precision == 1)
      k_farfield_f64<<<grid, FF_THREADS, 0, st>>>(a, xy, fo.g64, g.length, vi.N);
    else
      k_farfield_f32<FF_THREADS, FF_CHUNK><<<grid, FF_THREADS, 0, st>>>(a, fo.src, fo.centre32, fo.h2, fo.gsum);
  }
  return cudaGetLastError() == cudaSuccess ? VS_OK : VS_ERR_CUDA;
}

// IVNet (the paper's network architecture) on the MLP part's tensor-core GEMM.
#include "ivnet_host.cuh"
