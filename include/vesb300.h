/*
 * vesb300 -- C ABI of the B300 (sm_103a) vesicle-suspension time step.
 *
 * The method is the 2D boundary-integral vesicle scheme of VesNet (arXiv 2606.25569): the
 * per-time-step hot path of Algorithm 1 with exact operators, i.e. the elastic force
 * f = -kappa_b X_ssss + (sigma X_s)_s (Eq. elastic_force), the all-pairs far-field single layer
 * with the 2D Stokeslet (Eqs. single_layer, Stokeslet; Sec. 2.2.2), the advection step
 * (Eq. advection_disc), the implicit relaxation step (Eq. relaxation_disc), redistribution to
 * equal arclength (Sec. 4.2), the tension update (Eq. tension_disc) and the area/length
 * correction (Sec. 4.3). The problem statement of Algorithm 1 (Sec. 4.4) fixes the inputs: the
 * vesicle points, the bending modulus kappa_b, the viscosity mu, the background flow and dt.
 *
 * Conventions shared by every entry point:
 *  - Point layout ("CSR blocks"): vesicle v owns points offsets[v] .. offsets[v+1]-1
 *    (N_v = offsets[v+1] - offsets[v], even, 8 <= N_v <= 128). A per-point 2-vector field
 *    (positions, forces, velocities) is stored per vesicle as its N_v x-components followed by
 *    its N_v y-components, starting at index 2*offsets[v]. Scalar fields (tension) start at
 *    offsets[v]. Points run counter-clockwise.
 *  - No exceptions cross the ABI; every call returns a vs_status. The message of the last
 *    failure of a handle is kept per handle (vs_last_error).
 *  - Handles are not thread-safe; separate handles are independent.
 *  - All GPU work of a handle is enqueued on the CUDA stream given at creation. Errors found by
 *    kernels (a zero pivot, a non-finite state, a correction that did not converge) are stored
 *    on the device and reported by the next call that synchronises (vs_sync, vs_get_*).
 *  - The library copies its inputs; output buffers belong to the caller.
 *  - There is no CPU fallback: without a usable CUDA device every call fails with VS_ERR_CUDA.
 */
#ifndef VESB300_H
#define VESB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VS_OK = 0,
  VS_ERR_INVALID_ARG = 1,   /* bad sizes, layout, parameters or a null pointer */
  VS_ERR_CUDA = 2,          /* a CUDA call failed (no device, launch error) */
  VS_ERR_NOMEM = 3,         /* device allocation failed */
  VS_ERR_NOT_CONVERGED = 4, /* area/length correction, or the implicit step's GMRES, did not converge */
  VS_ERR_UNSTABLE = 5,      /* non-finite state or a singular per-vesicle system */
  VS_ERR_TIMEOUT = 6,       /* reserved for bounded device-side waits */
  VS_ERR_NO_NETWORK = 7     /* reserved for the learned (hybrid) path */
} vs_status;

/* Background flow u_inf (Sec. 5.3-5.5): p[0], p[1] as listed. */
typedef enum {
  VS_FLOW_NONE = 0,
  VS_FLOW_SHEAR = 1,        /* u = p0 (y, 0)                                        (Sec. 5.4) */
  VS_FLOW_TAYLOR_GREEN = 2, /* u = p0 (sin(pi x/p1) cos(pi y/p1), -cos(pi x/p1) sin(pi y/p1))
                                                                                  (Eq. tayGreenFlow) */
  VS_FLOW_POISEUILLE = 3    /* u = p0 (1 - (y/p1)^2) e_x, walls at y = +-p1           (Sec. 5.3) */
} vs_flow_kind;

typedef struct {
  int32_t kind;  /* vs_flow_kind */
  int32_t pad_;
  double p[4];
} vs_flow;

/* flags */
#define VS_FLAG_FARFIELD_FP64 1ull /* far field in FP64 instead of compensated FP32 */
/* Per-vesicle solves with FP64 dense operator products and FP64 LU instead of the default mixed
 * precision (FP32 products and factorisations refined to FP64 accuracy by matrix-free FP64
 * residuals). Both give the FP64 solution; the default is several times faster on B300. */
#define VS_FLAG_DIRECT_FP64 2ull
/* Keep the default FP32 far-field launch shape instead of timing the shapes at vs_create
 * (vs_farfield_variant). */
#define VS_FLAG_NO_AUTOTUNE 4ull
/* Build the FP32 operator products of the mixed-precision path on the tensor cores (each FP32 operand
 * split into three BF16 parts, FP32 accumulation) instead of with FP32 FMAs; both give FP32-quality
 * preconditioners and the same FP64-accurate results. At N <= 128 the FMA kernels are faster. */
#define VS_FLAG_TC_GEMM 8ull
/* Far field through vesicle multipole expansions (order 12 about each vesicle's centre): for vesicle pairs
 * whose centres are farther apart than twice the sum of their reach radii, translated into one local
 * expansion about each target vesicle's centre (summed over those sources, evaluated once per target
 * point); for the other pairs the expansion per target point beyond three reach radii of the source, point
 * sums inside (near test and lists unchanged). An approximation of the all-pairs sum (the paper names FMM
 * as the route to O(M) cost) whose truncation error is below about 1e-8 of a vesicle's density scale;
 * FP32 with compensated accumulation. */
#define VS_FLAG_FARFIELD_MULTIPOLE 16ull
/* The FP32 far field sums over every ordered pair with one thread per target (k_farfield_f32, launch
 * shape autotuned) instead of the default symmetric evaluation. The symmetric kernel (k_farfield_sym)
 * visits each unordered pair of points of different vesicles once and adds both reactions (the
 * Stokeslet is even in r), with a deterministic chunked double-float reduction, for any point counts
 * (vesicles padded to 32, 64 or 128 points). Its partial sums take 16 bytes per point and chunk of
 * vesicles; beyond a budget (1/8 of the device memory, or the byte count in the environment variable
 * VS_FFS_SLOT_BYTES, read when the suspension or plan is created) the chunks are taken in groups that
 * fit it, one group pair at a time (the same sums, their double-float grouping aside), and below four
 * slots a point the per-target kernel runs. The two kernels agree to FP32 rounding. */
#define VS_FLAG_FARFIELD_PER_TARGET 32ull
/* Near field by the Ying-Zorin scheme (Sec. 2.2.2, the caption of Fig. fig:near-singular: the near-singular
 * integration of the paper's BIEM ground truth) instead of the five layers and the RBF of Sec. 3.3: at each
 * near target, the closest point x0 of the source curve's trigonometric interpolant (Newton, FP64), the
 * on-curve single layer there (the self rule's values interpolated along the membrane), the single layer at
 * six points x0 + s i h/4 n (i = 1..6, on the target's side s) by FP32 trapezoid sums on the curve upsampled
 * by ceil(sqrt(N)), and the interpolating polynomial in the distance. Needs near_field = 1; the learned near
 * field (vs_set_near_networks) takes precedence in a hybrid suspension. */
#define VS_FLAG_NEAR_YZ 64ull
/* Form the FP32 operator products of the mixed-precision path (T, L, and the relaxation's W and A) with one
 * batched GEMM launch per product over all vesicles instead of the default fused kernels, which form each
 * vesicle's chain of products in shared memory with one CTA per vesicle (vesicles of at most 64 points; larger
 * ones always take the batched launches). Both give FP32-quality preconditioners and the same FP64-accurate
 * results. */
#define VS_FLAG_OPS_BATCHED 128ull
/* Multipole far field through a cluster tree (Sec. 4.1 and Sec. 4.5 name the fast multipole method as the
 * route to a far-field cost linear in the number of vesicles): a quadtree of the vesicle centres (rebuilt on
 * the device every evaluation; boxes of at most 8 vesicles at the leaves), every box's order-12 expansion
 * about the mean of its vesicles' centres shifted exactly from its members' (multipole-to-multipole), and
 * for each target vesicle a walk from the root that translates whole boxes farther than twice the summed
 * radii into its local expansion, as VS_FLAG_FARFIELD_MULTIPOLE does vesicle by vesicle. The point sums and
 * their near test are those of VS_FLAG_FARFIELD_MULTIPOLE; the results agree with it to the expansions'
 * truncation error, at O(M log M) translations instead of O(M^2). At most 16384 vesicles
 * (VS_ERR_INVALID_ARG beyond); takes precedence over VS_FLAG_FARFIELD_MULTIPOLE. */
#define VS_FLAG_FARFIELD_TREE 256ull

typedef struct {
  double kappa_b;    /* bending modulus, > 0 */
  double mu;         /* viscosity, > 0 */
  double dt;         /* time step, > 0 */
  double corr_tol;   /* relative area/length error that triggers the correction (Sec. 4.3: 0.01) */
  int32_t mode;      /* 0: plain boundary-integral step, 1: hybrid (learned relaxation, vs_set_network),
                        2: fully implicit step (Sec. 2.2.3, Eq. time_step_sc1) solved by GMRES (vs_set_gmres) */
  int32_t near_field;/* 1: exclude near pairs (distance <= h of the source) from the far field */
  int32_t use_graph; /* 1: replay each step from a captured CUDA graph (needs a non-NULL stream and
                        profiling off; otherwise steps are launched one kernel at a time) */
  int32_t exact_every; /* hybrid only: every exact_every-th step (counting from 1) takes the exact
                          relaxation instead of the learned one; 0: never */
  uint64_t flags;    /* VS_FLAG_* */
  double exact_gap;  /* hybrid only: a vesicle closer than exact_gap point spacings h = L/N (the larger of
                        the two vesicles') to another vesicle relaxes exactly; 0 selects 4 */
} vs_params;

typedef struct vs_suspension vs_suspension;
typedef struct vs_mlp vs_mlp;

/*
 * Create a suspension (Algorithm 1 input, Sec. 4.4).
 *  xy       host, 2*offsets[M] doubles in CSR blocks: the initial points.
 *  offsets  host, M+1 increasing int64, offsets[0] = 0.
 *  params, flow  host structs, copied.
 *  cuda_stream   cudaStream_t (NULL = legacy default stream) for all later work.
 * The points are redistributed to equal arclength (Sec. 4.2); the resulting area and length
 * become the reference A_0, L_0 of the correction (Sec. 4.3); the initial tension is
 * sigma^0 = -L^{-1} P (B X^0 + u_inf(X^0)) (self and background terms only).
 * Returns VS_ERR_INVALID_ARG for M < 1, odd N, N outside [8, 128], non-finite points or bad
 * parameters; VS_ERR_NOMEM / VS_ERR_CUDA on device failures. On success *out owns all device
 * memory of the suspension until vs_destroy.
 */
vs_status vs_create(const double* xy, const int64_t* offsets, int32_t M, const vs_params* params,
                    const vs_flow* flow, void* cuda_stream, vs_suspension** out);

/*
 * Enqueue nsteps plain time steps (Algorithm 1 with exact operators): force, far field +
 * u_inf, advection (Eq. advection_disc), relaxation (Eq. relaxation_disc), redistribution
 * (Sec. 4.2), tension at the new points (Eq. tension_disc), correction (Sec. 4.3).
 * Asynchronous: returns once the work is enqueued.
 */
vs_status vs_step(vs_suspension* s, int32_t nsteps);

/*
 * Fully implicit step (mode 2; Sec. 2.2.3, Eq. time_step_sc1). With every operator at X^n and the
 * density f = -kappa D_s^4 X^{n+1} + (sigma^{n+1} X_s)_s, the velocity U = S f + far field of f from the
 * other vesicles (+ the near-field correction of f when near_field is set) satisfies
 *   X^{n+1} - dt U = X^n + dt u_inf(X^n),   P U = -P u_inf(X^n)
 * for all vesicles at once. vs_step solves it by restarted flexible GMRES (right preconditioning with the
 * per-vesicle solve of the same system without the other vesicles: FP32 explicit inverses, or the FP64 LU
 * factors under VS_FLAG_DIRECT_FP64; the products with the system matrix are FP64 either way, apart from
 * the far field the flags select; two-pass classical Gram-Schmidt),
 * starting from (X^n, sigma^n), until ||b - A z|| <= tol ||b|| by GMRES's own residual estimate; then
 * redistributes X^{n+1} (Sec. 4.2; sigma^{n+1} evaluated at the new parameters by its trigonometric
 * interpolant) and applies the area/length correction (Sec. 4.3). The far field of each product is the
 * one the flags select, so with the FP32 far field the attainable residual is limited by its rounding.
 * Each GMRES iteration reads one Hessenberg column on the host (the stream is synchronised), so vs_step
 * returns after the work of mode-2 steps has finished and never uses CUDA graphs. vs_get_velocity is not
 * defined in mode 2.
 *  vs_set_gmres: tol > 0 (default 1e-10), 1 <= restart <= VS_GMRES_MAX_RESTART (default 30) Krylov vectors
 *    per cycle, max_iter >= 1 (default 300) iterations per step; vs_step returns VS_ERR_NOT_CONVERGED
 *    when a step needs more (the state is then not advanced past the failing solve). Device memory:
 *    (2 restart + 5) * 3 P doubles, allocated by the first mode-2 step.
 *  vs_gmres_stats: iterations and relative residual estimate of the last step, iterations over all
 *    steps; any pointer may be NULL.
 */
#define VS_GMRES_MAX_RESTART 200
vs_status vs_set_gmres(vs_suspension* s, double tol, int32_t restart, int32_t max_iter);
vs_status vs_gmres_stats(const vs_suspension* s, int32_t* last_iters, double* last_residual, int64_t* total_iters);

/* Wait for the handle's stream and report device-side errors of earlier steps. */
vs_status vs_sync(vs_suspension* s);

/*
 * Replace positions and tension from host buffers (same layout as vs_create; sigma has
 * offsets[M] doubles). The points are used as given (no redistribution); A_0, L_0 are kept. The
 * operators cached for a vesicle stay valid when its points are bitwise unchanged (state read back with
 * vs_get_positions and passed in again); vesicles with any changed coordinate rebuild them. Synchronous.
 */
vs_status vs_set_state(vs_suspension* s, const double* xy, const double* sigma);

/* Copy the state to caller-owned host buffers; cap = buffer length in doubles.
 * positions: 2*P doubles (CSR blocks), tension: P, velocity: 2*P -- the velocity u^n of
 * Algorithm 1 (far field + near-field exclusion + u_inf) at the points of the last step's start.
 * Synchronises the stream. VS_ERR_INVALID_ARG when cap is too small. */
vs_status vs_get_positions(vs_suspension* s, double* xy, int64_t cap);
vs_status vs_get_tension(vs_suspension* s, double* sigma, int64_t cap);
vs_status vs_get_velocity(vs_suspension* s, double* u, int64_t cap);

/* Reference area/length (A_0, L_0) per vesicle: 2*M doubles, A_0 then L_0. */
vs_status vs_get_reference(vs_suspension* s, double* a0l0, int64_t cap);

/* Device pointers of positions (2P doubles) and tension (P doubles), borrowed: valid until the
 * next vs_step / vs_set_state / vs_destroy. */
vs_status vs_get_device_ptrs(const vs_suspension* s, const double** xy, const double** sigma);

/* Counters (out has 5 int64): [0] steps taken, [1] corrections applied, [2] near (target,
 * vesicle) pairs in the last far-field evaluation (when near_field), [3] device error bits,
 * [4] kernels launched by this handle so far. Synchronises. */
vs_status vs_get_counters(vs_suspension* s, int64_t* out5);

/* Fallback statistics of the hybrid step (Algorithm 1 with the learned maps of Sec. 3.2-3.3; the plain
 * step is the learned step's fallback and judge). out3 (3 int64, host): [0] steps so far whose
 * relaxation was the learned map; [1] steps that ran the fallback test (learned relaxation steps, and
 * every step when the advection and tension networks are set); [2] vesicles that took the exact step
 * in those steps (in a near pair, or within exact_gap spacings h of another vesicle), summed over
 * them, so that [2] / ([1] M) is the mean fraction of vesicles stepped exactly. Zero outside hybrid
 * mode and for one vesicle. Synchronises. */
vs_status vs_get_hybrid_counters(vs_suspension* s, int64_t* out3);

/*
 * Checkpoint and resume (no counterpart in the paper). A checkpoint holds what a later run needs to
 * continue bit for bit: positions, tension, A_0 and L_0, the step count and the correction counter, with
 * kappa_b, mu, dt, mode and a hash of the point counts, in a versioned layout of
 * vs_checkpoint_size bytes of caller-owned HOST memory. vs_restore loads one into a suspension created
 * with the same offsets and parameters (otherwise VS_ERR_INVALID_ARG); its cached operators are rebuilt
 * from the restored points at the next step, which gives the same bits as the uninterrupted run. A
 * hybrid suspension needs its network set again. Both synchronise; vs_checkpoint reports pending
 * device errors.
 */
vs_status vs_checkpoint_size(vs_suspension* s, int64_t* bytes);
vs_status vs_checkpoint(vs_suspension* s, void* buf, int64_t cap);
vs_status vs_restore(vs_suspension* s, const void* buf, int64_t size);

/* Launch shape of the per-target FP32 far field (a tuning control; the paper has no counterpart).
 * vs_create times the per-target kernel in each of its launch shapes (threads per CTA x source points
 * staged per chunk) on the suspension's own sources and keeps the fastest, unless VS_FLAG_NO_AUTOTUNE
 * is set or the symmetric kernel is in use (VS_FLAG_FARFIELD_PER_TARGET); the choice is cached per
 * (device name, M, points, near mask) in the process, and in the text file named by the environment
 * variable VS_TUNE_CACHE when it is set. Every shape gives bitwise identical velocities. set >= 0
 * selects per-target shape `set` (leaving the symmetric kernel; captured step graphs are dropped),
 * set < 0 leaves the choice. On return *index, *threads and *chunk (each may be null) describe the
 * kernel in use: shape index, threads per CTA, source points staged per chunk; index -1 for the
 * symmetric kernel (threads per CTA, points per chunk of vesicles). VS_ERR_INVALID_ARG for a null
 * handle or set beyond the last shape. */
vs_status vs_farfield_variant(vs_suspension* s, int32_t set, int32_t* index, int32_t* threads, int32_t* chunk);

/* Per-kernel timing: while enabled, every kernel the handle launches is bracketed by CUDA
 * events on its stream. vs_profile(s, 1) clears the totals and starts recording, 0 stops.
 * vs_profile_read returns, for kernel name index idx (0, 1, ... until VS_ERR_INVALID_ARG), its
 * name (NUL-terminated, truncated to name_cap), total milliseconds and launch count.
 * Synchronises. */
vs_status vs_profile(vs_suspension* s, int32_t enable);
vs_status vs_profile_read(vs_suspension* s, int32_t idx, char* name, int32_t name_cap, double* total_ms,
                          int64_t* launches);

/*
 * Learned maps for the hybrid step (params.mode = 1; VesNet, Sec. 3.2 and Algorithm 1).
 * which = 0: the relaxation flow map X_X (Eq. relaxation_disc replaced by a network): the step
 * redistributes X* (Sec. 4.2), standardises it (Sec. 3.4.1), evaluates net on the Fourier features of the
 * standardised shape and adds out_scale * (the displacement synthesised from the output's features),
 * mapped back from the standard frame, to the redistributed X*; the result, with its modes |k| > K
 * removed (the network does not represent them; the exact relaxation leaves them at their tiny size),
 * is X^{n+1}. Features, K = min(filter_kmax, N/2 - 1): with a_k = (1/N) sum_j v_j cos(2 pi k j/N) and
 * b_k = -(1/N) sum_j v_j sin(2 pi k j/N) of v = x^o then y^o, a row is [a_0..a_K, b_1..b_K (x);
 * a_0..a_K, b_1..b_K (y); zeros] of width W = 16 ceil((4K + 2)/16); outputs use the same layout
 * (v_j = a_0 + 2 sum_k (a_k cos - b_k sin)). The network (borrowed, must outlive its use) needs widths W
 * in and out, batch capacity >= M, the suspension's stream, and one N for all vesicles; otherwise
 * VS_ERR_INVALID_ARG. net = NULL removes it; a hybrid step without it fails with VS_ERR_NO_NETWORK.
 */
vs_status vs_set_network(vs_suspension* s, int32_t which, vs_mlp* net, double out_scale, int32_t filter_kmax);

/* Exact relaxation step (Eq. relaxation_disc) of the given DEVICE points (CSR blocks) into
 * xy_out, with the suspension's kappa_b, mu and dt -- the map the learned relaxation is trained
 * on. Does not change the suspension's state. Asynchronous. */
vs_status vs_relax(vs_suspension* s, const double* xy_in, double* xy_out);

/*
 * Learned advection and tension (Sec. 3.2: Eq. advectionMap X_u^k: X -> (I - M) e^{ik alpha}, Eq. advTenMap
 * S_u^k: X -> L^{-1} P e^{ik alpha}, and S_sigma: X -> L^{-1} P B X; Table tab:networks). In each vesicle's
 * standard frame (vs_standardize) the interaction velocity u is expanded in the real Fourier modes
 * k = 0..Kf of each component: with its features f (a_0..a_Kf, b_1..b_Kf of x, then of y, as the network
 * input of vs_set_network), u = sum_i f_i psi_i for modes <= Kf, psi_i one component equal to 1, 2 cos(k
 * alpha) or -2 sin(k alpha). Two networks give, per vesicle, the columns of the maps at the standardised
 * shape, each represented by its Fourier features up to Kout:
 *   advection network: row = [ (I - M) psi_0 | (I - M) psi_1 | ... ], 2 (2 Kout + 1) floats per column,
 *     zero-padded to flow_adv_width = 16 ceil((4 Kf + 2) 2 (2 Kout + 1) / 16);
 *   tension network: row = [ L^{-1} P B X | L^{-1} P psi_0 | ... ], 2 Kout + 1 floats each, zero-padded to
 *     flow_ten_width = 16 ceil((4 Kf + 3)(2 Kout + 1) / 16);
 * both with the input of the relaxation network (its width and filter_kmax). (I - M) and L^{-1} P do not
 * depend on the vesicle's size; L^{-1} P B X is that of the unit-length shape over L^2.
 *
 * vs_set_flow_networks: a hybrid suspension (mode 1) with these networks set takes, in every step, the
 * advection X* = X^n + dt R^T shift(sum_i f_i Q_i) and the tension sigma^{n+1} = -shift(S_sigma) / L^2 -
 * shift(sum_i f_i S_i) from them (modes of u above Kf dropped) instead of the exact operators, which it
 * then builds at X^n and X^{n+1} only for the vesicles of the hybrid fallback (in a near pair this step or
 * within exact_gap spacings of another vesicle: those take the exact advection and tension) and for the
 * source vesicles of near pairs (their near-field layers need them); the relaxation stays as
 * vs_set_network and exact_every arrange. The relaxation
 * network must be set first; adv and ten are borrowed, share the suspension's stream, have batch capacity
 * >= M; Kf, Kout in [0, N/2 - 1]; both NULL removes them. Errors: VS_ERR_INVALID_ARG.
 *
 * vs_flow_maps: training data of the two networks from the exact operators. For the suspension's current
 * points (equal N): xin (DEVICE FP32, M x W) = the network input (filter_kmax as for vs_set_network),
 * adv (DEVICE FP32, M x flow_adv_width) and ten (DEVICE FP32, M x flow_ten_width) = the rows above, computed
 * at each vesicle's standardised shape with the operators of the step (FP64-accurate). The suspension's
 * state and its operator cache for the next step are left as they were. Synchronous; allocates scratch.
 */
vs_status vs_set_flow_networks(vs_suspension* s, vs_mlp* adv, vs_mlp* ten, int32_t Kf, int32_t Kout);
vs_status vs_flow_maps(vs_suspension* s, int32_t Kf, int32_t Kout, int32_t filter_kmax, float* xin, float* adv,
                       float* ten);

/*
 * Learned near field (Sec. 3.3, Eq. NearFieldMap: N_X^k maps a shape to the single layer of the density
 * e^{ik alpha} at the five layer points X + d h n, d in {-1, -1/2, 0, 1/2, 1}). The density's Fourier features
 * f (modes 0..Kf of each component, in the vesicle's standard frame, as for the flow networks) combine the
 * columns of each layer: network d gives, per vesicle, the layer-d velocities of the nb = 4 Kf + 2 basis
 * densities psi_i at the unit-length standardised shape with mu = 1, as velocity features up to Kout
 * (2 (2 Kout + 1) floats per column, in basis order: flow_adv_width(Kf, Kout) outputs). The layer velocities
 * are then those of the density's modes <= Kf, f_K:
 *   S[X, f_K] = L R^T shift(sum_i f_i Q_d,i) / mu - (L log L / (4 pi mu)) I_d,
 * I_d the integral of f_K over the unit-length curve by the layer's quadrature (the N points on the curve,
 * the curve upsampled by ceil(sqrt(N)) off it); the RBF interpolation to the near targets is unchanged.
 *
 * vs_set_near_networks: a hybrid suspension (mode 1, created with near_field = 1) with these networks set
 * takes the layer velocities of every near source vesicle from them in every step. nets: n = 5 borrowed
 * networks, layer order as above (-h first); input width that of the relaxation network (set it first),
 * batch capacity >= M, the suspension's stream; Kf, Kout in [0, N/2 - 1]. nets NULL removes them. Errors:
 * VS_ERR_INVALID_ARG.
 *
 * vs_near_maps: training data of the five networks from the exact layer velocities. For the suspension's
 * current points (equal N): xin (DEVICE FP32, M x W) = the network input (filter_kmax as for vs_set_network)
 * and out (DEVICE FP32, 5 x M x flow_adv_width(Kf, Kout), layer-major) = the rows above (on-curve layer by
 * the self rule, off-curve layers by FP32 sums on the upsampled curve, as the plain near field computes
 * them). The suspension's state and its operator cache for the next step are left as they were.
 * Synchronous; allocates scratch.
 */
vs_status vs_set_near_networks(vs_suspension* s, vs_mlp* const* nets, int32_t n, int32_t Kf, int32_t Kout);
vs_status vs_near_maps(vs_suspension* s, int32_t Kf, int32_t Kout, int32_t filter_kmax, float* xin, float* out);

/* Training pairs of the relaxation map: for DEVICE points xy_in (CSR blocks, equal N), xin (device
 * FP32, M x W) = the network input of vs_set_network's map and yout (device FP32, M x W) = the
 * features of (relax(xy_in) - xy_in) in each vesicle's standard frame, divided by out_scale; W and the
 * features as for vs_set_network with the same filter_kmax. Asynchronous. */
vs_status vs_training_pairs(vs_suspension* s, const double* xy_in, float* xin, float* yout, double out_scale,
                            int32_t filter_kmax);

const char* vs_last_error(const vs_suspension* s);
void vs_destroy(vs_suspension* s);

/*
 * Far-field single layer alone (Sec. 2.2.2; the "direct evaluation" of Table tab:timings):
 *   u(x_i) = sum over vesicles v != vesicle(i) [not near x_i when near_mask] of
 *            sum_j G(x_i - X_vj) f_vj |X_alpha|_vj (2 pi / N_v),
 *   G = (1/4 pi mu)(-log|r| I + r r^T / |r|^2).
 * A plan holds the layout and its device buffers.
 *  offsets     host, M+1 int64 as in vs_create.
 *  precision   0: compensated FP32 (vesicle-relative coordinates; the symmetric pair kernel when every
 *              vesicle has 32, 64 or 128 points, see VS_FLAG_FARFIELD_PER_TARGET), 1: FP64, 2: FP32 with
 *              vesicle multipole expansions for far source vesicles (VS_FLAG_FARFIELD_MULTIPOLE),
 *              3: compensated FP32 with the per-target kernel whatever the point counts, 4: as 2 with
 *              the expansions of whole clusters of vesicles from a tree (VS_FLAG_FARFIELD_TREE; at most
 *              16384 vesicles).
 * vs_farfield_eval takes DEVICE pointers in CSR blocks: xy (2P), f (2P); writes u (2P, device,
 * overwritten) on the plan's stream. Asynchronous.
 */
typedef struct vs_farfield_plan vs_farfield_plan;
vs_status vs_farfield_plan_create(const int64_t* offsets, int32_t M, double mu, int32_t near_mask,
                                  int32_t precision, void* cuda_stream, vs_farfield_plan** out);
vs_status vs_farfield_eval(vs_farfield_plan* plan, const double* xy, const double* f, double* u);
/* Device error bits of the last evaluation (near-list overflow) and the number of near pairs.
 * Synchronises. */
vs_status vs_farfield_counters(vs_farfield_plan* plan, int64_t* out2);
const char* vs_farfield_last_error(const vs_farfield_plan* plan);
void vs_farfield_plan_destroy(vs_farfield_plan* plan);

/*
 * Per-vesicle self single-layer matrices (Eq. single_layer with the Kress product rule for the
 * log singularity, trapezoid weights otherwise; Sec. 2.2.2), for testing and for callers that
 * build their own operators. xy: device, CSR blocks. S_out: device, sum_v (2 N_v)^2 doubles,
 * vesicle v's row-major 2N_v x 2N_v matrix starting at 4 * sum_{u<v} N_u^2 (rows: u_x then u_y;
 * columns: f_x then f_y). Synchronous.
 */
vs_status vs_self_matrices(const double* xy, const int64_t* offsets, int32_t M, double mu,
                           double* S_out, void* cuda_stream);

/*
 * Batched FP32 inverse (the preconditioners of the mixed-precision solves are built with it): a_inv[v] =
 * a[v]^{-1} for batch row-major n x n DEVICE matrices (n <= 128; a and a_inv may be the same memory) by
 * register Gauss-Jordan exchange steps, first without pivoting and, for a matrix where a pivot falls to
 * 1e-4 of its largest entry or below, again with partial pivoting; *fallbacks (host, may be NULL) gets
 * the number of such matrices. A zero pivot column under pivoting is VS_ERR_UNSTABLE. Synchronous.
 */
vs_status vs_batched_inverse32(const float* a, float* a_inv, int32_t n, int32_t batch, int32_t* fallbacks,
                               void* cuda_stream);

/*
 * FP32 throughput probe: the measured denominator of the symmetric far field's roofline (its work is FP32
 * arithmetic, Sec. 2.2.2's all-pairs sum). Runs a register-only kernel, two CTAs of 256 threads per SM (the
 * far field's residency), after one warm-up launch: mix 0 times independent chains of paired FMAs (the
 * FP32 pipe's own limit), mix 1 the arithmetic of the far field's paired pair loop without its loads and
 * lane exchanges (per two pairs 18 paired FP32 instructions, 2 lg2 and 2 rcp: the ceiling of that
 * instruction mix). iters: loop rounds (1 .. 2^20; about 2048 take a few ms). tera_lane_ops (host): FP32
 * lane operations per second / 1e12 from CUDA events on cuda_stream; ms (host, may be NULL): the timed
 * launch. Synchronous; VS_ERR_INVALID_ARG for another mix or iters out of range.
 */
vs_status vs_fp32_rate(int32_t mix, int32_t iters, double* tera_lane_ops, double* ms, void* cuda_stream);

/*
 * Standardisation of every vesicle for the networks (Sec. 3.4.1): centroid, principal axis along
 * +y, unit length, cyclic relabelling so that point 0 is the right-most upward crossing of the x
 * axis, Fourier filter keeping modes |k| <= kmax (< N/2). xy: device CSR blocks. xin: device FP32, row v =
 * [x^o(N_max), y^o(N_max)] at offset 2 N_max v (first 2 N_v entries used). frames: device, 6 doubles
 * per vesicle (c_x, c_y, cos t, sin t, 1/L, first-point label). Synchronous.
 */
vs_status vs_standardize(const double* xy, const int64_t* offsets, int32_t M, int32_t kmax, float* xin,
                         double* frames, void* cuda_stream);

/*
 * Learned part (Sec. 3.2-3.4): a fully connected network (ReLU hidden layers, affine output)
 * evaluated and trained on the tensor cores with BF16 operands and FP32 accumulation.
 *  dims        host, nlayers+1 widths d_0 .. d_L, each a multiple of 16 in [16, 16384].
 *  max_batch   largest batch a call may pass.
 *  ncomp, beta the loss ||Yhat - Y||/||Y|| + beta ||D(Yhat - Y)||/||D Y|| averaged over the batch,
 *              D the periodic difference inside each of ncomp equal blocks of an output row
 *              (Sec. 3.4.2).
 * Parameters are one flat FP32 vector: every W_l (d_{l+1} x d_l, row-major), then every b_l.
 * x, y are DEVICE row-major FP32 (batch x d_0, batch x d_L). vs_mlp_forward / vs_mlp_train_step
 * are asynchronous on the handle's stream unless a host loss pointer is given. Errors: bad sizes
 * VS_ERR_INVALID_ARG; a tensor-core wait that runs out VS_ERR_TIMEOUT (reported on the next
 * synchronising call).
 */
typedef struct {
  float lr, beta1, beta2, eps, weight_decay;  /* AdamW (Sec. 3.4.2: lr 1e-3) */
} vs_adamw;
vs_status vs_mlp_create(const int32_t* dims, int32_t nlayers, int32_t max_batch, int32_t ncomp, float beta,
                        void* cuda_stream, vs_mlp** out);
vs_status vs_mlp_num_params(const vs_mlp* m, int64_t* n);
/* host FP32 parameters in / out; set also clears the AdamW moments */
vs_status vs_mlp_set_params(vs_mlp* m, const float* params, int64_t n);
vs_status vs_mlp_get_params(vs_mlp* m, float* params, int64_t n);
/*
 * Per-feature affine maps around the layers (feature normalisation of the training data, Sec. 3.4.2):
 * the first layer sees (x_j - in_shift_j) in_scale_j (FP32, then BF16), and the output is
 * z_j out_scale_j + out_shift_j for the last layer's value z. Training compares z with the targets
 * mapped the other way, (y_j - out_shift_j) (1/out_scale_j) in FP32, so the loss above is taken in
 * the normalised output coordinates. set: host arrays of d_0, d_0, d_L, d_L floats; a NULL shift
 * is 0 and a NULL scale 1; all four NULL removes both maps; a zero or non-finite value is
 * VS_ERR_INVALID_ARG. get: host arrays (each may be NULL). fit: in_shift / out_shift = column means
 * and in_scale = 1/sd, out_scale = sd of the DEVICE FP32 rows x (rows x d_0) and y (rows x d_L), FP64
 * sums, with sd raised to rel_floor times the largest deviation of its matrix (rel_floor >= 0; columns
 * whose spread is rounding noise then stay small) and 1 for a constant column; synchronises.
 */
vs_status vs_mlp_set_affine(vs_mlp* m, const float* in_shift, const float* in_scale, const float* out_shift,
                            const float* out_scale);
vs_status vs_mlp_get_affine(vs_mlp* m, float* in_shift, float* in_scale, float* out_shift, float* out_scale);
vs_status vs_mlp_fit_affine(vs_mlp* m, const float* x, const float* y, int32_t rows, double rel_floor);
/* y (device, batch x d_L) = network(x), output map included */
vs_status vs_mlp_forward(vs_mlp* m, const float* x, int32_t batch, float* y);
/* loss (host) and, when grad (host, n floats) is non-null, its gradient; synchronises */
vs_status vs_mlp_loss_grad(vs_mlp* m, const float* x, const float* y, int32_t batch, float* loss, float* grad,
                           int64_t n);
/* one AdamW step on the batch; loss (host) may be null to stay asynchronous */
vs_status vs_mlp_train_step(vs_mlp* m, const float* x, const float* y, int32_t batch, const vs_adamw* opt,
                            float* loss);
vs_status vs_mlp_sync(vs_mlp* m);
const char* vs_mlp_last_error(const vs_mlp* m);
void vs_mlp_destroy(vs_mlp* m);

/*
 * IVNet (Sec. 3.4.2, Fig. fig:net), the paper's network, for periodic 1D signals: a sample is in_channels
 * signals of a vesicle's N points (rows [s_0(N), s_1(N), ...], in_channels N floats: [x(N), y(N)] for two)
 * and the output two (rows [x(N), y(N)]). Architecture: a lifting convolution (k = 3, in_channels -> C
 * channels), nblocks blocks of two stride-2 restriction levels (each two paths of C/2 channels, dilations 1
 * and 2, concatenated), two periodic linear interpolations by 2 each followed by a convolution (k = 3),
 * the interpolations added to the descent's finer signals (r1, then the block's input), a mixing
 * convolution (k = 1) added to the block's input, and a projection (k = 1, C -> 2); ReLU after
 * every convolution but the mixing ones and the projection; all convolutions circular. Every convolution
 * runs as a BF16 tensor-core GEMM of its gathered input columns (FP32 accumulation). Loss, affine maps
 * and AdamW as for vs_mlp (ncomp = 2).
 *  vs_ivnet_create: N a multiple of 4 in [8, 128], in_channels in [1, 16], C a multiple of 32 in [32, 1024],
 *    nblocks >= 1, max_batch >= 1, beta >= 0 (the loss's derivative weight), stream as for vs_mlp_create.
 *  Parameters (host FP32, vs_ivnet_num_params of them): per convolution in the order lift, (R_1^1, R_1^2,
 *    R_2^1, R_2^2, I_1, I_2, C_m) per block, projection: W (C_out x C_in x k, row-major) then b (C_out).
 *    set also clears the AdamW moments.
 *  vs_ivnet_set_affine / vs_ivnet_fit_affine: per-feature maps of inputs (in_channels N) and outputs (2N) as
 *    for vs_mlp_set_affine / vs_mlp_fit_affine.
 *  vs_ivnet_forward: x (batch x in_channels N), y (batch x 2N) DEVICE FP32 rows, batch <= max_batch;
 *    asynchronous.
 *  vs_ivnet_loss_grad: loss (host) and, with grad non-NULL, the gradient (host, n = num_params); synchronous.
 *  vs_ivnet_train_step: one AdamW step on (x, y); loss (host) or NULL (then asynchronous).
 * vs_feature_points: samples of signals given by Fourier feature rows (modes <= K, the relaxation network's
 * layout, row stride ld) as rows [x(N), y(N)]; DEVICE FP32; asynchronous on cuda_stream.
 */
typedef struct vs_ivnet vs_ivnet;
vs_status vs_ivnet_create(int32_t N, int32_t in_channels, int32_t C, int32_t nblocks, int32_t max_batch, float beta,
                          void* cuda_stream, vs_ivnet** out);
vs_status vs_ivnet_num_params(const vs_ivnet* net, int64_t* n);
vs_status vs_ivnet_set_params(vs_ivnet* net, const float* params, int64_t n);
vs_status vs_ivnet_get_params(vs_ivnet* net, float* params, int64_t n);
vs_status vs_ivnet_set_affine(vs_ivnet* net, const float* in_shift, const float* in_scale, const float* out_shift,
                              const float* out_scale);
vs_status vs_ivnet_fit_affine(vs_ivnet* net, const float* x, const float* y, int32_t rows, double rel_floor);
vs_status vs_ivnet_forward(vs_ivnet* net, const float* x, int32_t batch, float* y);
vs_status vs_ivnet_loss_grad(vs_ivnet* net, const float* x, const float* y, int32_t batch, float* loss, float* grad,
                             int64_t n);
vs_status vs_ivnet_train_step(vs_ivnet* net, const float* x, const float* y, int32_t batch, const vs_adamw* opt,
                              float* loss);
vs_status vs_ivnet_sync(vs_ivnet* net);
const char* vs_ivnet_last_error(const vs_ivnet* net);
void vs_ivnet_destroy(vs_ivnet* net);
vs_status vs_feature_points(const float* feat, int32_t rows, int64_t ld, int32_t N, int32_t K, float* out,
                            void* cuda_stream);


/*
 * Far field without any device allocation (no counterpart in the paper; a deployment variant of
 * vs_farfield_eval). Some callers cannot call cudaMalloc: code running inside another
 * framework's memory pool or allocator, a host process that has handed all device memory to
 * someone else, or a real-time loop that must not allocate. This entry point computes the same
 * far-field sum as vs_farfield_eval with near_mask = 0 (every pair of different vesicles), but
 * keeps all of its scratch in one static device array of fixed size that is part of the library
 * image, so it calls no cudaMalloc / cudaFree and no allocating library routine.
 *  offsets      host, M+1 int64 (as in vs_create); at most VS_STATIC_MAX_VESICLES vesicles and
 *               VS_STATIC_MAX_POINTS points in total; N_v even in [8, 128]. Validated on the host,
 *               then copied to the device with cudaMemcpyAsync on cuda_stream: pageable memory may be
 *               reused once the call returns; page-locked memory must stay unchanged until the stream
 *               has executed the call.
 *  precision    0: compensated FP32, 1: FP64.
 *  xy, f        DEVICE, CSR blocks (2P doubles each); u DEVICE output (2P doubles, overwritten).
 *  cuda_stream  stream for all work (NULL = legacy default stream). Asynchronous.
 * Sizes beyond the limits, odd or out-of-range N, null pointers: VS_ERR_INVALID_ARG. A failed
 * launch or copy: VS_ERR_CUDA. The kernels have no data-dependent error conditions here (the near
 * test, whose list overflow is the far field's only one, is off), so there is no device error word
 * to read back.
 * The scratch array (about 13 MB) is reserved on every GPU that loads the library until the
 * process exits. The first call on a device does a one-time set-up on that device (looks up the
 * array's device address and fills its tables with one kernel); make that first call outside
 * any stream capture. All calls share the one array and it keeps the last call's contents:
 * calls that overlap on the GPU (different streams, or another host thread) race on it and must
 * be serialised by the caller.
 */
#define VS_STATIC_MAX_VESICLES 4096
#define VS_STATIC_MAX_POINTS 131072
vs_status vs_farfield_eval_static(const int64_t* offsets, int32_t M, double mu, int32_t precision,
                                  const double* xy, const double* f, double* u, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* VESB300_H */
