/*
 * sphere_bie.h -- C interface of the GB300 (sm_103a) library for the spectral
 * boundary integral method for N rigid spheres in Stokes flow
 * (Corona & Veerapaneni, arXiv:1707.06551).
 *
 * Conventions shared by every call
 *   - Viscosity is 1 (Sec. 5, Eq. 5.1).
 *   - Each sphere k (centre c_k, radius a_k) carries the (p+1) x (2p+2) grid of
 *     Eq. 4.2: Gauss-Legendre nodes t_j in cos(theta), j = 0..p, ordered from the
 *     north pole (theta ascending), and phi_k = 2 pi k / (2p+2).  Node order is
 *     sphere-major, then latitude j, then longitude k; the node count is
 *     N = n_spheres (p+1)(2p+2).
 *   - Densities and nodal outputs are arrays of N x 3 doubles (x, y, z per node,
 *     row-major).  Per-sphere quantities are n_spheres x 3 doubles.
 *   - Memory: with opts.mem_kind = 0 every pointer argument is host memory; the
 *     library copies in and out and returns after the result is on the host.
 *     With mem_kind = 1 the data pointers of apply/solve calls are device
 *     pointers on the current CUDA device; work is ordered on opts.stream (or
 *     the context's own stream if NULL) and the call returns when the result is
 *     in place (the stream is synchronised).  Geometry passed to
 *     sphere_bie_create is always host memory.
 *   - Ownership: the caller owns every array it passes; the context owns all of
 *     its device memory and frees it in sphere_bie_destroy.
 *   - Errors: every call returns sbie_status; SBIE_OK == 0.  No exception or
 *     CUDA error crosses the interface.  sphere_bie_last_error(ctx) returns a
 *     message for the last failure on that context (a static string for NULL).
 *     Nothing on any path falls back to the CPU.
 *   - Threads: calls on one context must not overlap (a context holds one
 *     stream, its work buffers and its captured GMRES cycles); different
 *     contexts may be used from different host threads.
 */
#ifndef SPHERE_BIE_H
#define SPHERE_BIE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sbie_ctx sbie_ctx;

typedef enum {
    SBIE_OK = 0,
    SBIE_ERR_ARG = 1,           /* bad argument (size, p, radius, NULL pointer, NaN) */
    SBIE_ERR_OVERLAP = 2,       /* two spheres overlap or touch (gap <= 0)          */
    SBIE_ERR_CUDA = 3,          /* a CUDA runtime call failed                        */
    SBIE_ERR_OOM = 4,           /* device allocation failed                          */
    SBIE_ERR_NOT_CONVERGED = 5, /* solve stopped at max_iter; outputs still filled   */
    SBIE_ERR_TIMEOUT = 6,       /* a bounded device wait gave up                     */
    SBIE_ERR_NUMERIC = 7        /* NaN/Inf met in a solve                            */
} sbie_status;

typedef enum {
    SBIE_FP64 = 0,    /* every kernel in native FP64                                  */
    SBIE_MIXED = 1,   /* GMRES on an operator whose far field and close-pair
                         evaluation run in FP32 (compensated accumulation), inside
                         iterative refinement on the FP64-accurate operator of
                         SBIE_FP64_DF; tables, coefficients and Arnoldi in FP64.
                         The first residual is b - A x with the FP64-accurate
                         operator; a later one is r - A d with the FP32 operator
                         when e ||d|| <= 0.1 tol ||x||, e = 10 x the FP32
                         operator's relative error measured on A x at the first
                         residual, clamped to [1e-6, 2e-5]; else b - A x again.  */
    SBIE_FP64_DF = 2  /* FP64-accurate operator whose far-field pair arithmetic is
                         double-float (a value = sum of two FP32 numbers, about 48
                         significant bits; ~1e-13 relative); everything else FP64   */
} sbie_precision;

typedef enum {
    SBIE_OP_S = 0,          /* sum_k S_k: single layer, Eq. 2.21; self by Theorem 2           */
    SBIE_OP_D = 1,          /* sum_k D_k: double layer, Eq. 2.21, self = principal value        */
    SBIE_OP_K = 2,          /* sum_k K_k: traction of the single layer, Eq. 2.22, self = PV     */
    SBIE_OP_MOBILITY = 3,   /* 1/2 I + sum_k (K_k + L_k), the mobility BIE operator, Eq. 5.8     */
    SBIE_OP_RESISTANCE = 4, /* 1/2 I + sum_k (D_k + N_k), completed double layer, Eq. 5.19       */
    SBIE_OP_POROUS = 5,     /* 1/2 I + sum_k (S_k + D_k), porous-media flow, Eq. 5.4              */
    SBIE_OP_SQUIRMER = 6    /* (1/2 I + sum_k (S_k + D_k)) (I - P) - P: Eq. 5.17 with the force-
                               and torque-free conditions of Eq. 5.15 in square form; P mu is,
                               on each sphere, the rigid field F/(4 pi a^2) + 3/(8 pi a^4) T x
                               (x - c_k) with F = int mu, T = int (y - c_k) x mu             */
} sbie_op;

typedef struct {
    int p;                  /* VSH order (Sec. 2.1); 1 <= p <= 24                              */
    double eta;             /* close-pair parameter of Eq. 4.5: spheres i != k are "near" when
                               |c_i - c_k| - a_i - a_k < eta * max(2 a_i, 2 a_k); default 1.0   */
    int prec;               /* sbie_precision                                                  */
    double tol;             /* GMRES stop: ||b - A x||_2 / ||b||_2 <= tol (nodal l2)            */
    int restart;            /* GMRES restart length                                            */
    int max_iter;           /* total GMRES iterations allowed                                  */
    int use_learned_precond;/* 0 none; 1 pair network (mlp_weights_path); 2 exact pair blocks */
    const char* mlp_weights_path; /* pair-network file written by sphere_bie_train_pair_network */
    int mem_kind;           /* 0 host pointers, 1 device pointers                              */
    void* stream;           /* cudaStream_t for mem_kind = 1, or NULL                          */
    int use_graphs;         /* 1: each GMRES restart cycle runs on the device as one CUDA
                               graph launch (a WHILE node over the Arnoldi iteration, no host
                               round trip per iteration); 0: the same device iteration stepped
                               from the host.  Profiling (sphere_bie_profile) always steps.    */
    int near_scheme;        /* close pairs: 0 direct evaluation of the exterior expansions at the
                               target nodes (Sec. 4.1); 1 the rotated, FFT-accelerated scheme of
                               Sec. 4.2 (Fig. 2: source coefficients rotated to the pair's
                               pole, evaluation on the target's pole-aligned grid, forward
                               transform, rotation back), which projects the close-pair field
                               onto degree <= p on the target sphere                          */
} sbie_opts;

typedef struct {
    int iters;              /* inner GMRES iterations (all restarts / refinements)             */
    int restarts;
    int refinements;        /* outer FP64 residual corrections (SBIE_MIXED)                    */
    double rel_residual_true; /* ||b - A x|| / ||b|| recomputed with the FP64 operator        */
    double t_setup_ms;      /* wall time of the context's create, preconditioner included      */
    double t_solve_ms;      /* wall time of this solve call                                    */
    long long n_near_pairs; /* directed close pairs (i, k)                                     */
    int graph_cycles;       /* restart cycles that ran as one CUDA graph launch each            */
    long long kernel_launches; /* kernels this call executed (those inside graphs included)     */
    int fp32_residual_updates; /* SBIE_MIXED: residuals formed as r - A d with the FP32 operator
                                  because the correction d was small enough (see SBIE_MIXED)  */
    double fp32_op_err;     /* SBIE_MIXED: measured ||A64 x - A32 x|| / ||A64 x|| at the first
                               FP64-accurate residual (worst problem)                        */
    double last_correction; /* SBIE_MIXED: ||d|| / ||x|| of the last correction (worst problem) */
} sbie_solve_info;

/* Fills *opts with defaults: p = 8, eta = 1, FP64, tol = 1e-8, restart = 60,
 * max_iter = 600, host memory, NULL stream, graphs on. */
sbie_status sphere_bie_default_opts(sbie_opts* opts);

/* Builds the grid (Eq. 4.2), smooth weights (Eq. 4.4), close-pair lists
 * (Eq. 4.5) and device tables for n_spheres spheres.  centres: host [n][3],
 * radii: host [n].  Fails with SBIE_ERR_OVERLAP on overlapping spheres and
 * SBIE_ERR_ARG on bad sizes.  On success *out owns all device memory. */
sbie_status sphere_bie_create(int n_spheres, const double* centres, const double* radii,
                              const sbie_opts* opts, sbie_ctx** out);

/* A batch of independent problems (suspensions) in one context: problem q has
 * n_spheres[q] spheres and VSH order p_per_problem[q] (opts->p is ignored);
 * centres [sum n][3] and radii [sum n] are the problems' arrays concatenated
 * in problem order (host memory).  Nodes, densities and per-sphere arrays of
 * every later call are likewise concatenated in problem order.  Close pairs
 * (Eq. 4.5) and the far field (Eq. 4.4) never couple different problems, and
 * a solve runs one GMRES per problem (each to opts->tol) with one operator
 * launch sequence per distinct p serving all problems of that order.
 * sphere_bie_create is this call with one problem. */
sbie_status sphere_bie_create_batch(int n_problems, const int* n_spheres, const int* p_per_problem,
                                    const double* centres, const double* radii, const sbie_opts* opts,
                                    sbie_ctx** out);

/* Number of quadrature nodes N = sum over spheres of (p+1)(2p+2). */
sbie_status sphere_bie_num_nodes(const sbie_ctx* ctx, long long* n_nodes);

/* Host copies of node positions, outward normals ([N][3] each) and smooth
 * quadrature weights ([N], Eq. 4.4).  Any pointer may be NULL to skip it. */
sbie_status sphere_bie_nodes(const sbie_ctx* ctx, double* xyz, double* normals, double* weights);

/* out = A density for the chosen operator, at every node (Sec. 4.3): self term
 * by VSH analysis, signature and synthesis (Sec. 4.1, Theorem 2); far field by
 * the smooth quadrature of Eq. 4.4 over well-separated spheres; close pairs by
 * the exterior expansions of Eqs. 3.6-3.11 and the traction of Eq. 3.18.
 * density, out: [N][3]; host or device per opts.mem_kind; must not alias.
 * Precision per opts.prec. */
sbie_status sphere_bie_apply_operator(sbie_ctx* ctx, sbie_op op, const double* density, double* out);

/* For a batch the solve outputs are per problem, concatenated; info reports
 * the total inner iterations and the worst true residual over problems. */

/* Mobility problem (Problem 2, Eqs. 5.5-5.8): given force F_k and torque T_k
 * on each sphere ([n][3] each), solve (1/2 I + K + L) mu = -(1/2 I + K) rho
 * with rho_k = F_k / (4 pi a^2) + 3 / (8 pi a^4) T_k x (x - c_k), evaluate
 * u = S[mu + rho] on every sphere and return its rigid part: vel_k =
 * int u / (4 pi a^2) and omega_k = 3 / (8 pi a^4) int (x - c_k) x u.
 * info may be NULL.  Returns SBIE_ERR_NOT_CONVERGED (outputs still filled)
 * when the tolerance is not met within max_iter. */
sbie_status sphere_bie_solve_mobility(sbie_ctx* ctx, const double* forces, const double* torques,
                                      double* vel, double* omega, sbie_solve_info* info);

/* Resistance problem (Problem 5, Eqs. 5.18-5.19): given rigid motions
 * (vel_k, omega_k) and an optional background flow u_inf(x) = u0 + G x
 * (bg_u0: [3] or NULL; bg_grad: G as [3][3] row-major or NULL), solve
 * (1/2 I + D + N) psi = vel_k + omega_k x (x - c_k) - u_inf(x) and return
 * forces F_k = int psi and torques T_k = int (y - c_k) x psi (the force and
 * torque each sphere exerts on the fluid).  bg_u0 / bg_grad are host memory
 * for either mem_kind. */
sbie_status sphere_bie_solve_resistance(sbie_ctx* ctx, const double* vel, const double* omega,
                                        const double* bg_u0, const double* bg_grad,
                                        double* forces, double* torques, sbie_solve_info* info);

/* Porous-media flow (Problem 1, Eqs. 5.3-5.4): fixed spheres in the imposed
 * flow u_inf(x) = u0 + G x (bg_u0: [3] or NULL; bg_grad: G as [3][3]
 * row-major or NULL; host memory for either mem_kind).  Solves
 * (1/2 I + S + D) mu = -u_inf and returns forces F_k = int mu and torques
 * T_k = int (y - c_k) x mu ([n][3] each: what each sphere exerts on the fluid;
 * the double layer carries none); the flow is u = u_inf + (S + D) mu.  The
 * pair preconditioner is not used for this operator.  info may be NULL;
 * SBIE_ERR_NOT_CONVERGED (outputs filled) when max_iter is reached. */
sbie_status sphere_bie_solve_porous(sbie_ctx* ctx, const double* bg_u0, const double* bg_grad, double* forces,
                                    double* torques, sbie_solve_info* info);

/* Active particles (Problem 4, Eqs. 5.14-5.17): force- and torque-free spheres
 * with a prescribed slip velocity.  slip: [N][3] nodal u_s at the nodes in
 * sphere_bie_nodes order (memory kind of the context).  Solves the square form
 * (1/2 I + S + D)(mu - P mu) - P mu = u_s (SBIE_OP_SQUIRMER): mu - P mu is the
 * density of u = (S + D)(mu - P mu) (Eq. 5.16), its force and torque on every
 * sphere vanish (Eq. 5.15), and P mu = vel_k + omega_k x (x - c_k) is each
 * sphere's rigid velocity, returned as vel_k = int mu / (4 pi a^2) and
 * omega_k = 3 / (8 pi a^4) int (y - c_k) x mu ([n][3] each).
 * sphere_bie_solution_density then returns mu - P mu.  The pair
 * preconditioner is not used.  info may be NULL. */
sbie_status sphere_bie_solve_squirmer(sbie_ctx* ctx, const double* slip, double* vel, double* omega,
                                      sbie_solve_info* info);

/* Laplace layer operators (Sec. 2.2, Eq. 2.18) on a scalar nodal density q
 * ([N], sphere_bie_nodes order, memory kind of the context) of a single-order
 * context: op 0 the single layer S^L, 1 the double layer D^L, 2 the flux
 * K^L = n(x) . grad S^L (Sec. 3.3, Eq. 3.16), each summed over all spheres:
 * self term by Theorem 1 (Eq. 3.5; D^L and K^L as principal values, both
 * -1/(2(2n+1)); S^L times the radius), smooth quadrature (Eq. 4.4) between
 * separated spheres, the exterior expansions of Eqs. 3.3-3.4 for close pairs.
 * FP64 in every precision mode.  out: [N], must not alias q.  SBIE_ERR_ARG for
 * another op or a batch context. */
sbie_status sphere_bie_apply_laplace(sbie_ctx* ctx, int op, const double* q, double* out);

/* Paramagnetic spheres in a uniform field (Problem 3, Eqs. 5.9-5.13) moving
 * in Stokes flow: solves (1/2 I + eta K^L) q = eta H0 . n for the single-layer
 * density of phi = -H0 . x + S^L[q] (eta = (mu - mu0)/(mu + mu0), -1 < eta < 1;
 * H0: [3] host memory), forms the field H = H0 - grad S^L[q] outside each
 * sphere and its Maxwell traction f = (H . n) H - |H|^2 n / 2 (mu0 = 1), and
 * solves the mobility problem (Eq. 5.8) with f as the incident force density.
 * Returns the magnetic force F_k = int f and torque T_k = int (x - c_k) x f on
 * each particle and its rigid motion (vel_k, omega_k) ([n][3] each, memory kind
 * of the context).  info (may be NULL) sums the iterations of both solves and
 * reports the worse of their true residuals.  Single-order contexts only
 * (SBIE_ERR_ARG for a batch); the magnetic solve runs in FP64. */
sbie_status sphere_bie_solve_mhd(sbie_ctx* ctx, const double* H0, double eta, double* forces, double* torques,
                                 double* vel, double* omega, sbie_solve_info* info);

/* Stage timing.  Stages: 0 far field (density pack, pair kernel and split
 * reduction), 1 close pairs (Sec. 4.1), 2 self term (analysis, signature,
 * synthesis), 3 completion / rigid-mode terms and 1/2 I, 4 Arnoldi vector
 * work, 5 the pair preconditioner's apply, 6 the FP32 far-field pair kernel alone, 7 the FP64 far-field
 * pair kernel alone.  ms[s] is the total device time between CUDA events
 * recorded on the context stream around each launch of that stage;
 * launches[s] counts them.  far_pairs_f32 / _f64 count the (target node,
 * source node) kernel evaluations of the far-field launches in each
 * precision; kernel_launches counts every CUDA kernel the context launched. */
typedef struct {
    double ms[8];
    long long launches[8];
    long long far_pairs_f32, far_pairs_f64;
    long long kernel_launches;
    long long arnoldi_vectors; /* algorithmic 3N-vector accesses of the profiled
                                  Arnoldi iterations: 4k + 4 for an iteration
                                  with k basis vectors (two Gram-Schmidt passes,
                                  the new vector's norm and scaling)           */
} sbie_profile;

/* Tiling of the FP32 far-field pair kernel (Sec. 4.1 smooth quadrature). */
typedef struct {
    int threads;             /* threads per CTA                                   */
    int targets_per_thread;  /* target nodes per thread (held in FP32 pairs)      */
    int split;               /* source-range splits (partial sums added in order) */
    int tile;                /* sources staged in shared memory per tile          */
    double ms;               /* measured time of one launch with this tiling and  *
                              * the reduction of its partial sums                 */
    int candidates;          /* tilings timed                                     */
    int min_blocks;          /* FP32 build for 64-thread CTAs requiring 8, 10 or 16 resident
                                CTAs per SM (about 128, 96, 64 registers); 0: no register cap */
} sbie_far_tuning;

/* Autotuner: times every admissible tiling of the far-field kernels used by
 * `op` (SBIE_OP_S, _D or _K; _MOBILITY tunes K, _RESISTANCE tunes D) in the
 * context's precision -- the FP32 kernel (SBIE_MIXED) and the double-float
 * kernel (SBIE_MIXED, SBIE_FP64_DF) -- on this context's geometry with CUDA
 * events, keeps the fastest for this context and caches it for later contexts
 * of the same (n_spheres, p, SM count) in this process.  chosen, if not NULL,
 * points to two records: [0] FP32 kernel, [1] double-float kernel (zeroed when
 * not tuned).  SBIE_FP64 contexts keep their default tiling. */
sbie_status sphere_bie_autotune(sbie_ctx* ctx, sbie_op op, sbie_far_tuning* chosen);

/* enable != 0 starts recording (and resets the counters); 0 stops.  While
 * recording, solves step their GMRES cycles from the host so that every stage
 * can be timed.  SBIE_ERR_ARG for a NULL context. */
sbie_status sphere_bie_profile(sbie_ctx* ctx, int enable);
/* Synchronises the context stream and writes the totals since the last reset
 * to *out (host memory, owned by the caller).  SBIE_ERR_ARG for NULL. */
sbie_status sphere_bie_profile_read(sbie_ctx* ctx, sbie_profile* out);

/* Raw layer operator without any device allocation.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc (a memory
 * manager owns the device, or allocation is banned inside their hot loop).
 * Computes out = sum_k S_k, D_k or K_k (op = SBIE_OP_S, _D or _K) in FP64 at
 * every node: what sphere_bie_apply_operator returns for that op on a context
 * created with eta = 0 (self term plus the far field over every other sphere,
 * no close-pair correction).  centres [n][3], radii [n], density and out [N][3]
 * (N = n_spheres (p+1)(2p+2)) must be device (or managed) memory of the
 * current device -- anything else returns SBIE_ERR_ARG before any work is
 * queued; work runs on `stream` (a cudaStream_t or NULL) and the call returns
 * when out is complete.
 * Limits: 1 <= n_spheres <= 4096, 1 <= p <= 24, N <= 65536; larger sizes
 * return SBIE_ERR_ARG with a message.  All intermediates live in one static
 * 20 MiB __device__ array that every GPU loading this library holds until
 * exit; no cudaMalloc, cudaFree or allocating library routine is called.  The
 * first call on a device looks up that array's address (and uploads the
 * Legendre tables for its p), so make it before any stream capture.  Every
 * call shares the array, which keeps the last call's contents: calls whose
 * work overlaps on the GPU (different streams or host threads) race. */
sbie_status sphere_bie_apply_layer_noalloc(sbie_op op, int n_spheres, int p, const double* centres,
                                           const double* radii, const double* density, double* out,
                                           void* stream);

/* ---- learned pair preconditioner ------------------------------------------
 * With opts.use_learned_precond = 1 (networks read from opts.mlp_weights_path
 * at create) or 2 (exact blocks), the first resistance or mobility solve on a
 * context builds a right preconditioner for GMRES on that operator:
 *   M^{-1} r = H r + Z C^{-1} Z^+ r,
 * Z^+ the VSH analysis restricted to degree <= 4 (73 real coefficients per
 * sphere), H the exact inverse of each sphere's own operator above degree 4
 * (1/D+ = 1/K- of Theorem 2, and 2 on the non-band-limited remainder), C^{-1}
 * an additive Schwarz inverse over close pairs of the low-mode pair systems
 * [[L_i, B_ik], [B_ki, L_k]] of that operator (L probed exactly; B probed
 * exactly, or for 1 predicted by the pair network in the pair frame and
 * rotated).  The operator and the true residual are unchanged: the
 * preconditioner changes the iteration count, not the answer.  A weights file
 * without a network for the solve's operator leaves that solve
 * unpreconditioned. */

typedef struct {
    int n_samples;         /* two-sphere configurations generated (>= 16)          */
    int p;                 /* VSH order of the probed grid (4..24)                 */
    double gap_min, gap_max; /* surface gaps, log-uniform                          */
    double radius;         /* both radii, or the lower end of their range          */
    int epochs, batch;
    double lr;             /* Adam learning rate                                   */
    unsigned long long seed;
    double val_frac;       /* held-out fraction for the validation error           */
    int ops;               /* networks to train: bit 0 resistance blocks (Eq. 5.19),
                              bit 1 mobility blocks (Eq. 5.8); one file holds both  */
    double radius_max;     /* > radius: each radius uniform in [radius, radius_max];
                              0 or radius: fixed radius                             */
} sbie_pair_train_opts;

typedef struct {
    double train_loss;     /* mean squared error of the last epoch (standardised; worst network) */
    double val_rel_err;    /* mean relative Frobenius error of held-out blocks (worst network)   */
    double t_data_s, t_train_s;  /* block generation and training, all networks   */
    int n_train, n_val;
} sbie_pair_train_info;

/* Generates exact pair-frame low-mode blocks of two-sphere configurations
 * (probing the close-pair path of the operator on the GPU), trains the pair
 * network on them with the library's own kernels, and writes it to path (the
 * file a context reads through opts.mlp_weights_path).  info may be NULL.
 * SBIE_ERR_ARG for out-of-range options (checked before any device work),
 * SBIE_ERR_CUDA / SBIE_ERR_OOM for device failures, SBIE_ERR_ARG if path cannot
 * be written. */
sbie_status sphere_bie_train_pair_network(const sbie_pair_train_opts* opts, const char* path,
                                          sbie_pair_train_info* info);

/* Exact pair-frame blocks: source of radius a_src at the origin, target of
 * radius a_tgt at (0, 0, dist[q]); blocks: host [n][73][73] (target row,
 * source column) of operator op (SBIE_OP_RESISTANCE or SBIE_OP_MOBILITY),
 * grid order p.  All arrays are host memory owned by the caller.  SBIE_ERR_ARG
 * for n < 1, NULL arrays, p outside [4, 24], another operator, a radius <= 0
 * or spheres that touch or overlap (dist <= a_src + a_tgt), all before any
 * device work. */
sbie_status sphere_bie_pair_blocks(int n, const double* dist, const double* a_src, const double* a_tgt, int p,
                                   sbie_op op, double* blocks);

/* Density of the last solve on ctx, at the nodes in sphere_bie_nodes order
 * ([N][3], memory kind of the context): psi of Eq. 5.19 after a resistance
 * solve, mu of Eq. 5.8 after a mobility solve.  SBIE_ERR_ARG before any solve. */
sbie_status sphere_bie_solution_density(sbie_ctx* ctx, double* density);

/* Pair preconditioner of a context for operator op (SBIE_OP_RESISTANCE or
 * SBIE_OP_MOBILITY): kind (0 none or not yet built, 1 network, 2 exact),
 * undirected pairs in the pair systems, close pairs left out because they lie
 * outside the network's trained input range (kind 1), and the wall time of
 * its setup (inside the first solve with op).  Output pointers may be NULL. */
sbie_status sphere_bie_precond_info(const sbie_ctx* ctx, sbie_op op, int* kind, int* n_pairs, int* n_dropped,
                                    double* setup_ms);

/* Number of network parameters (FP32, layer by layer: W1 (5x128), b1, ...).
 * SBIE_ERR_ARG for NULL. */
sbie_status sphere_bie_pair_network_size(long long* n_params);

/* Loss (mean squared error over all outputs) and its gradient for raw
 * network inputs X [n][5] and targets Y [n][5329], with the weights rounded to
 * BF16 as in training; params and grads hold sphere_bie_pair_network_size
 * floats.  All arrays are host memory owned by the caller.  SBIE_ERR_ARG for
 * NULL arrays or n < 1 (before any device work). */
sbie_status sphere_bie_pair_network_gradients(const float* params, int n, const float* X, const float* Y,
                                              float* grads, double* loss);

/* Measured FP32 throughput of this GPU (no counterpart in the paper): the
 * best of three timed launches of a kernel of independent packed FP32x2 FMA
 * chains (the far-field kernel's instruction) filling every SM, on the current
 * device.  *tflops: TFLOP/s (an FMA counts 2); *ms (may be NULL): the launch
 * time.  Allocates and frees a small buffer.  SBIE_ERR_ARG for NULL tflops,
 * SBIE_ERR_CUDA on a device failure. */
sbie_status sphere_bie_fp32_peak_probe(double* tflops, double* ms);

/* Frees every device buffer and the context.  NULL is accepted. */
sbie_status sphere_bie_destroy(sbie_ctx* ctx);

/* Message for the last failure on ctx (or the last create failure if ctx is NULL). */
const char* sphere_bie_last_error(const sbie_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SPHERE_BIE_H */
