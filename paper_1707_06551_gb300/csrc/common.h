// Internal declarations of the sphere BIE library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "../../include/sphere_bie.h"

namespace sbie {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxP = 24;

enum class Kern { S = 0, D = 1, K = 2 };

// Arithmetic of one operator apply: FP64 everywhere; FP32 far field and
// close-pair evaluation; FP64 with the far field in double-float arithmetic.
constexpr int kModeF64 = 0, kModeF32 = 1, kModeDF = 2;

// Offsets into the packed FP64 table of one order p (device copy in Ctx::tab).
struct TabLayout {
    int p, nlat, nlon, npn;
    int o_ct, o_st, o_w;       // [nlat]   cos theta_j, sin theta_j, 2 pi lambda_j / (2p+2)
    int o_cph, o_sph;          // [nlon]   cos phi_k, sin phi_k
    int o_cmk, o_smk;          // [p+1][nlon] cos(m phi_k), sin(m phi_k)
    int o_P, o_dP, o_mS;       // [p+1 (m)][p+1 (n)][nlat]: Pbar_n^m, d/dtheta Pbar_n^m, m Pbar_n^m / sin
    int total;
};

constexpr TabLayout tab_layout(int p) {
    TabLayout t{};
    t.p = p;
    t.nlat = p + 1;
    t.nlon = 2 * p + 2;
    t.npn = t.nlat * t.nlon;
    int o = 0;
    t.o_ct = o; o += t.nlat;
    t.o_st = o; o += t.nlat;
    t.o_w = o; o += t.nlat;
    t.o_cph = o; o += t.nlon;
    t.o_sph = o; o += t.nlon;
    t.o_cmk = o; o += (p + 1) * t.nlon;
    t.o_smk = o; o += (p + 1) * t.nlon;
    const int leg = (p + 1) * (p + 1) * t.nlat;
    t.o_P = o; o += leg;
    t.o_dP = o; o += leg;
    t.o_mS = o; o += leg;
    t.total = o;
    return t;
}
// Fills host table (size layout.total) for order p: Gauss-Legendre grid and
// normalised associated Legendre functions (normalised recurrences).
void build_tables(int p, std::vector<double>& host);
// Degree blocks of f -> f o R_x(+90 deg) (Mp) and f -> f o R_x(-90 deg) (Mm) on
// the spherical harmonics (tables.cu)
void rotx90_tables(int p, std::vector<double>& Mp, std::vector<double>& Mm);

// Real solid-harmonic basis used by the close-pair kernels: functions
// Re/Im J_nm, J_nm = P_n^m(cos th) e^{i m ph} / r^{n+1} (no Condon-Shortley),
// ordered m-major: for m = 0..L, for n = m..L: Re (m >= 1: Re, Im).
__host__ __device__ inline int sh_offset_m(int L, int m) {
    // entries before order m
    if (m == 0) return 0;
    // (L+1) for m = 0, then 2 (L+1-mm) for mm = 1..m-1
    return (L + 1) + 2 * ((m - 1) * (L + 1) - (m - 1) * m / 2);
}
__host__ __device__ inline int sh_index(int L, int n, int m, int part) {
    if (m == 0) return n;
    return sh_offset_m(L, m) + 2 * (n - m) + part;
}
__host__ __device__ inline int sh_count(int L) { return (L + 1) * (L + 1); }

// Channels per close-pair source expansion.
constexpr int kVelChannels = 10;   // grad Pa (3), grad Pb (3), Pc (1), grad Pd (3)
constexpr int kTracChannels = 26;  // hess Pa (6), grad Pb (3), hess Pb (6), Pc (1), grad Pc (3), hess Pd (6), Pe (1)
constexpr int kLapChannels = 6;    // Laplace: Phi_S, grad Phi_S (3), Phi_D, one zero (even width)

// Laplace operators (laplace.cu) on scalar densities held in component 0 of [N][3]:
// single layer, double layer, flux of the single layer, exterior gradient of the single layer.
constexpr int kLapSL = 0, kLapDL = 1, kLapKL = 2, kLapGrad = 3;

struct FarTune {
    int threads;  // threads per CTA (multiple of 32)
    int tpt;      // targets per thread (1, 2 or 4)
    int split;    // source-range splits (partial sums reduced afterwards)
    int tile;     // sources staged per tile
    int minb = 0; // FP32 kernel, 64 threads: build requiring 8, 10 or 16 resident CTAs per SM (0: no cap)
};

struct Profile {
    bool on = false;
    double ms[8] = {0};
    long long launches[8] = {0};
    long long pairs_f32 = 0, pairs_f64 = 0;
    long long arnoldi_vectors = 0;  // sum of 4k + 4 over profiled Arnoldi iterations
    long long kernels0 = 0;  // kernel-launch counter at the last reset
};
enum Stage {
    ST_FAR = 0, ST_NEAR = 1, ST_SELF = 2, ST_COMPL = 3, ST_BLAS = 4, ST_OTHER = 5,
    ST_FARK32 = 6, ST_FARK64 = 7  // the far-field pair kernel alone
};

// Device state of one GMRES restart cycle (krylov.cu), for P problems and at
// most m iterations.  Passed by value to the kernels.
constexpr int kStWords = 8;  // words of ArnoldiDev::st
struct ArnoldiDev {
    int m = 0, P = 0;
    int* st = nullptr;        // [kStWords] k, iteration limit, continue flag, non-finite flag, any live
    int* live = nullptr;      // [P] problem still iterating
    int* kd = nullptr;        // [P] columns of the problem's Hessenberg matrix
    double* nb = nullptr;     // [P] norm of the right-hand side
    double* tol = nullptr;    // [P] relative tolerance
    double* H = nullptr;      // [P][m+1][m] rotated Hessenberg matrix
    double* cs = nullptr;     // [P][m] Givens cosines
    double* sn = nullptr;     // [P][m] Givens sines
    double* g = nullptr;      // [P][m+1] rotated right-hand side of the least-squares problem
    double* h1 = nullptr;     // [m+1][P] first Gram-Schmidt pass
    double* h2 = nullptr;     // [m+1][P] second pass
    double* nrm = nullptr;    // [P] squared norm of the new vector
    double* scale = nullptr;  // [P] 1 / its norm (0 once the problem stopped)
    double* y = nullptr;      // [m][P] least-squares solution of the cycle
    double* w = nullptr;      // [3N] new Krylov vector (fixed address for the captured operator)
    double* pack = nullptr;   // [4P+1] cycle inputs staged from the host: nb, tol, beta, active, limit
};

// One restart cycle captured as a CUDA graph (a WHILE node whose body is one
// Arnoldi iteration), for one operator / arithmetic / preconditioner choice.
struct CycleGraph {
    int key = -1;
    unsigned long long epoch = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long body_launches = 0;
};

// Pair preconditioner of one operator of a context (slot 0: resistance,
// Eq. 5.19; slot 1: mobility, Eq. 5.8), built at the first solve with it.
struct PrecState {
    int kind = 0;              // 0 none, 1 pair network, 2 exact pair blocks
    bool built = false;        // set up, or found unavailable, for this operator
    int n_pairs = 0;           // undirected pairs in the pair systems
    int n_dropped = 0;         // close pairs outside the network's trained range
    double setup_ms = 0.0;
    int* d_pp_ptr = nullptr;   // [n+1] per-sphere lists of the pairs
    int* d_pp_idx = nullptr;   // partner sphere
    int* d_pp_pair = nullptr;  // pair index into d_pinv
    float* d_pinv = nullptr;   // [n_pairs][146][146] inverses of the pair systems
    float* d_sinv = nullptr;   // [n][73][73] inverses of the spheres' own low-mode blocks
    int n_entries = 0;         // entries of the per-sphere pair lists (2 n_pairs)
    int* d_pp_own = nullptr;   // [n_entries] sphere owning each entry (FP32 coarse correction)
    float* d_cpart = nullptr;  // [n_entries][73] per-entry products of the FP32 coarse correction
};
constexpr int prec_slot(int op) { return op == SBIE_OP_MOBILITY ? 1 : 0; }

struct PairNetSet;  // trained pair networks (api.cu)

// Self-kernel signature of the pair preconditioner's high-mode part: 1/D+
// above degree 4 (the exterior eigenvalues of Theorem 2), 0 at or below, minus 2.
constexpr int kOpPrecHigh = 3;

// Self-term matrices of the FP32 operator applied by the tensor-core GEMM
// (selfgemm.cu): single layer (unit radius), double layer = traction
// (principal value), and the pair preconditioner's H with the low-mode rows.
constexpr int kSelfS = 0, kSelfDK = 1, kSelfPrec = 2, kSelfMats = 3;
struct SelfGemm;

}  // namespace sbie

struct sbie_ctx {
    int n = 0, p = 0, nlat = 0, nlon = 0, npn = 0;
    long long N = 0;
    sbie_opts opts{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int sm_count = 0;
    std::string err;

    // problems held by this context (a batch of independent suspensions with
    // one VSH order): spheres h_prob_sph[q] .. h_prob_sph[q+1]-1 form problem q
    int n_prob = 1;
    std::vector<int> h_prob_sph;
    int* d_prob_sph = nullptr;   // [n_prob+1]
    int* d_sph_prob = nullptr;   // [n] problem of each sphere

    // a batch of problems with several VSH orders: one part per distinct p
    bool is_batch = false;
    std::vector<sbie_ctx*> parts;
    std::vector<long long> part_off3;   // offset of each part in the batch vector (doubles)
    std::vector<int> prob_part, prob_local;  // user problem -> (part, problem within part)
    std::vector<long long> prob_user_node, prob_user_sph;  // user offsets (nodes, spheres)
    std::vector<long long> seg3;        // problem segments of the internal vector (doubles), internal order
    int* d_node_prob = nullptr;         // internal node -> internal problem index
    long long* d_seg3 = nullptr;        // device copy of seg3
    double* d_H = nullptr;              // [restart+1][n_prob_total] small device matrix
    double* d_pvec = nullptr;           // [n_prob_total] per-problem scalars
    size_t red_cap = 0, hred_cap = 0;

    // pair preconditioner (precond.cu), per operator; the low-mode tables and
    // work vectors are shared by both operators
    sbie::PrecState prec[2];
    std::shared_ptr<sbie::PairNetSet> nets;  // networks of opts.mlp_weights_path (top context)
    double* d_ZS = nullptr;        // [npn][3][73] low-mode synthesis
    float* d_ZSf = nullptr;        // the same in FP32 (mixed-precision contexts)
    double* d_ZA = nullptr;        // [73][npn][3] low-mode analysis
    int4* d_modes = nullptr;       // [73] (type, n, m, part)
    double* d_low = nullptr;       // [n][73]
    double* d_lowe = nullptr;      // [n][73]
    double* d_pz = nullptr;        // preconditioned vector (system level)
    double* d_sq = nullptr;        // [2][3N] squirmer operator: mu - P mu and P mu
    double* d_lcoef = nullptr;     // [n][p+1][p+1][2] scalar coefficients of a Laplace density (close pairs)
    // rotated close-pair scheme (opts.near_scheme = 1), per entry e of the close-pair lists
    double* d_rotp = nullptr;      // degree blocks of f -> f o R_x(+90)
    double* d_rotm = nullptr;      // f -> f o R_x(-90)
    double* d_fgeo = nullptr;      // [n_near][8] frame angles, distances, source radius
    double* d_fcoef = nullptr;     // [n_near][3][p+1][p+1][2] rotated source coefficients
    double* d_fchan = nullptr;     // [n_near][sh_count(p+2)][kTracChannels]
    double* d_fblk = nullptr;      // [n_near][3][p+1][p+1][2] target-side blocks
    int* d_fiota = nullptr;        // [n_near+1] 0, 1, ..., n_near
    // FP32 copies for the FP32 operator of mixed-precision contexts
    float* d_tabf = nullptr;       // the tables of d_tab
    float* d_rotpf = nullptr;
    float* d_rotmf = nullptr;
    float* d_fcoeff = nullptr;     // [n_near][3][p+1][p+1][2]
    float* d_fchanf = nullptr;     // [n_near][sh_count(p+2)][28] (rows padded to a multiple of 4)
    float* d_fblkf = nullptr;      // [n_near][3][p+1][p+1][2]
    double mag_eta = 0.0;          // eta of the magnetic operator (Eq. 5.13) of the running solve
    double t_create_ms = 0.0;      // wall time of create (grid, tables, close pairs, preconditioner)
    bool has_solution = false;     // d_xsol holds the density of the last solve

    // host geometry
    std::vector<double> h_c, h_a;
    std::vector<int> h_near_ptr, h_near_idx;
    long long n_near = 0;

    // device geometry
    double* d_c = nullptr;       // [n][3]
    double* d_a = nullptr;       // [n]
    double* d_x = nullptr;       // [N][4]  position (x, y, z, weight)
    float4* d_xhi = nullptr;     // [N] float hi of position, .w = weight
    float4* d_xlo = nullptr;     // [N] float lo of position
    float4* d_nrm = nullptr;     // [N] outward normal (float)
    double* d_nrm64 = nullptr;   // [N][4] outward normal (double)
    int* d_sph = nullptr;        // [N] sphere index of each node
    long long far_pair_count = 0;  // (target, source) node pairs of the far field per apply
    // Per-problem flags of the running GMRES cycle (system numbering from
    // far_live_off): the far field skips target spheres of stopped problems,
    // whose Krylov vectors are zero.  Null outside the cycle.
    const int* far_live = nullptr;
    int far_live_off = 0;
    int* d_near_ptr = nullptr;   // [n+1] CSR of close pairs by target sphere
    int* d_near_idx = nullptr;
    double* d_tab = nullptr;
    sbie::TabLayout tl{};

    // scratch (owned)
    double* d_coef = nullptr;    // [n][3][p+1][p+1][2]  VSH coefficients of the last analysed density
    double* d_chan = nullptr;    // [n][sh_count(p+2)][kTracChannels]  close-pair expansions
    float* d_chanf = nullptr;    // float copy
    double* d_mom = nullptr;     // [n][6] moments int psi, int (y - c) x psi
    double* d_part = nullptr;    // far-field partials [split][N][3] (double)
    size_t part_cap = 0;
    double4* d_src64 = nullptr;  // [N] density x weight (double)
    float4* d_srcf = nullptr;    // [N] density x weight (float)
    double* d_in = nullptr;      // [N][3] host-staged inputs
    double* d_out = nullptr;     // [N][3]
    double* d_tmp = nullptr;     // [N][3]
    double* d_tmp2 = nullptr;    // [N][3]
    double* d_small = nullptr;   // [n][3] x 4 per-sphere small arrays
    double* d_red = nullptr;     // reduction scratch
    double* h_red = nullptr;     // pinned host mirror of reduction results
    // Krylov space
    double* d_V = nullptr;       // [restart+1][3N]
    sbie::ArnoldiDev ad{};       // device state of a restart cycle (krylov.cu)
    double* d_ad = nullptr;      // storage of the doubles of ad
    int* d_adi = nullptr;        // storage of the ints of ad
    double* d_vk = nullptr;      // [3N] current Krylov vector (fixed address)
    int* h_st = nullptr;         // pinned mirror of ad.st
    double* h_pack = nullptr;    // pinned staging of ad.pack
    std::vector<sbie::CycleGraph> graphs;
    double* d_xsol = nullptr;    // [3N]
    double* d_rhs = nullptr;     // [3N]
    double* d_res = nullptr;     // [3N]
    int krylov_m = 0;

    sbie::SelfGemm* sg = nullptr;  // self-term GEMMs of the FP32 operator (mixed-precision contexts)
    sbie::FarTune tune64[3]{}, tune32[3]{}, tunedf[3]{};  // per far-field kernel (S, D, K)
    sbie::Profile prof;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events[8];
    int prof_used[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long n_launch = 0;  // kernels launched by this context
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace sbie {

// CUDA events around one stage launch on the context stream (profiling on).
struct StageScope {
    sbie_ctx* c;
    int stage;
    int idx = -1;
    StageScope(sbie_ctx* cc, int st) : c(cc), stage(st) {
        if (!c->prof.on) return;
        auto& v = c->prof_events[stage];
        idx = c->prof_used[stage]++;
        if (idx >= (int)v.size()) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            v.push_back({a, b});
        }
        cudaEventRecord(v[idx].first, c->stream);
    }
    ~StageScope() {
        if (idx >= 0) cudaEventRecord(c->prof_events[stage][idx].second, c->stream);
    }
};

// Message returned by sphere_bie_last_error(NULL).
void set_last_error(const std::string& msg);

// --- kernels launchers (each returns cudaError_t of the launch) ---
// self.cu
cudaError_t launch_self(sbie_ctx* c, Kern op, const double* dens, double* out, bool accumulate, bool write_coef);
cudaError_t launch_self_precond(sbie_ctx* c, const double* v, double* out);
// VSH coefficients of dens into c->d_coef only (FP64 analysis, no synthesis)
cudaError_t launch_self_analysis(sbie_ctx* c, const double* dens);
// `count` independent unit-radius-free probes: the self kernel with signature
// `op` (Kern or kOpPrecHigh) on count densities of 3 npn values each, radius
// per probe from `radius`, coefficients to `coef` if not null
cudaError_t launch_self_probe(sbie_ctx* c, int op, int count, const double* dens, double* out, const double* radius,
                              double* coef);
// selfgemm.cu
cudaError_t self_gemm_build(sbie_ctx* c, int which);
bool self_gemm_ready(const sbie_ctx* c, int which);
cudaError_t launch_self_gemm(sbie_ctx* c, int which, const double* dens, double* out, bool accumulate);
cudaError_t self_gemm_error(sbie_ctx* c, int* flag);
void self_gemm_free(sbie_ctx* c);
// precond.cu
void lowmode_tables(int p, std::vector<double>& ZS, std::vector<double>& ZA);
void lowmode_rotation(const double Q[9], std::vector<double>& R);
// the degree blocks D_0 .. D_4 of lowmode_rotation, row-major, 165 values
void lowmode_rotation_blocks(const double Q[9], float* Dc);
// pair systems of the learned preconditioner assembled on the device (see precond.cu)
cudaError_t launch_pair_systems(cudaStream_t s, int np, const int2* pairs, const int* uid, const float* Lu,
                                const float* Y, const float* mean, const float* sd, const float* Dr, const float* Di,
                                float* sys);
cudaError_t launch_own_systems(cudaStream_t s, int n, const int* uid, const float* Lu, float* S);
std::vector<int4> low_mode_table();
cudaError_t launch_gauss_jordan(cudaStream_t s, int n, int count, float* mats, int* d_bad);
cudaError_t launch_probe_density(sbie_ctx* c, int sph_per_prob, int side, int beta, const double* ZS, double* dens);
cudaError_t launch_probe_analysis(sbie_ctx* c, const double* ZA, const double* u, int beta, double* blocks);
// G low modes per pass on single-sphere problems: sphere j carries mode
// b0 + j mod G; blocks[j / G][row][mode]
cudaError_t launch_probe_density_multi(sbie_ctx* c, int G, int b0, const double* ZS, double* dens);
cudaError_t launch_probe_analysis_multi(sbie_ctx* c, int G, int b0, const double* ZA, const double* u,
                                        double* blocks);
// M^{-1} v; f32: the FP32 inner solves' form (H and the low-mode analysis by
// the tensor-core GEMM), else FP64 throughout
cudaError_t precond_apply(sbie_ctx* c, int slot, const double* v, double* out, bool f32);
// far.cu
cudaError_t launch_pack(sbie_ctx* c, const double* dens, int mode);
cudaError_t launch_far(sbie_ctx* c, Kern op, int mode, double* out, bool accumulate = false);
// Times one launch of the far-field pair kernel with tiling `tu` (no reduce); *ms = event time.
cudaError_t time_far(sbie_ctx* c, Kern op, int mode, const FarTune& tu, float* ms);
long long far_pairs(const sbie_ctx* c);
int far_occupancy(sbie_ctx* c, Kern op, int mode, const FarTune& tu);
// register-cap builds of the FP32 pair kernel for `tpt` targets per thread
// (FarTune::minb values, at most 4); returns their count
int far_f32_builds(int tpt, int* minb);
// near.cu
cudaError_t launch_near(sbie_ctx* c, Kern op, bool f32, double* out);
cudaError_t launch_near_laplace(sbie_ctx* c, int mode, double* out);
// channels (near_prep) of `count` coefficient sets, one per entry (iota =
// 0..count), from FP64 (coef) or FP32 (coeff) coefficients; FP64 channels in
// chan and, when chanf is given, an FP32 copy with rows padded to a multiple of 4
cudaError_t launch_near_prep_pairs(sbie_ctx* c, int kind, int count, const double* coef, const float* coeff,
                                   const int* iota, double* chan, float* chanf);
// nearfft.cu: close pairs by the rotated scheme of Sec. 4.2
cudaError_t launch_near_fft(sbie_ctx* c, Kern op, bool f32, double* out);
size_t fft_eval_smem(int p, int kind, size_t elem);
// laplace.cu
cudaError_t laplace_apply(sbie_ctx* c, int mode, const double* q, double* out);
cudaError_t launch_magnetic_finalize(sbie_ctx* c, double eta, const double* in, double* out);
cudaError_t launch_magnetic_rhs(sbie_ctx* c, double eta, const double* H0, double* b);
cudaError_t launch_maxwell_traction(sbie_ctx* c, const double* H0, double* g);
// compl.cu
cudaError_t launch_moments(sbie_ctx* c, const double* dens);
cudaError_t launch_completion(sbie_ctx* c, bool f32, double* out);
cudaError_t launch_finalize(sbie_ctx* c, int op, const double* dens, double* out);
cudaError_t launch_rho(sbie_ctx* c, const double* F, const double* T, double* rho);
// squirmer operator: from the moments in d_mom (launch_moments of dens),
// r = P dens (rigid part on each sphere) and q = dens - r
cudaError_t launch_rigid_split(sbie_ctx* c, const double* dens, double* q, double* r);
cudaError_t launch_rigid_projection(sbie_ctx* c, const double* u, double* vel, double* omega);
cudaError_t launch_resistance_rhs(sbie_ctx* c, const double* vel, const double* omega, const double* u0,
                                  const double* G, double* b);
cudaError_t launch_geometry(sbie_ctx* c);
// blas.cu (FP64 vectors of length n)
cudaError_t blas_axpy(sbie_ctx* c, double a, const double* x, double* y, long long n);
cudaError_t blas_lincomb(sbie_ctx* c, double a, const double* x, double b, const double* y, double* out, long long n);
// segmented (one segment per independent problem; see blas.cu)
int seg_blocks(long long n3, int P);
cudaError_t seg_dots(sbie_ctx* c, const double* V, int k, long long ld, const double* w, long long n3,
                     const long long* d_seg, int P, double* d_out);
cudaError_t seg_scale(sbie_ctx* c, const double* x, const double* d_scale, const int* d_node_prob, double* y,
                      long long n3);
// krylov.cu (device-resident GMRES restart cycle)
cudaError_t arnoldi_cycle_init(sbie_ctx* c, const ArnoldiDev& A);
cudaError_t arnoldi_copy_k(sbie_ctx* c, const ArnoldiDev& A, const double* V, long long n3, double* dst);
cudaError_t arnoldi_orthogonalise(sbie_ctx* c, const ArnoldiDev& A, double* V, long long n3, const long long* d_seg,
                                  const int* d_node_prob);
cudaError_t arnoldi_step_end(sbie_ctx* c, const ArnoldiDev& A, double* V, long long n3, const int* d_node_prob,
                             cudaGraphConditionalHandle cond, bool has_cond);
cudaError_t arnoldi_finish(sbie_ctx* c, const ArnoldiDev& A, const double* V, long long n3, const int* d_node_prob,
                           double* out);

}  // namespace sbie
