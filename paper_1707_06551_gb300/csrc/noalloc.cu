// sphere_bie_apply_layer_noalloc: the FP64 raw layer operators for callers
// that cannot allocate device memory.  It has no counterpart in the paper.
//
// Some callers cannot call cudaMalloc: code running under a memory manager
// that owns the whole device (a pool or arena handed out by a host
// framework), or a latency-critical loop that has banned allocation after
// start-up.  For them this entry point computes what sphere_bie_apply_operator
// computes for SBIE_OP_S, _D or _K on a context created with eta = 0 (self
// term plus the far field over every other sphere, no close-pair correction),
// with the same kernels, but keeps every intermediate -- Legendre tables, node
// geometry, packed sources, the far-field partial sums -- in one file-scope
// __device__ array of kNoallocBytes (20 MiB).  Every GPU that loads the
// library holds that array until the process exits.
#include <mutex>

#include "common.h"

namespace {

constexpr long long kNoallocMaxNodes = 65536;  // N = n_spheres (p+1)(2p+2)
constexpr int kNoallocMaxSpheres = 4096;
constexpr int kNoallocSplit = 4;               // far-field source splits
constexpr size_t kNoallocBytes = 20u << 20;
constexpr int kMaxDevices = 128;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Slots {
    size_t tab, x64, xhi, xlo, nrm, nrm64, sph, near_ptr, near_idx, sph_prob, prob_sph, src64, part, end;
};

constexpr Slots slots() {
    Slots s{};
    size_t o = 0;
    s.tab = o;      o = align256(o + sizeof(double) * (size_t)sbie::tab_layout(sbie::kMaxP).total);
    s.x64 = o;      o = align256(o + sizeof(double) * 4 * kNoallocMaxNodes);
    s.xhi = o;      o = align256(o + sizeof(float4) * kNoallocMaxNodes);
    s.xlo = o;      o = align256(o + sizeof(float4) * kNoallocMaxNodes);
    s.nrm = o;      o = align256(o + sizeof(float4) * kNoallocMaxNodes);
    s.nrm64 = o;    o = align256(o + sizeof(double) * 4 * kNoallocMaxNodes);
    s.sph = o;      o = align256(o + sizeof(int) * kNoallocMaxNodes);
    s.near_ptr = o; o = align256(o + sizeof(int) * (kNoallocMaxSpheres + 1));
    s.near_idx = o; o = align256(o + sizeof(int));
    s.sph_prob = o; o = align256(o + sizeof(int) * kNoallocMaxSpheres);
    s.prob_sph = o; o = align256(o + sizeof(int) * 2);
    s.src64 = o;    o = align256(o + sizeof(double) * 4 * kNoallocMaxNodes);
    s.part = o;     o = align256(o + sizeof(double) * 3 * kNoallocSplit * kNoallocMaxNodes);
    s.end = o;
    return s;
}

// The largest accepted problem (p = 24 tables, 65,536 nodes, 4,096 spheres,
// kNoallocSplit partial sums) fits the array: checked when this file compiles.
static_assert(slots().end <= kNoallocBytes, "no-allocation scratch layout exceeds its static array");

// Device or managed memory that kernels on device `dev` may read and write.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
int g_tab_p[kMaxDevices] = {};

}  // namespace

// The scratch.  In host code this name is only a stand-in for the device
// array; the address passed to kernels comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

extern "C" sbie_status sphere_bie_apply_layer_noalloc(sbie_op op, int n_spheres, int p, const double* centres,
                                                      const double* radii, const double* density, double* out,
                                                      void* stream) {
    using namespace sbie;
    if (op != SBIE_OP_S && op != SBIE_OP_D && op != SBIE_OP_K) {
        set_last_error("noalloc: op must be SBIE_OP_S, SBIE_OP_D or SBIE_OP_K");
        return SBIE_ERR_ARG;
    }
    if (p < 1 || p > kMaxP) {
        set_last_error("noalloc: p must be in [1, 24]");
        return SBIE_ERR_ARG;
    }
    const long long npn = (long long)(p + 1) * (2 * p + 2);
    const long long N = (long long)n_spheres * npn;
    if (n_spheres < 1 || n_spheres > kNoallocMaxSpheres || N > kNoallocMaxNodes) {
        set_last_error("noalloc: needs 1 <= n_spheres <= 4096 and n_spheres (p+1)(2p+2) <= 65536 nodes "
                       "(the size of its static scratch); use sphere_bie_create / sphere_bie_apply_operator for "
                       "larger problems");
        return SBIE_ERR_ARG;
    }
    if (!centres || !radii || !density || !out || density == out) {
        set_last_error("noalloc: NULL or aliased pointer");
        return SBIE_ERR_ARG;
    }
    constexpr Slots sl = slots();
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_last_error(std::string("noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return SBIE_ERR_CUDA;
    }
    // Host memory or another GPU's memory would reach the kernels as a bad
    // address: refuse it before any work is queued.
    if (!on_device(centres, dev) || !on_device(radii, dev) || !on_device(density, dev) || !on_device(out, dev)) {
        set_last_error("noalloc: centres, radii, density and out must be device (or managed) memory of the "
                       "current device");
        return SBIE_ERR_ARG;
    }
    unsigned char* base = nullptr;
    bool need_tables = false;
    {
        // Set-up, once per device with that device current: the device address
        // of the scratch array.
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) {
                set_last_error(std::string("noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                return SBIE_ERR_CUDA;
            }
            g_addr[dev] = ptr;
        }
        base = static_cast<unsigned char*>(g_addr[dev]);
        need_tables = g_tab_p[dev] != p;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        set_last_error(std::string("noalloc: device attribute: ") + cudaGetErrorString(e));
        return SBIE_ERR_CUDA;
    }

    // A context that only points into the scratch and at the caller's arrays;
    // nothing in it owns device memory.
    sbie_ctx c;
    c.n = n_spheres;
    c.p = p;
    c.nlat = p + 1;
    c.nlon = 2 * p + 2;
    c.npn = (int)npn;
    c.N = N;
    c.stream = static_cast<cudaStream_t>(stream);
    c.sm_count = sms;
    c.tl = tab_layout(p);
    c.d_c = const_cast<double*>(centres);
    c.d_a = const_cast<double*>(radii);
    c.d_tab = reinterpret_cast<double*>(base + sl.tab);
    c.d_x = reinterpret_cast<double*>(base + sl.x64);
    c.d_xhi = reinterpret_cast<float4*>(base + sl.xhi);
    c.d_xlo = reinterpret_cast<float4*>(base + sl.xlo);
    c.d_nrm = reinterpret_cast<float4*>(base + sl.nrm);
    c.d_nrm64 = reinterpret_cast<double*>(base + sl.nrm64);
    c.d_sph = reinterpret_cast<int*>(base + sl.sph);
    c.d_near_ptr = reinterpret_cast<int*>(base + sl.near_ptr);
    c.d_near_idx = reinterpret_cast<int*>(base + sl.near_idx);
    c.d_sph_prob = reinterpret_cast<int*>(base + sl.sph_prob);
    c.d_prob_sph = reinterpret_cast<int*>(base + sl.prob_sph);
    c.n_prob = 1;
    c.d_src64 = reinterpret_cast<double4*>(base + sl.src64);
    c.d_part = reinterpret_cast<double*>(base + sl.part);
    c.n_near = 0;
    {
        int th = (int)std::min<long long>(256, ((npn + 31) / 32) * 32);
        int chunks = (int)((npn + th - 1) / th);
        long long ctas = (long long)n_spheres * chunks;
        int split = (int)std::min<long long>(kNoallocSplit, std::max<long long>(1, (4LL * sms + ctas - 1) / ctas));
        for (int op = 0; op < 3; ++op) c.tune64[op] = FarTune{th, 1, split, 128};
    }
    const Kern k = op == SBIE_OP_S ? Kern::S : (op == SBIE_OP_D ? Kern::D : Kern::K);

    if (need_tables) {
        std::vector<double> h;
        build_tables(p, h);
        e = cudaMemcpyAsync(c.d_tab, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, c.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
        if (e != cudaSuccess) {
            set_last_error(std::string("noalloc: tables: ") + cudaGetErrorString(e));
            return SBIE_ERR_CUDA;
        }
        std::lock_guard<std::mutex> lk(g_mu);
        g_tab_p[dev] = p;
    }
    // The scratch keeps the previous call's contents: the close-pair list must
    // start empty and every sphere belongs to the one problem [0, n_spheres);
    // every other slot is fully rewritten below before it is read.
    const int one_problem[2] = {0, n_spheres};
    e = cudaMemsetAsync(c.d_near_ptr, 0, sizeof(int) * (n_spheres + 1), c.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c.d_sph_prob, 0, sizeof(int) * n_spheres, c.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c.d_prob_sph, one_problem, sizeof(one_problem), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = launch_geometry(&c);
    if (e == cudaSuccess) e = launch_pack(&c, density, kModeF64);
    if (e == cudaSuccess) e = launch_far(&c, k, kModeF64, out);
    if (e == cudaSuccess) e = launch_self(&c, k, density, out, true, false);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) {
        set_last_error(std::string("noalloc: ") + cudaGetErrorString(e));
        return SBIE_ERR_CUDA;
    }
    return SBIE_OK;
}
