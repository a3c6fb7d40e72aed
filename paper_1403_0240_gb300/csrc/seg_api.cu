// libseg host side: validation, device state, the per-batch stepper that replays one
// captured CUDA graph per iteration, and the C-ABI entry points declared in seg.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "seg_internal.cuh"

using namespace segk;

namespace segk {
thread_local bool g_pdl = false;

// launches made while a stepper captures its graph count towards the graph, not the process
thread_local bool g_count_into_graph = false;
thread_local unsigned long long g_graph_kernels = 0;
std::atomic<unsigned long long> g_kernel_launches{0};

void count_launch()
{
    if (g_count_into_graph) g_graph_kernels++;
    else g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
}
}

namespace {

thread_local std::string g_last_cuda;

int cuda_fail(cudaError_t e, const char* what)
{
    g_last_cuda = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return SEG_ECUDA;
}

#define CK(x)                                              \
    do {                                                   \
        cudaError_t e_ = (x);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #x);   \
    } while (0)

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Sub-allocation plan of one device allocation.
struct Arena {
    size_t bytes = 0;
    std::vector<std::pair<void**, size_t>> parts;
    template <class T>
    void add(T** p, size_t count)
    {
        parts.push_back({(void**)p, align256(count * sizeof(T) + 1)});
        bytes += parts.back().second;
    }
    void assign(char* base)
    {
        size_t off = 0;
        for (auto& pr : parts) {
            *pr.first = base + off;
            off += pr.second;
        }
    }
};

// Device memory of contexts comes from a library-owned stream-ordered pool per device, so
// that creating and destroying contexts (served jobs) neither pays for a fresh allocation
// each time nor synchronises the device; the pool keeps freed memory for reuse and is
// trimmed once no context holds memory.
struct DevicePool {
    cudaMemPool_t pool = nullptr;
    long long live = 0;
};
std::mutex g_pool_mu;
DevicePool g_pools[64];

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        DevicePool& d = g_pools[dev];
        if (!d.pool) {
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            if ((e = cudaMemPoolCreate(&d.pool, &props)) != cudaSuccess) return e;
            unsigned long long keep = ~0ull;
            cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        pool = d.pool;
        d.live++;
    }
    e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        g_pools[dev].live--;
    }
    return e;
}

void dev_free(void* p, cudaStream_t s)
{
    if (!p) return;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    cudaFreeAsync(p, s);
    std::lock_guard<std::mutex> lock(g_pool_mu);
    DevicePool& d = g_pools[dev];
    if (--d.live == 0 && d.pool) {
        cudaStreamSynchronize(s);
        cudaMemPoolTrimTo(d.pool, 0);
    }
}

// Topology tables (adjacency masks and the tabulated simple-point decisions), built once
// per process, before the first context or simple-point query.
cudaError_t ensure_topology_tables()
{
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] { err = topology_tables_init(); });
    return err;
}

// Pinned host mirrors of the per-context counters, handed out from slabs that live as long
// as the process (a pinned allocation per context would cost more than the context).
std::mutex g_pin_mu;
std::vector<Counters*> g_pin_free;

Counters* pinned_counters()
{
    std::lock_guard<std::mutex> lock(g_pin_mu);
    if (g_pin_free.empty()) {
        constexpr int kSlab = 64;
        Counters* slab = nullptr;
        if (cudaMallocHost(&slab, sizeof(Counters) * kSlab) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        for (int i = kSlab - 1; i >= 0; i--) g_pin_free.push_back(slab + i);
    }
    Counters* c = g_pin_free.back();
    g_pin_free.pop_back();
    return c;
}

void release_counters(Counters* c)
{
    if (!c) return;
    std::lock_guard<std::mutex> lock(g_pin_mu);
    g_pin_free.push_back(c);
}

}  // namespace

struct Stepper;

struct seg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    seg_params params{};
    Job h{};                      // host copy of the job descriptor
    Job* d_self = nullptr;        // device copy used by init-time kernels
    Counters* d_ctr = nullptr;
    char* inputs = nullptr;       // image, labels and the input scan record
    char* arena = nullptr;
    size_t arena_bytes = 0;
    char* parena = nullptr;       // particle and candidate buffers (regrown on demand)
    size_t parena_bytes = 0;
    Stepper* own = nullptr;       // stepper used by seg_step
    seg_batch* batch = nullptr;
    Counters* h_ctr = nullptr;    // pinned host mirror
};

struct Stepper {
    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    std::vector<seg_ctx*> members;
    Job* d_jobs = nullptr;
    int cap_jobs = 0;
    int* d_ids = nullptr;          // group job ids (2D then 3D)
    unsigned* d_prefix = nullptr;  // group tile prefixes (2D then 3D)
    int cap_ids = 0;
    BatchCtl* d_bc = nullptr;
    Counters* d_gather = nullptr;
    Counters* h_gather = nullptr;
    int cap_gather = 0;
    Group grp[2]{};
    size_t smem_x[2]{}, smem_s[2]{};
    int commit_grid = 0, commit_block = 1024;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool use_graph = true;
    bool dirty = true;
    bool any_global = false;       // a member uses E = |Gamma| (adds its two launches to the step)
    bool any_deconv = false;       // a member uses the deconvolving model (adds its PSF passes)
    bool any_split = false;        // a member may split regions (adds the relabelling passes)
    bool any_curv = false;         // a member uses the curvature regulariser (adds its ball counts)
    bool any_fuse = false;         // a member may fuse regions (adds the fusion passes)
    bool profile = false;
    unsigned long long graph_kernels = 0;   // kernels in one replay of the graph
    cudaEvent_t ev[11]{};
    cudaStream_t work = nullptr;   // library stream: graphs are captured and launched here
    cudaEvent_t fence_in = nullptr, fence_out = nullptr;
};

constexpr int kStages = 9;

struct seg_batch {
    Stepper st;
};

namespace {


int validate(const seg_params* p)
{
    if (!p) return SEG_EINVAL;
    if (p->ndim != 2 && p->ndim != 3) return SEG_EINVAL;
    if (p->dtype != SEG_F32 && p->dtype != SEG_U16) return SEG_EINVAL;
    for (int i = 0; i < 3; i++)
        if (p->shape[i] < 1) return SEG_EINVAL;
    if (p->ndim == 2 && p->shape[0] != 1) return SEG_EINVAL;
    long double npix = (long double)p->shape[0] * p->shape[1] * p->shape[2];
    if (npix >= 2147483647.0L) return SEG_EINVAL;
    if (p->model != SEG_PC && p->model != SEG_PS && p->model != SEG_PS_POISSON && p->model != SEG_PC_DECONV)
        return SEG_EINVAL;
    if ((p->ndim == 2 && p->connectivity != 4) || (p->ndim == 3 && p->connectivity != 6)) return SEG_EINVAL;
    if (!(p->lambda >= 0.0) || !std::isfinite(p->lambda)) return SEG_EINVAL;
    if (!(p->cutoff > 0.0) || p->cutoff > 32.0) return SEG_EINVAL;
    if (is_ps(p->model) && (!(p->ps_radius >= 1.0) || p->ps_radius > 64.0)) return SEG_EINVAL;
    if (p->gradient != SEG_SOBOLEV && p->gradient != SEG_L2 && p->gradient != SEG_SOBOLEV_GLOBAL) return SEG_EINVAL;
    if (p->gradient == SEG_SOBOLEV_GLOBAL) {
        // the E = |Gamma| kernel table spans every squared distance in the image
        const long double d2 = (long double)(p->shape[0] - 1) * (p->shape[0] - 1) +
                               (long double)(p->shape[1] - 1) * (p->shape[1] - 1) +
                               (long double)(p->shape[2] - 1) * (p->shape[2] - 1);
        if (d2 >= (long double)(1 << 24)) return SEG_EINVAL;
    }
    if (p->osc_window < 0) return SEG_EINVAL;
    if (p->stats_mode != SEG_STATS_EXACT && p->stats_mode != SEG_STATS_F64 && p->stats_mode != SEG_STATS_KAHAN32)
        return SEG_EINVAL;
    int need = (int)std::ceil(p->cutoff);
    if (p->cell_edge != 0 && (p->cell_edge < need || p->cell_edge > 256)) return SEG_EINVAL;
    for (int i = 0; i < 3; i++)
        if (p->tile[i] < 0 || p->tile[i] > 1024) return SEG_EINVAL;
    if (p->ndim == 2 && p->tile[0] > 1) return SEG_EINVAL;
    if (p->topology < 0 || p->topology > (SEG_TOPO_VANISH | SEG_TOPO_SPLIT | SEG_TOPO_FUSE)) return SEG_EINVAL;
    // fusion: the piecewise-constant model with exact statistics
    if ((p->topology & SEG_TOPO_FUSE) && (p->model != SEG_PC || p->stats_mode != SEG_STATS_EXACT)) return SEG_EINVAL;
    if (p->max_labels < 0 || p->max_labels > (1 << 24)) return SEG_EINVAL;
    if (p->regulariser != SEG_REG_LENGTH && p->regulariser != SEG_REG_CURVATURE) return SEG_EINVAL;
    if (p->regulariser == SEG_REG_CURVATURE && (!(p->curv_radius >= 1.0) || p->curv_radius > 16.0)) return SEG_EINVAL;
    if (p->reserved) return SEG_EINVAL;
    return SEG_OK;
}

// Label capacity: the initial count M0, or with SEG_TOPO_SPLIT max_labels (default
// max(2 M0, M0 + 256)), so that the pieces of split regions can take new labels.
int label_capacity(const seg_params* p, int M0)
{
    if (!(p->topology & SEG_TOPO_SPLIT)) return M0;
    if (p->max_labels) return std::max(p->max_labels, M0);
    return (int)std::min<long long>(1LL << 24, std::max<long long>(2LL * M0, (long long)M0 + 256));
}

// Eq. 5 in FP64, then rounded to float for the interaction table.
double kernel_eq5(double r, double E)
{
    const double eps = 1.0 / 24.0;
    double x = r / E;
    double num = x * x - x + 1.0 / 6.0;
    return (1.0 / E) * (1.0 + num / (2.0 * eps));
}

int largest_d2_below(double cutoff)
{
    const double r2 = cutoff * cutoff;
    long long k = (long long)std::ceil(r2) - 1;
    if (k < 0) k = 0;
    while ((double)(k + 1) < r2) k++;
    while (k > 0 && !((double)k < r2)) k--;
    return (int)k;
}

// Geometry, tables and the plan of the fixed device allocation.
struct Plan {
    Job h{};
    std::vector<float> klut, klut_lo;
    std::vector<double> klut64;
    std::vector<int4> ps_off, nb_off, cv_off;
    Arena fixed;
};

void make_geometry(const seg_params* p, int M, int slot_lo, int nS, Plan& P)
{
    Job& h = P.h;
    h.ndim = p->ndim;
    h.D = (int)p->shape[0];
    h.H = (int)p->shape[1];
    h.W = (int)p->shape[2];
    h.npix = (long long)h.D * h.H * h.W;
    h.fd_W = make_fastdiv((unsigned)h.W);
    h.fd_HW = make_fastdiv((unsigned)((long long)h.W * h.H));
    h.dtype = p->dtype;
    h.model = p->model;
    h.conn = p->connectivity;
    h.cell = p->cell_edge ? p->cell_edge : std::max(1, (int)std::ceil(p->cutoff));
    const int s = h.cell;
    h.fd_cell = make_fastdiv((unsigned)s);
    h.ncx = (h.W + s - 1) / s;
    h.ncy = (h.H + s - 1) / s;
    h.ncz = h.ndim == 3 ? (h.D + s - 1) / s : h.D;
    // tiles: a whole number of cells per axis (default 32 x 64 pixels in 2D, 8 x 8 x 32 in 3D)
    const int tx = p->tile[2] > 0 ? p->tile[2] : (h.ndim == 2 ? 64 : 32);
    const int ty = p->tile[1] > 0 ? p->tile[1] : (h.ndim == 2 ? 32 : 8);
    const int tz = p->tile[0] > 0 ? p->tile[0] : 8;
    h.tcx = std::max(1, tx / s);
    h.tcy = std::max(1, ty / s);
    h.tcz = h.ndim == 2 ? 1 : std::max(1, tz / s);
    h.ntx = (h.ncx + h.tcx - 1) / h.tcx;
    h.nty = (h.ncy + h.tcy - 1) / h.tcy;
    h.ntz = (h.ncz + h.tcz - 1) / h.tcz;
    h.ntiles = h.ntx * h.nty * h.ntz;
    const int R = (int)std::floor(p->ps_radius);
    h.ps_staged = (is_ps(h.model) && h.ndim == 2 && R <= 32) ? 1 : 0;
    h.halo = h.ps_staged ? std::max(1, R) : 1;
    h.curv = p->regulariser == SEG_REG_CURVATURE ? 1 : 0;
    // with the curvature regulariser the length term's weight is zero and the ball term's weight w
    h.lambda64 = h.curv ? 0.0 : p->lambda;
    h.lambda32 = (float)h.lambda64;
    if (h.curv) {
        const double r = p->curv_radius;
        h.curv_w64 = h.ndim == 3 ? p->lambda * (4.0 / (3.141592653589793 * (r * r * r * r)))
                                 : p->lambda * (3.0 / (2.0 * (r * r * r)));
        h.curv_w32 = (float)h.curv_w64;
    }
    h.cutoff = p->cutoff;
    h.E = 2.0 * p->cutoff;
    h.r2max = largest_d2_below(p->cutoff);
    h.M = M;
    h.global_E = p->gradient == SEG_SOBOLEV_GLOBAL ? 1 : 0;
    h.gd2max = h.global_E ? (int)((long long)(h.D - 1) * (h.D - 1) + (long long)(h.H - 1) * (h.H - 1) +
                                  (long long)(h.W - 1) * (h.W - 1))
                          : 0;
    h.osc_window = p->osc_window;
    h.topo_vanish = (p->topology & SEG_TOPO_VANISH) ? 1 : 0;
    h.topo_split = (p->topology & SEG_TOPO_SPLIT) ? 1 : 0;
    h.topo_fuse = (p->topology & SEG_TOPO_FUSE) ? 1 : 0;
    h.fz_lam64 = p->lambda;
    h.nbr_stride = h.ndim == 3 ? 26 : 8;
    h.slot_lo = slot_lo;
    h.nS = nS;
    h.nQ = 2 * (nS - 1) + 25;
    P.klut.resize(h.r2max + 1);
    P.klut_lo.resize(h.r2max + 1);
    P.klut64.resize(h.r2max + 1);
    for (int d2 = 0; d2 <= h.r2max; d2++) {
        P.klut64[d2] = kernel_eq5(std::sqrt((double)d2), h.E);
        P.klut[d2] = (float)P.klut64[d2];
        P.klut_lo[d2] = (float)(P.klut64[d2] - (double)P.klut[d2]);   // exact difference, rounded once
    }
    const int rz = h.ndim == 3 ? 1 : 0;
    if (is_ps(h.model)) {
        const double R2 = p->ps_radius * p->ps_radius;
        for (int dz = -R * rz; dz <= R * rz; dz++)
            for (int dy = -R; dy <= R; dy++)
                for (int dx = -R; dx <= R; dx++) {
                    int d2 = dz * dz + dy * dy + dx * dx;
                    if ((double)d2 <= R2) P.ps_off.push_back(make_int4(dz, dy, dx, d2));
                }
    }
    if (h.curv) {
        const int Rc = (int)std::floor(p->curv_radius);
        const double R2 = p->curv_radius * p->curv_radius;
        for (int dz = -Rc * rz; dz <= Rc * rz; dz++)
            for (int dy = -Rc; dy <= Rc; dy++)
                for (int dx = -Rc; dx <= Rc; dx++) {
                    int d2 = dz * dz + dy * dy + dx * dx;
                    if ((double)d2 <= R2) P.cv_off.push_back(make_int4(dz, dy, dx, d2));
                }
    }
    h.cv_n = (int)P.cv_off.size();
    const int rr = (int)std::floor(std::sqrt((double)h.r2max));
    for (int dz = -rr * rz; dz <= rr * rz; dz++)
        for (int dy = -rr; dy <= rr; dy++)
            for (int dx = -rr; dx <= rr; dx++) {
                int d2 = dz * dz + dy * dy + dx * dx;
                if (d2 <= h.r2max) P.nb_off.push_back(make_int4(dz, dy, dx, d2));
            }
    h.ps_n = (int)P.ps_off.size();
    h.nb_n = (int)P.nb_off.size();
    // exact ball sums: |q| < 2^(23 + nS) for float32 (2^16 for uint16); a ball sum of ps_n terms
    // needs log2(ps_n) more bits, a sum of shifted values one more; int64 holds 63 bits and an
    // FP64 partial sum is exact below 2^53 units
    int lg = 0;
    while ((1LL << lg) < (long long)std::max(1, h.ps_n)) lg++;
    const int qbits = h.dtype == SEG_F32 ? 23 + nS : 16;
    h.e_min = h.dtype == SEG_F32 ? slot_lo - 150 : 0;
    const bool unit_ok = h.e_min >= -120 && h.e_min <= 100;
    h.ps_int = (is_ps(h.model) && unit_ok && qbits + lg + 1 <= 62) ? 1 : 0;
    h.ps_exact64 = (h.ps_int && qbits + lg <= 53) ? 1 : 0;
    h.ps_q32 = (h.ps_int && h.dtype == SEG_F32 && qbits <= 31) ? 1 : 0;
    h.unit32 = unit_ok ? std::ldexp(1.0f, h.e_min) : 0.0f;
    h.unit64 = std::ldexp(1.0, h.e_min);

    Arena& A = P.fixed;
    const long long npix = h.npix;
    const long long ncell = (long long)h.ncx * h.ncy * h.ncz;
    const size_t esz = h.dtype == SEG_F32 ? 4 : 2;
    (void)esz;                     // image and labels live in the context's input buffer
    A.add(&h.pmap, npix);
    A.add(&h.cell_start, ncell);
    A.add(&h.cell_count, ncell);
    A.add(&h.tile_word, h.ntiles);
    A.add(&h.tile_start, h.ntiles);
    A.add(&h.tile_count, h.ntiles);
    A.add(&h.st_n, M);
    A.add(&h.st_S, (size_t)M * (h.dtype == SEG_F32 ? h.nS : 1));
    A.add(&h.st_Q, (size_t)M * (h.dtype == SEG_F32 ? h.nQ : 1));
    h.stats_mode = p->stats_mode;
    if (h.stats_mode == SEG_STATS_F64) A.add(&h.sf64, 2 * (size_t)M);
    if (h.stats_mode == SEG_STATS_KAHAN32) A.add(&h.sk32, 2 * (size_t)M);
    A.add(&h.S64, M);
    A.add(&h.Q64, M);
    A.add(&h.mu64, M);
    A.add(&h.wp64, M);
    A.add(&h.wm64, M);
    A.add(&h.mu32, M);
    A.add(&h.wp32, M);
    A.add(&h.wm32, M);
    A.add((float**)&h.klut, P.klut.size());
    A.add((float**)&h.klut_lo, P.klut_lo.size());
    A.add((double**)&h.klut64, P.klut64.size());
    A.add((int4**)&h.ps_off, std::max<size_t>(1, P.ps_off.size()));
    A.add((int4**)&h.nb_off, P.nb_off.size());
    if (h.curv) A.add((int4**)&h.cv_off, P.cv_off.size());
    A.add(&h.gK32, (size_t)h.gd2max + 1);
    A.add(&h.gK32l, (size_t)h.gd2max + 1);
    A.add(&h.gK64, (size_t)h.gd2max + 1);
    h.psf_r = -1;
    if (h.topo_fuse) {
        // touching pairs: a planar label graph has fewer than 3 M edges; 16 M slots (at least
        // 4096, at most 2^22) keep the table at most a quarter full in 2D
        unsigned cap = 4096;
        while (cap < (1u << 22) && (long long)cap < 16LL * M) cap <<= 1;
        h.fz_cap = cap;
        A.add(&h.fz_key, cap);
        A.add(&h.fz_cnt, cap);
        A.add(&h.fz_list, cap);
        A.add(&h.fz_ab, cap);
        A.add(&h.fz_u, cap);
        A.add(&h.fz_B, cap);
        A.add(&h.fz_state, cap);
        A.add(&h.fz_best_u, M);
        A.add(&h.fz_best_ab, M);
        A.add(&h.fz_used, M);
        A.add(&h.fz_to, M);
        A.add(&h.fz_done, M);
    }
    if (h.topo_split) {
        A.add(&h.cc_parent, npix);
        A.add(&h.cc_newl, npix);
        A.add(&h.cc_first, M);
        A.add(&h.cc_list, M);
    }
    if (h.model == SEG_PC_DECONV) {
        A.add(&h.psf, 2 * SEG_PSF_MAX_RADIUS + 1);
        A.add(&h.psf_n, (size_t)h.W + h.H + h.D);
        A.add(&h.dc_T, npix);
        if (h.ndim == 3) A.add(&h.dc_T2, npix);
        A.add(&h.dc_R, npix);
        A.add(&h.dc_G, npix);
    }
    A.add(&h.ctr, 1);
}

// Tensor maps for the extraction tiles: labels (int32) and, when the piecewise-smooth image
// is staged, the image. Box: tma_bx x (tile rows + 2 halo) [x (tile slices + 2 halo)], from
// an x coordinate aligned down to 8 elements, so every copy starts on a 16-byte boundary.
// Row pitches that are not multiples of 16 bytes keep the row-by-row load.
void setup_tma(Job& h)
{
    h.use_tma = 0;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
        cudaGetLastError();
    }
    if (!encode) return;
    const int s = h.cell, sz = h.ndim == 3 ? h.cell : 1;
    const int hz = h.ndim == 3 ? h.halo : 0;
    const int bx = ((h.tcx * s + 2 * h.halo + 7 + 7) / 8) * 8;
    const int by = h.tcy * s + 2 * h.halo;
    const int bz = h.tcz * sz + 2 * hz;
    if (bx > 256 || by > 256 || bz > 256) return;
    const size_t esz = h.dtype == SEG_F32 ? 4 : 2;
    if ((h.W * 4) % 16 != 0) return;
    if (h.ps_staged && (h.W * esz) % 16 != 0) return;
    const cuuint32_t rank = h.ndim == 3 ? 3 : 2;
    cuuint64_t gdim[3] = {(cuuint64_t)h.W, (cuuint64_t)h.H, (cuuint64_t)h.D};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    cuuint32_t estr[3] = {1, 1, 1};
    cuuint64_t gstr_l[2] = {(cuuint64_t)h.W * 4, (cuuint64_t)h.W * h.H * 4};
    if (encode((CUtensorMap*)h.tmap_L, CU_TENSOR_MAP_DATA_TYPE_INT32, rank, (void*)h.L, gdim, gstr_l, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return;
    if (h.ps_staged) {
        cuuint64_t gstr_i[2] = {(cuuint64_t)h.W * esz, (cuuint64_t)h.W * h.H * esz};
        if (encode((CUtensorMap*)h.tmap_I, h.dtype == SEG_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16,
                   rank, (void*)h.I, gdim, gstr_i, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return;
    }
    h.tma_bx = bx;
    h.use_tma = 1;
}

size_t particle_bytes(long long pcap, int stride)
{
    Arena A;
    Job h{};
    A.add(&h.p_idx, pcap);
    A.add(&h.p_l, pcap);
    A.add(&h.p_c, pcap);
    A.add(&h.p_dE, pcap);
    A.add(&h.p_dEl, pcap);
    A.add(&h.p_eE, pcap);
    A.add(&h.p_dE64, pcap);
    A.add(&h.p_g, pcap);
    A.add(&h.p_eg, pcap);
    A.add(&h.p_key, pcap);
    A.add(&h.p_nbm, pcap);
    A.add(&h.p_flags, pcap);
    A.add(&h.p_qc, pcap);
    A.add(&h.p_ql, pcap);
    A.add(&h.p_nc, pcap);
    A.add(&h.p_nl, pcap);
    A.add(&h.pix_cand, pcap);
    A.add(&h.flag_list, pcap);
    A.add(&h.c_best, pcap);
    A.add(&h.c_key, pcap);
    A.add(&h.c_pix, pcap);
    A.add(&h.c_ge, pcap);
    A.add(&h.c_state, pcap);
    A.add(&h.c_nnbr, pcap);
    A.add(&h.c_nbr, pcap * stride);
    return A.bytes;
}

void assign_particles(Job& h, char* base, long long pcap)
{
    Arena A;
    A.add(&h.p_idx, pcap);
    A.add(&h.p_l, pcap);
    A.add(&h.p_c, pcap);
    A.add(&h.p_dE, pcap);
    A.add(&h.p_dEl, pcap);
    A.add(&h.p_eE, pcap);
    A.add(&h.p_dE64, pcap);
    A.add(&h.p_g, pcap);
    A.add(&h.p_eg, pcap);
    A.add(&h.p_key, pcap);
    A.add(&h.p_nbm, pcap);
    A.add(&h.p_flags, pcap);
    A.add(&h.p_qc, pcap);
    A.add(&h.p_ql, pcap);
    A.add(&h.p_nc, pcap);
    A.add(&h.p_nl, pcap);
    A.add(&h.pix_cand, pcap);
    A.add(&h.flag_list, pcap);
    A.add(&h.c_best, pcap);
    A.add(&h.c_key, pcap);
    A.add(&h.c_pix, pcap);
    A.add(&h.c_ge, pcap);
    A.add(&h.c_state, pcap);
    A.add(&h.c_nnbr, pcap);
    A.add(&h.c_nbr, pcap * h.nbr_stride);
    A.assign(base);
    h.pcap = pcap;
}

long long default_pcap(long long npix, int ndim)
{
    long long worst = 2LL * ndim * npix;
    long long want = std::max<long long>(65536, npix / 2);
    return std::min(worst, want);
}

// initial capacity once the initial particle count n0 is known: room for the contour to
// double (more regrows the buffers between iterations)
long long initial_pcap(long long npix, int ndim, long long n0)
{
    long long worst = 2LL * ndim * npix;
    return std::min(worst, std::max<long long>(65536, 2 * n0 + 65536));
}

size_t input_bytes(long long npix, int dtype)
{
    return align256(npix * (dtype == SEG_F32 ? 4 : 2) + 1) + align256(npix * 4 + 1) + 256;
}

int grow_particles(seg_ctx* c, long long need)
{
    long long pcap = std::max<long long>(need + need / 2, c->h.pcap * 2);
    pcap = std::min<long long>(pcap, 2LL * c->h.ndim * c->h.npix);
    if (pcap < need) return SEG_ENOMEM;
    size_t bytes = particle_bytes(pcap, c->h.nbr_stride);
    char* mem = nullptr;
    CK(cudaStreamSynchronize(c->stream));
    cudaError_t e = dev_alloc((void**)&mem, bytes, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SEG_ENOMEM;
    }
    dev_free(c->parena, c->stream);
    c->parena = mem;
    c->parena_bytes = bytes;
    assign_particles(c->h, mem, pcap);
    CK(cudaMemcpyAsync(c->d_self, &c->h, sizeof(Job), cudaMemcpyHostToDevice, c->stream));
    return SEG_OK;
}

// ---------------------------------------------------------------------------
void stepper_free_graph(Stepper& s)
{
    if (s.exec) cudaGraphExecDestroy(s.exec);
    if (s.graph) cudaGraphDestroy(s.graph);
    s.exec = nullptr;
    s.graph = nullptr;
}

int stepper_build(Stepper& s)
{
    stepper_free_graph(s);
    const int n = (int)s.members.size();
    if (!s.d_bc) {
        CK(cudaMalloc(&s.d_bc, sizeof(BatchCtl)));
        CK(cudaMemsetAsync(s.d_bc, 0, sizeof(BatchCtl), s.stream));
    }
    if (n > s.cap_jobs) {
        if (s.d_jobs) CK(cudaFree(s.d_jobs));
        if (s.d_ids) CK(cudaFree(s.d_ids));
        if (s.d_prefix) CK(cudaFree(s.d_prefix));
        if (s.d_gather) CK(cudaFree(s.d_gather));
        if (s.h_gather) CK(cudaFreeHost(s.h_gather));
        int cap = std::max(n, 2 * s.cap_jobs);
        CK(cudaMalloc(&s.d_jobs, sizeof(Job) * cap));
        CK(cudaMalloc(&s.d_ids, sizeof(int) * cap));
        CK(cudaMalloc(&s.d_prefix, sizeof(unsigned) * (cap + 2)));
        CK(cudaMalloc(&s.d_gather, sizeof(Counters) * cap));
        CK(cudaMallocHost(&s.h_gather, sizeof(Counters) * cap));
        s.cap_jobs = cap;
    }
    std::vector<Job> jobs(n);
    std::vector<int> ids;
    std::vector<unsigned> prefix;
    s.any_global = false;
    s.any_deconv = false;
    s.any_split = false;
    s.any_curv = false;
    s.any_fuse = false;
    for (int i = 0; i < n; i++) {
        jobs[i] = s.members[i]->h;
        if (jobs[i].model == SEG_PC_DECONV && jobs[i].psf_r < 0) return SEG_ESTATE;   // no PSF yet
        s.any_global = s.any_global || jobs[i].global_E;
        s.any_deconv = s.any_deconv || jobs[i].model == SEG_PC_DECONV;
        s.any_split = s.any_split || jobs[i].topo_split;
        s.any_curv = s.any_curv || jobs[i].curv;
        s.any_fuse = s.any_fuse || jobs[i].topo_fuse;
    }
    int id_off[2] = {0, 0}, pf_off[2] = {0, 0};
    for (int gidx = 0; gidx < 2; gidx++) {
        const int nd = gidx == 0 ? 2 : 3;
        id_off[gidx] = (int)ids.size();
        pf_off[gidx] = (int)prefix.size();
        unsigned acc = 0;
        size_t sx = 0, ss = 0;
        int cnt = 0;
        for (int i = 0; i < n; i++) {
            if (jobs[i].ndim != nd) continue;
            ids.push_back(i);
            prefix.push_back(acc);
            acc += (unsigned)jobs[i].ntiles;
            sx = std::max(sx, extract_smem_bytes(jobs[i]));
            ss = std::max(ss, sobolev_smem_bytes(jobs[i]));
            cnt++;
        }
        prefix.push_back(acc);
        Group& g = s.grp[gidx];
        g.jobs = s.d_jobs;
        g.njobs = cnt;
        g.total_tiles = cnt ? acc : 0;
        g.ticket = &s.d_bc->ticket[gidx];
        s.smem_x[gidx] = sx;
        s.smem_s[gidx] = ss;
    }
    if ((int)prefix.size() > s.cap_jobs + 2 || (int)ids.size() > s.cap_jobs) return SEG_EINVAL;
    for (int gidx = 0; gidx < 2; gidx++) {
        s.grp[gidx].job_ids = s.d_ids + id_off[gidx];
        s.grp[gidx].tile_prefix = s.d_prefix + pf_off[gidx];
    }
    if (n) CK(cudaMemcpyAsync(s.d_jobs, jobs.data(), sizeof(Job) * n, cudaMemcpyHostToDevice, s.stream));
    if (!ids.empty()) CK(cudaMemcpyAsync(s.d_ids, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice, s.stream));
    CK(cudaMemcpyAsync(s.d_prefix, prefix.data(), sizeof(unsigned) * prefix.size(), cudaMemcpyHostToDevice, s.stream));
    CK(configure_kernels(s.smem_x[0], s.smem_x[1], s.smem_s[0], s.smem_s[1]));
    int per_sm = 0;
    CK(commit_occupancy(s.commit_block, &per_sm));
    if (per_sm < 1) return cuda_fail(cudaErrorCooperativeLaunchTooLarge, "commit occupancy");
    s.commit_grid = s.sms * std::min(per_sm, 1);
    CK(cudaStreamSynchronize(s.stream));
    s.dirty = false;
    return SEG_OK;
}

thread_local bool g_capturing = false;

cudaError_t stage_mark(Stepper& s, int k)
{
    if (!s.profile) return cudaSuccess;
    if (g_capturing) return cudaEventRecordWithFlags(s.ev[k], s.work, cudaEventRecordExternal);
    return cudaEventRecord(s.ev[k], s.work);
}

cudaError_t stepper_enqueue_stages(Stepper& s);

// One iteration's stages; their launches overlap each other's ramp and drain (programmatic
// dependent launch) unless per-stage events are recorded between them. That pays for
// latency-bound iterations (tile grids of a few waves); with many waves of tiles the early
// scheduled blocks only wait, so large grids keep plain stream order.
cudaError_t stepper_enqueue(Stepper& s)
{
    const long long tiles = (long long)s.grp[0].total_tiles + s.grp[1].total_tiles;
    g_pdl = !s.profile && tiles <= 8LL * s.sms;
    const cudaError_t e = stepper_enqueue_stages(s);
    g_pdl = false;
    return e;
}

cudaError_t stepper_enqueue_stages(Stepper& s)
{
    cudaError_t e;
    const int n = (int)s.members.size();
    if ((e = stage_mark(s, 0)) != cudaSuccess) return e;
    if (s.any_deconv)                   // the deconvolving model's fields, before extraction reads them
        for (int i = 0; i < n; i++)
            if (s.members[i]->h.model == SEG_PC_DECONV &&
                (e = launch_deconv(s.d_jobs, i, s.members[i]->h, s.sms, s.work)) != cudaSuccess)
                return e;
    if ((e = stage_mark(s, 1)) != cudaSuccess) return e;
    for (int gidx = 0; gidx < 2; gidx++)
        if (s.grp[gidx].njobs && (e = launch_extract(s.grp[gidx], gidx + 2, s.smem_x[gidx], s.work)) != cudaSuccess) return e;
    if (s.any_curv)                     // the curvature term, before the Sobolev sums read dE
        for (int i = 0; i < n; i++)
            if (s.members[i]->h.curv && (e = launch_curvature(s.d_jobs, i, s.sms, s.work)) != cudaSuccess) return e;
    if ((e = stage_mark(s, 2)) != cudaSuccess) return e;
    if (s.any_global && (e = launch_global_lut(s.d_jobs, n, s.sms, s.work)) != cudaSuccess) return e;
    for (int gidx = 0; gidx < 2; gidx++)
        if (s.grp[gidx].njobs && (e = launch_sobolev(s.grp[gidx], s.d_bc, gidx + 2, s.smem_s[gidx], s.work)) != cudaSuccess) return e;
    for (int gidx = 0; gidx < 2; gidx++)
        if (s.any_global && s.grp[gidx].njobs && (e = launch_sobolev_global(s.grp[gidx], gidx + 2, s.work)) != cudaSuccess)
            return e;
    if ((e = stage_mark(s, 3)) != cudaSuccess) return e;
    if (s.any_global)                   // E = |Gamma|: its candidates (the other modes select in k_sobolev)
        for (int gidx = 0; gidx < 2; gidx++)
            if (s.grp[gidx].njobs && (e = launch_select(s.grp[gidx], s.d_bc, s.work)) != cudaSuccess) return e;
    if ((e = stage_mark(s, 4)) != cudaSuccess) return e;
    if ((e = launch_lists(s.d_jobs, n, s.sms, s.work)) != cudaSuccess) return e;
    if ((e = stage_mark(s, 5)) != cudaSuccess) return e;
    if ((e = launch_fixup(s.d_jobs, n, s.sms, s.work)) != cudaSuccess) return e;
    if ((e = stage_mark(s, 6)) != cudaSuccess) return e;
    if ((e = launch_rounds(s.d_jobs, n, s.d_bc, s.commit_grid, s.commit_block, s.work)) != cudaSuccess) return e;
    if ((e = stage_mark(s, 7)) != cudaSuccess) return e;
    if ((e = launch_moves(s.d_jobs, n, s.d_bc, s.sms, s.work)) != cudaSuccess) return e;
    if (s.any_split)                    // split regions: pieces get new labels, statistics rebuilt
        for (int i = 0; i < n; i++)
            if (s.members[i]->h.topo_split &&
                (e = launch_relabel(s.d_jobs, i, s.members[i]->h, s.sms, s.work)) != cudaSuccess)
                return e;
    if (s.any_fuse)                     // touching regions whose fusion lowers the energy merge
        for (int i = 0; i < n; i++)
            if (s.members[i]->h.topo_fuse && (e = launch_fuse(s.d_jobs, i, s.sms, s.work)) != cudaSuccess) return e;
    if ((e = stage_mark(s, 8)) != cudaSuccess) return e;
    if ((e = launch_finish(s.d_jobs, n, s.d_bc, s.sms, s.work)) != cudaSuccess) return e;
    return stage_mark(s, 9);
}

int stepper_set_profile(Stepper& s, bool on)
{
    if (on && !s.ev[0])
        for (int k = 0; k <= kStages; k++) CK(cudaEventCreate(&s.ev[k]));
    if (s.profile != on) {
        s.profile = on;
        stepper_free_graph(s);
    }
    return SEG_OK;
}

int stepper_stage_times(Stepper& s, float* ms, int n)
{
    if (!s.profile || !s.ev[0]) return SEG_ESTATE;
    if (!ms || n < kStages) return SEG_EINVAL;
    CK(cudaStreamSynchronize(s.stream));
    if (s.work) CK(cudaStreamSynchronize(s.work));
    for (int k = 0; k < kStages; k++) CK(cudaEventElapsedTime(&ms[k], s.ev[k], s.ev[k + 1]));
    return SEG_OK;
}

void stepper_release(Stepper& s)
{
    stepper_free_graph(s);
    if (s.d_jobs) cudaFree(s.d_jobs);
    if (s.d_ids) cudaFree(s.d_ids);
    if (s.d_prefix) cudaFree(s.d_prefix);
    if (s.d_bc) cudaFree(s.d_bc);
    if (s.d_gather) cudaFree(s.d_gather);
    if (s.h_gather) cudaFreeHost(s.h_gather);
    for (int k = 0; k <= kStages; k++)
        if (s.ev[k]) cudaEventDestroy(s.ev[k]);
    if (s.work) cudaStreamSynchronize(s.work);
    if (s.fence_in) cudaEventDestroy(s.fence_in);
    if (s.fence_out) cudaEventDestroy(s.fence_out);
    if (s.work) cudaStreamDestroy(s.work);
    cudaGetLastError();
}

int stepper_run(Stepper& s, int iters)
{
    if (s.dirty) {
        int rc = stepper_build(s);
        if (rc) return rc;
    }
    if (s.members.empty() || iters <= 0) return SEG_OK;
    if (!s.work) {
        CK(cudaStreamCreateWithFlags(&s.work, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&s.fence_in, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&s.fence_out, cudaEventDisableTiming));
    }
    if (s.use_graph && !s.exec) {
        cudaError_t e = cudaStreamBeginCapture(s.work, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            g_capturing = true;
            g_count_into_graph = true;
            g_graph_kernels = 0;
            cudaError_t e2 = stepper_enqueue(s);
            g_count_into_graph = false;
            s.graph_kernels = g_graph_kernels;
            g_capturing = false;
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(s.work, &g);
            if (e2 == cudaSuccess && e == cudaSuccess && g) {
                e = cudaGraphInstantiate(&s.exec, g, 0);
                s.graph = g;
                if (e != cudaSuccess) {
                    stepper_free_graph(s);
                    s.use_graph = false;
                }
            } else {
                if (g) cudaGraphDestroy(g);
                s.use_graph = false;
            }
        } else {
            s.use_graph = false;
        }
        cudaGetLastError();
    }
    // order the work after everything already queued on the caller's stream, and make
    // the caller's stream wait for it
    CK(cudaEventRecord(s.fence_in, s.stream));
    CK(cudaStreamWaitEvent(s.work, s.fence_in, 0));
    for (int i = 0; i < iters; i++) {
        if (s.use_graph) {
            CK(cudaGraphLaunch(s.exec, s.work));
            g_kernel_launches.fetch_add(s.graph_kernels, std::memory_order_relaxed);
        } else {
            CK(stepper_enqueue(s));
        }
    }
    CK(cudaEventRecord(s.fence_out, s.work));
    CK(cudaStreamWaitEvent(s.stream, s.fence_out, 0));
    return SEG_OK;
}

int stepper_read(Stepper& s)
{
    const int n = (int)s.members.size();
    if (!n) return SEG_OK;
    CK(launch_gather_counters(s.d_jobs, n, s.d_gather, s.stream));
    CK(cudaMemcpyAsync(s.h_gather, s.d_gather, sizeof(Counters) * n, cudaMemcpyDeviceToHost, s.stream));
    CK(cudaStreamSynchronize(s.stream));
    for (int i = 0; i < n; i++) *s.members[i]->h_ctr = s.h_gather[i];
    return SEG_OK;
}

// Run `iters` iterations of every member; members whose particle buffers overflowed are
// regrown and finish their remaining iterations in further passes.
int stepper_step(Stepper& s, int iters)
{
    const int n = (int)s.members.size();
    std::vector<long long> target(n);
    int rc = SEG_OK;
    if (s.dirty && (rc = stepper_build(s)) != SEG_OK) return rc;
    rc = stepper_read(s);
    if (rc) return rc;
    for (int i = 0; i < n; i++) target[i] = s.members[i]->h_ctr->t + iters;
    int todo = iters;
    for (int pass = 0; pass < 64; pass++) {
        if (pass > 0 || todo > 0) {
            if (todo <= 0) break;
            rc = stepper_run(s, todo);
            if (rc) return rc;
            rc = stepper_read(s);
            if (rc) return rc;
        }
        todo = 0;
        bool regrown = false;
        for (int i = 0; i < n; i++) {
            seg_ctx* c = s.members[i];
            Counters& h = *c->h_ctr;
            if (h.error) return h.error;
            if (h.need) {
                rc = grow_particles(c, h.need);
                if (rc) return rc;
                // clear the overflow and move to a fresh tag so that no pixel-map or
                // look-back word of the abandoned pass can be taken for a current one
                h.need = 0;
                h.skip = h.converged;
                h.iter_tag += 1;
                CK(cudaMemcpyAsync(c->d_ctr, &h, sizeof h, cudaMemcpyHostToDevice, s.stream));
                CK(cudaStreamSynchronize(s.stream));
                regrown = true;
            }
        }
        if (regrown) {
            s.dirty = true;
            if (s.members.size() > 1) return SEG_OK;   // batch: members report their own t
            todo = (int)(target[0] - s.members[0]->h_ctr->t);
        }
        if (todo <= 0) break;
    }
    return SEG_OK;
}

int ensure_device(int dev)
{
    int cur = -1;
    CK(cudaGetDevice(&cur));
    if (cur != dev) CK(cudaSetDevice(dev));
    return SEG_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

int seg_estimate_bytes(const seg_params* p, int32_t nlabels, size_t* bytes)
{
    int rc = validate(p);
    if (rc) return rc;
    if (nlabels < 1 || !bytes) return SEG_EINVAL;
    if ((p->topology & SEG_TOPO_SPLIT) && p->max_labels && p->max_labels < nlabels) return SEG_EINVAL;
    Plan P;
    make_geometry(p, label_capacity(p, nlabels), 1, 254, P);
    *bytes = input_bytes(P.h.npix, p->dtype) + P.fixed.bytes +
             particle_bytes(default_pcap(P.h.npix, P.h.ndim), P.h.nbr_stride);
    return SEG_OK;
}

int seg_autotune(const seg_params* p, const void* image, const int32_t* labels0, int32_t iters, void* cuda_stream,
                 seg_params* best, seg_tune_entry* entries, int32_t max_entries, int32_t* n_entries)
{
    int rc = validate(p);
    if (rc) return rc;
    if (!image || !labels0 || !best || iters < 1 || max_entries < 0) return SEG_EINVAL;
    if (n_entries) *n_entries = 0;
    const int c0 = p->cell_edge ? p->cell_edge : std::max(1, (int)std::ceil(p->cutoff));
    static const int t2[5][3] = {{1, 16, 16}, {1, 32, 32}, {1, 32, 64}, {1, 64, 64}, {1, 64, 128}};
    static const int t3[5][3] = {{8, 8, 8}, {8, 8, 32}, {16, 16, 16}, {8, 16, 32}, {16, 16, 32}};
    const int (*tiles)[3] = p->ndim == 2 ? t2 : t3;
    std::vector<std::array<int, 4>> seen;   // (cell, tcz, tcy, tcx) already tried
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "autotune events");
    }
    int n = 0, first_err = SEG_OK;
    float best_ms = -1.0f;
    for (int ci = 0; ci < 2; ci++) {
        const int cell = c0 * (ci + 1);
        if (cell > 256) continue;
        for (int ti = 0; ti < 5; ti++) {
            seg_params q = *p;
            q.cell_edge = cell;
            q.tile[0] = p->ndim == 2 ? 0 : tiles[ti][0];
            q.tile[1] = tiles[ti][1];
            q.tile[2] = tiles[ti][2];
            std::array<int, 4> key = {cell, p->ndim == 2 ? 1 : std::max(1, q.tile[0] / cell),
                                      std::max(1, q.tile[1] / cell), std::max(1, q.tile[2] / cell)};
            if (std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
            seen.push_back(key);
            float ms = -1.0f;
            seg_ctx* c = nullptr;
            int r = seg_init(&q, image, labels0, cuda_stream, &c);
            if (r == SEG_OK) r = seg_step(c, 2, nullptr);
            if (r == SEG_OK) {
                if (cudaEventRecord(e0, stream) != cudaSuccess) r = SEG_ECUDA;
                if (r == SEG_OK) r = seg_step_async(c, iters);
                if (r == SEG_OK && cudaEventRecord(e1, stream) != cudaSuccess) r = SEG_ECUDA;
                if (r == SEG_OK && cudaEventSynchronize(e1) != cudaSuccess) r = SEG_ECUDA;
                if (r == SEG_OK) r = seg_poll(c, nullptr);
                float t = 0.0f;
                if (r == SEG_OK && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms = t / (float)iters;
                else if (r == SEG_OK) r = SEG_ECUDA;
            }
            if (c) seg_destroy(c);
            if (r != SEG_OK && first_err == SEG_OK) first_err = r;
            if (r != SEG_OK) ms = -1.0f;
            if (entries && n < max_entries) {
                entries[n].cell_edge = cell;
                for (int i = 0; i < 3; i++) entries[n].tile[i] = q.tile[i];
                entries[n].ms_per_iter = ms;
                entries[n].status = r;
            }
            n++;
            if (ms >= 0.0f && (best_ms < 0.0f || ms < best_ms)) {
                best_ms = ms;
                *best = q;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_entries) *n_entries = std::min(n, max_entries);
    if (best_ms < 0.0f) return first_err ? first_err : SEG_EINVAL;
    return SEG_OK;
}

int seg_init(const seg_params* p, const void* image, const int32_t* labels0, void* cuda_stream, seg_ctx** out)
{
    if (!out) return SEG_EINVAL;
    *out = nullptr;
    int rc = validate(p);
    if (rc) return rc;
    if (!image || !labels0) return SEG_EINVAL;
    const long long npix = p->shape[0] * p->shape[1] * p->shape[2];
    const size_t esz = p->dtype == SEG_F32 ? 4 : 2;
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    seg_ctx* c = new seg_ctx();
    c->params = *p;
    c->stream = stream;
    auto fail = [&](int code) {
        seg_destroy(c);
        return code;
    };
#define CKF(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return fail(cuda_fail(e_, #x)); } while (0)
    CKF(cudaGetDevice(&c->device));
    // inputs on the device, then one scan kernel for what the plan needs to know about them
    const size_t ib = align256(npix * esz + 1), lb = align256(npix * 4 + 1);
    cudaError_t e = dev_alloc((void**)&c->inputs, input_bytes(npix, p->dtype), stream);
    if (e != cudaSuccess) { cudaGetLastError(); c->inputs = nullptr; return fail(SEG_ENOMEM); }
    void* dI = c->inputs;
    int32_t* dL = (int32_t*)(c->inputs + ib);
    InputScan* dscan = (InputScan*)(c->inputs + ib + lb);
    CKF(cudaMemcpyAsync(dI, image, npix * esz, cudaMemcpyDefault, stream));
    CKF(cudaMemcpyAsync(dL, labels0, npix * 4, cudaMemcpyDefault, stream));
    InputScan scan{0x7fffffff, -0x7fffffff - 1, 0x7fffffff, -1, 0u, 0, 0, 0ull, 0ull};
    CKF(cudaMemcpyAsync(dscan, &scan, sizeof scan, cudaMemcpyHostToDevice, stream));
    CKF(launch_scan_inputs(dI, p->dtype, dL, p->ndim, (int)p->shape[0], (int)p->shape[1], (int)p->shape[2], dscan,
                           stream));
    CKF(cudaMemcpyAsync(&scan, dscan, sizeof scan, cudaMemcpyDeviceToHost, stream));
    CKF(cudaStreamSynchronize(stream));
    if (scan.lab_min < 0 || scan.lab_max >= (1 << 24) || scan.bad) return fail(SEG_EINVAL);
    if (p->model == SEG_PS_POISSON && scan.neg) return fail(SEG_EINVAL);   // Poisson counts are >= 0
    const int M0 = scan.lab_max + 1;                 // labels in use
    if ((p->topology & SEG_TOPO_SPLIT) && p->max_labels && p->max_labels < M0) return fail(SEG_EINVAL);
    const int M = label_capacity(p, M0);             // label tables (room for new labels from splits)
    int slot_lo = 1, slot_hi = 1;
    float maxabs = 0.0f;
    if (p->dtype == SEG_F32) {
        if (scan.slot_hi >= scan.slot_lo) { slot_lo = scan.slot_lo; slot_hi = scan.slot_hi; }
        std::memcpy(&maxabs, &scan.maxabs, sizeof maxabs);
    } else {
        maxabs = (float)scan.maxabs;
    }
    if (p->validate) {
        // every foreground label forms one connected component (union-find on the host)
        std::vector<int32_t> hl(npix);
        CKF(cudaMemcpy(hl.data(), dL, npix * 4, cudaMemcpyDeviceToHost));
        const int32_t* L0 = hl.data();
        const long long D = p->shape[0], H = p->shape[1], W = p->shape[2];
        std::vector<int64_t> parent(npix);
        std::iota(parent.begin(), parent.end(), 0);
        auto find = [&](int64_t a) {
            while (parent[a] != a) { parent[a] = parent[parent[a]]; a = parent[a]; }
            return a;
        };
        auto unite = [&](int64_t a, int64_t b) { a = find(a); b = find(b); if (a != b) parent[a] = b; };
        for (long long z = 0; z < D; z++)
            for (long long y = 0; y < H; y++)
                for (long long x = 0; x < W; x++) {
                    long long i = (z * H + y) * W + x;
                    if (!L0[i]) continue;
                    if (x + 1 < W && L0[i + 1] == L0[i]) unite(i, i + 1);
                    if (y + 1 < H && L0[i + W] == L0[i]) unite(i, i + W);
                    if (z + 1 < D && L0[i + W * H] == L0[i]) unite(i, i + W * H);
                }
        std::vector<int64_t> root(M, -1);
        for (long long i = 0; i < npix; i++) {
            if (!L0[i]) continue;
            int64_t r = find(i);
            if (root[L0[i]] < 0) root[L0[i]] = r;
            else if (root[L0[i]] != r) return fail(SEG_EINVAL);
        }
    }

    Plan P;
    make_geometry(p, M, slot_lo, slot_hi - slot_lo + 1, P);
    P.h.maxabs = maxabs;
    P.h.mu_floor64 = std::ldexp(std::max(1.0, (double)maxabs), -20);
    P.h.mu_floor32 = (float)P.h.mu_floor64;
    c->h = P.h;
    e = dev_alloc((void**)&c->arena, P.fixed.bytes, stream);
    if (e != cudaSuccess) { cudaGetLastError(); c->arena = nullptr; return fail(SEG_ENOMEM); }
    c->arena_bytes = P.fixed.bytes;
    // the plan recorded addresses of fields of P.h: re-point them into c->h
    for (auto& pr : P.fixed.parts) pr.first = (void**)((char*)&c->h + ((char*)pr.first - (char*)&P.h));
    P.fixed.assign(c->arena);
    c->h.I = dI;
    c->h.L = dL;
    c->d_ctr = c->h.ctr;
    setup_tma(c->h);
    long long pcap = initial_pcap(c->h.npix, c->h.ndim, (long long)scan.particles);
    size_t pb = particle_bytes(pcap, c->h.nbr_stride);
    e = dev_alloc((void**)&c->parena, pb, stream);
    if (e != cudaSuccess) { cudaGetLastError(); c->parena = nullptr; return fail(SEG_ENOMEM); }
    c->parena_bytes = pb;
    assign_particles(c->h, c->parena, pcap);
    e = dev_alloc((void**)&c->d_self, sizeof(Job), stream);
    if (e != cudaSuccess) { c->d_self = nullptr; return fail(cuda_fail(e, "job descriptor")); }
    if (!(c->h_ctr = pinned_counters())) return fail(cuda_fail(cudaErrorMemoryAllocation, "pinned counters"));

    const cudaError_t topo_err = ensure_topology_tables();
    if (topo_err != cudaSuccess) return fail(cuda_fail(topo_err, "topology tables"));
    topology_for_job(c->h);
    Counters hc{};
    hc.iter_tag = 1;
    hc.mode = p->gradient;
    hc.best_A = -1;
    hc.perim = (long long)scan.pairs;
    hc.n_labels = M0;
    memset(c->h_ctr, 0, sizeof(Counters));
    c->h_ctr->n_labels = M0;
    CKF(cudaMemsetAsync(c->h.pmap, 0, npix * 8, stream));
    CKF(cudaMemsetAsync(c->h.tile_word, 0, (size_t)c->h.ntiles * 8, stream));
    CKF(cudaMemsetAsync(c->h.st_n, 0, (size_t)M * 8, stream));
    CKF(cudaMemsetAsync(c->h.st_S, 0, (size_t)M * (p->dtype == SEG_F32 ? c->h.nS : 1) * 8, stream));
    CKF(cudaMemsetAsync(c->h.st_Q, 0, (size_t)M * (p->dtype == SEG_F32 ? c->h.nQ : 1) * 8, stream));
    if (c->h.sf64) CKF(cudaMemsetAsync(c->h.sf64, 0, 2 * (size_t)M * 8, stream));
    if (c->h.sk32) CKF(cudaMemsetAsync(c->h.sk32, 0, 2 * (size_t)M * 8, stream));
    CKF(cudaMemcpyAsync((void*)c->h.klut, P.klut.data(), P.klut.size() * 4, cudaMemcpyHostToDevice, stream));
    CKF(cudaMemcpyAsync((void*)c->h.klut_lo, P.klut_lo.data(), P.klut_lo.size() * 4, cudaMemcpyHostToDevice, stream));
    CKF(cudaMemcpyAsync((void*)c->h.klut64, P.klut64.data(), P.klut64.size() * 8, cudaMemcpyHostToDevice, stream));
    if (!P.ps_off.empty())
        CKF(cudaMemcpyAsync((void*)c->h.ps_off, P.ps_off.data(), P.ps_off.size() * sizeof(int4), cudaMemcpyHostToDevice, stream));
    CKF(cudaMemcpyAsync((void*)c->h.nb_off, P.nb_off.data(), P.nb_off.size() * sizeof(int4), cudaMemcpyHostToDevice, stream));
    if (c->h.topo_fuse) {
        CKF(cudaMemsetAsync(c->h.fz_key, 0xff, (size_t)c->h.fz_cap * 8, stream));
        CKF(cudaMemsetAsync(c->h.fz_cnt, 0, (size_t)c->h.fz_cap * 4, stream));
        CKF(cudaMemsetAsync(c->h.fz_to, 0xff, (size_t)M * 4, stream));
        CKF(cudaMemsetAsync(c->h.fz_used, 0, (size_t)M * 4, stream));
    }
    if (!P.cv_off.empty())
        CKF(cudaMemcpyAsync((void*)c->h.cv_off, P.cv_off.data(), P.cv_off.size() * sizeof(int4), cudaMemcpyHostToDevice, stream));
    CKF(cudaMemcpyAsync(c->d_ctr, &hc, sizeof hc, cudaMemcpyHostToDevice, stream));
    CKF(cudaMemcpyAsync(c->d_self, &c->h, sizeof(Job), cudaMemcpyHostToDevice, stream));
    CKF(launch_stats_init(c->d_self, 0, npix, stream));
    CKF(launch_stats_finalize(c->d_self, 1, stream));
    CKF(cudaStreamSynchronize(stream));
    c->own = new Stepper();
    c->own->device = c->device;
    c->own->stream = stream;
    CKF(cudaDeviceGetAttribute(&c->own->sms, cudaDevAttrMultiProcessorCount, c->device));
    c->own->members.push_back(c);
#undef CKF
    *out = c;
    return SEG_OK;
}

int seg_step(seg_ctx* c, int32_t iters, seg_status* out)
{
    if (!c || iters < 0) return SEG_EINVAL;
    if (c->batch) return SEG_ESTATE;
    int rc = ensure_device(c->device);
    if (rc) return rc;
    rc = stepper_step(*c->own, iters);
    if (rc) return rc;
    if (iters == 0) {
        rc = stepper_read(*c->own);
        if (rc) return rc;
    }
    if (out) *out = c->h_ctr->last;
    return c->h_ctr->error ? c->h_ctr->error : SEG_OK;
}

int seg_step_async(seg_ctx* c, int32_t iters)
{
    if (!c || iters < 0) return SEG_EINVAL;
    if (c->batch) return SEG_ESTATE;
    int rc = ensure_device(c->device);
    if (rc) return rc;
    return stepper_run(*c->own, iters);
}

int seg_poll(seg_ctx* c, seg_status* out)
{
    if (!c) return SEG_EINVAL;
    int rc = ensure_device(c->device);
    if (rc) return rc;
    Stepper& s = c->batch ? c->batch->st : *c->own;
    if (s.dirty && (rc = stepper_build(s)) != SEG_OK) return rc;
    rc = stepper_read(s);
    if (rc) return rc;
    if (out) *out = c->h_ctr->last;
    return c->h_ctr->error ? c->h_ctr->error : SEG_OK;
}

int seg_profile(seg_ctx* c, int32_t on)
{
    if (!c) return SEG_EINVAL;
    if (c->batch) return SEG_ESTATE;
    int rc = ensure_device(c->device);
    if (rc) return rc;
    return stepper_set_profile(*c->own, on != 0);
}

int seg_stage_times(seg_ctx* c, float* ms, int32_t n)
{
    if (!c) return SEG_EINVAL;
    if (c->batch) return SEG_ESTATE;
    int rc = ensure_device(c->device);
    if (rc) return rc;
    return stepper_stage_times(*c->own, ms, n);
}

int seg_labels(seg_ctx* c, int32_t* out, size_t n_out)
{
    if (!c || !out) return SEG_EINVAL;
    if ((long long)n_out < c->h.npix) return SEG_EINVAL;
    int rc = ensure_device(c->device);
    if (rc) return rc;
    CK(cudaMemcpyAsync(out, c->h.L, c->h.npix * 4, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return SEG_OK;
}

int seg_particles(seg_ctx* c, const seg_particle_buffers* b, int64_t cap, int64_t* n)
{
    if (!c || !b || !n || cap < 0) return SEG_EINVAL;
    int rc = ensure_device(c->device);
    if (rc) return rc;
    unsigned np = 0;
    CK(cudaMemcpyAsync(&np, &c->d_ctr->n_particles, 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if ((long long)np > c->h.pcap) np = (unsigned)c->h.pcap;
    *n = np;
    long long k = std::min<long long>(np, cap);
    if (k > 0) {
        if (b->idx) CK(cudaMemcpyAsync(b->idx, c->h.p_idx, k * 4, cudaMemcpyDefault, c->stream));
        if (b->l) CK(cudaMemcpyAsync(b->l, c->h.p_l, k * 4, cudaMemcpyDefault, c->stream));
        if (b->c) CK(cudaMemcpyAsync(b->c, c->h.p_c, k * 4, cudaMemcpyDefault, c->stream));
        if (b->dE) CK(cudaMemcpyAsync(b->dE, c->h.p_dE, k * 4, cudaMemcpyDefault, c->stream));
        if (b->eE) CK(cudaMemcpyAsync(b->eE, c->h.p_eE, k * 4, cudaMemcpyDefault, c->stream));
        if (b->g) CK(cudaMemcpyAsync(b->g, c->h.p_g, k * 4, cudaMemcpyDefault, c->stream));
        if (b->eg) CK(cudaMemcpyAsync(b->eg, c->h.p_eg, k * 4, cudaMemcpyDefault, c->stream));
        if (b->key) CK(cudaMemcpyAsync(b->key, c->h.p_key, k * 8, cudaMemcpyDefault, c->stream));
        if (b->flags) CK(cudaMemcpyAsync(b->flags, c->h.p_flags, k, cudaMemcpyDefault, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return SEG_OK;
}

int seg_stats(seg_ctx* c, int64_t* n, double* S, double* Q, int32_t max_labels)
{
    if (!c || max_labels < 0) return SEG_EINVAL;
    int rc = ensure_device(c->device);
    if (rc) return rc;
    int k = std::min(max_labels, c->h.M);
    if (k > 0) {
        // the sums of squares are rounded from the exact sums here (the iteration needs only S)
        if (Q) CK(launch_stats_finalize(c->d_self, 1, c->stream));
        if (n) CK(cudaMemcpyAsync(n, c->h.st_n, k * 8, cudaMemcpyDeviceToHost, c->stream));
        if (S) CK(cudaMemcpyAsync(S, c->h.S64, k * 8, cudaMemcpyDeviceToHost, c->stream));
        if (Q) CK(cudaMemcpyAsync(Q, c->h.Q64, k * 8, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    for (int m = k; m < max_labels; m++) {
        if (n) n[m] = 0;
        if (S) S[m] = 0.0;
        if (Q) Q[m] = 0.0;
    }
    return SEG_OK;
}

int seg_get_state(seg_ctx* c, seg_state* out)
{
    if (!c || !out) return SEG_EINVAL;
    Counters h;
    int rc = ensure_device(c->device);
    if (rc) return rc;
    CK(cudaMemcpyAsync(&h, c->d_ctr, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    out->t = h.t;
    out->best_A = h.best_A;
    out->t_best = h.t_best;
    out->mode = h.mode;
    out->converged = h.converged;
    return SEG_OK;
}

int seg_set_state(seg_ctx* c, const seg_state* in)
{
    if (!c || !in) return SEG_EINVAL;
    if (in->mode != SEG_SOBOLEV && in->mode != SEG_L2) return SEG_EINVAL;
    if (in->t < 0 || in->t_best < 0 || in->t_best > in->t || in->best_A < -1) return SEG_EINVAL;
    int rc = ensure_device(c->device);
    if (rc) return rc;
    Counters h;
    CK(cudaMemcpyAsync(&h, c->d_ctr, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    h.t = in->t;
    h.best_A = in->best_A;
    h.t_best = in->t_best;
    h.mode = in->mode;
    h.converged = in->converged ? 1 : 0;
    h.skip = h.converged || h.error || h.need;
    CK(cudaMemcpyAsync(c->d_ctr, &h, sizeof h, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return SEG_OK;
}

int seg_info(seg_ctx* c, int32_t* nlabels, int64_t shape[3])
{
    if (!c) return SEG_EINVAL;
    if (nlabels) *nlabels = c->h_ctr->n_labels;   // grows when regions split
    if (shape) {
        shape[0] = c->h.D;
        shape[1] = c->h.H;
        shape[2] = c->h.W;
    }
    return SEG_OK;
}

void seg_destroy(seg_ctx* c)
{
    if (!c) return;
    if (c->batch) seg_batch_remove(c->batch, c);
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != c->device) cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->own) {
        stepper_release(*c->own);
        delete c->own;
    }
    dev_free(c->arena, c->stream);
    dev_free(c->parena, c->stream);
    dev_free(c->d_self, c->stream);
    dev_free(c->inputs, c->stream);
    release_counters(c->h_ctr);
    cudaGetLastError();
    if (cur >= 0 && cur != c->device) cudaSetDevice(cur);
    delete c;
}

int seg_batch_create(void* cuda_stream, seg_batch** out)
{
    if (!out) return SEG_EINVAL;
    seg_batch* b = new seg_batch();
    b->st.stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&b->st.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->st.sms, cudaDevAttrMultiProcessorCount, b->st.device);
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "seg_batch_create");
    }
    *out = b;
    return SEG_OK;
}

int seg_batch_add(seg_batch* b, seg_ctx* c)
{
    if (!b || !c) return SEG_EINVAL;
    if (c->batch) return SEG_ESTATE;
    if (c->device != b->st.device) return SEG_EINVAL;
    CK(cudaStreamSynchronize(c->stream));
    b->st.members.push_back(c);
    c->batch = b;
    b->st.dirty = true;
    return SEG_OK;
}

int seg_batch_remove(seg_batch* b, seg_ctx* c)
{
    if (!b || !c || c->batch != b) return SEG_EINVAL;
    CK(cudaStreamSynchronize(b->st.stream));
    auto& m = b->st.members;
    m.erase(std::remove(m.begin(), m.end(), c), m.end());
    c->batch = nullptr;
    b->st.dirty = true;
    return SEG_OK;
}

int seg_batch_size(seg_batch* b) { return b ? (int)b->st.members.size() : 0; }

int seg_batch_profile(seg_batch* b, int32_t on)
{
    if (!b) return SEG_EINVAL;
    int rc = ensure_device(b->st.device);
    if (rc) return rc;
    return stepper_set_profile(b->st, on != 0);
}

int seg_batch_stage_times(seg_batch* b, float* ms, int32_t n)
{
    if (!b) return SEG_EINVAL;
    int rc = ensure_device(b->st.device);
    if (rc) return rc;
    return stepper_stage_times(b->st, ms, n);
}

int seg_kernel_launches(uint64_t* out)
{
    if (!out) return SEG_EINVAL;
    *out = (uint64_t)g_kernel_launches.load(std::memory_order_relaxed);
    return SEG_OK;
}

int seg_batch_step(seg_batch* b, int32_t iters, seg_status* statuses, int32_t n_statuses)
{
    if (!b || iters < 0) return SEG_EINVAL;
    int rc = ensure_device(b->st.device);
    if (rc) return rc;
    rc = stepper_step(b->st, iters);
    if (rc) return rc;
    if (iters == 0) {
        rc = stepper_read(b->st);
        if (rc) return rc;
    }
    int err = SEG_OK;
    for (size_t i = 0; i < b->st.members.size(); i++) {
        const Counters& h = *b->st.members[i]->h_ctr;
        if (statuses && (int)i < n_statuses) statuses[i] = h.last;
        if (h.error && !err) err = h.error;
    }
    return err;
}

int seg_batch_step_async(seg_batch* b, int32_t iters)
{
    if (!b || iters < 0) return SEG_EINVAL;
    int rc = ensure_device(b->st.device);
    if (rc) return rc;
    return stepper_run(b->st, iters);
}

int seg_batch_poll(seg_batch* b, seg_status* statuses, int32_t n_statuses)
{
    if (!b) return SEG_EINVAL;
    int rc = ensure_device(b->st.device);
    if (rc) return rc;
    if (b->st.dirty && (rc = stepper_build(b->st)) != SEG_OK) return rc;
    rc = stepper_read(b->st);
    if (rc) return rc;
    int err = SEG_OK;
    for (size_t i = 0; i < b->st.members.size(); i++) {
        const Counters& h = *b->st.members[i]->h_ctr;
        if (statuses && (int)i < n_statuses) statuses[i] = h.last;
        if (h.error && !err) err = h.error;
    }
    return err;
}

void seg_batch_destroy(seg_batch* b)
{
    if (!b) return;
    if (b->st.stream) cudaStreamSynchronize(b->st.stream);
    for (auto* c : b->st.members) c->batch = nullptr;
    stepper_release(b->st);
    delete b;
}

int seg_set_psf(seg_ctx* c, const double* k, int32_t radius)
{
    if (!c || !k || radius < 0 || radius > SEG_PSF_MAX_RADIUS) return SEG_EINVAL;
    if (c->h.model != SEG_PC_DECONV) return SEG_ESTATE;
    for (int u = 0; u <= 2 * radius; u++)
        if (!std::isfinite(k[u]) || k[u] != k[2 * radius - u]) return SEG_EINVAL;
    int rc = ensure_device(c->device);
    if (rc) return rc;
    if (c->batch) CK(cudaStreamSynchronize(c->batch->st.stream));
    CK(cudaStreamSynchronize(c->stream));
    c->h.psf_r = radius;
    CK(cudaMemcpyAsync(c->h.psf, k, sizeof(double) * (2 * radius + 1), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_self, &c->h, sizeof(Job), cudaMemcpyHostToDevice, c->stream));
    CK(launch_psf_norms(c->d_self, c->h, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->own->dirty = true;                       // the steppers' job tables are rebuilt
    if (c->batch) c->batch->st.dirty = true;
    return SEG_OK;
}

int seg_debug_inject(seg_ctx* c, int32_t what)
{
    if (!c || (what != SEG_INJECT_NONE && what != SEG_INJECT_WITHHELD_COPY)) return SEG_EINVAL;
    int rc = ensure_device(c->device);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream));
    c->h.inject = what;
    CK(cudaMemcpyAsync(c->d_self, &c->h, sizeof(Job), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->own->dirty = true;                       // the stepper's job table is rebuilt
    if (c->batch) c->batch->st.dirty = true;
    return SEG_OK;
}

int seg_debug_simple(int32_t ndim, const uint32_t* masks, int32_t n, uint8_t* out)
{
    if ((ndim != 2 && ndim != 3) || n < 0 || (n && (!masks || !out))) return SEG_EINVAL;
    if (!n) return SEG_OK;
    CK(ensure_topology_tables());
    unsigned* dm = nullptr;
    unsigned char* dout = nullptr;
    CK(cudaMalloc(&dm, (size_t)n * 4));
    cudaError_t e = cudaMalloc(&dout, n);
    if (e == cudaSuccess) e = cudaMemcpy(dm, masks, (size_t)n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_debug_simple(dm, ndim, n, dout, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, n, cudaMemcpyDeviceToHost);
    cudaFree(dm);
    if (dout) cudaFree(dout);
    if (e != cudaSuccess) return cuda_fail(e, "seg_debug_simple");
    return SEG_OK;
}

const char* seg_strerror(int code)
{
    switch (code) {
        case SEG_OK: return "ok";
        case SEG_EINVAL: return "invalid argument";
        case SEG_ENOMEM: return "out of device memory";
        case SEG_ECUDA: return "CUDA runtime error";
        case SEG_ETIMEOUT: return "bounded device wait timed out";
        case SEG_ESTATE: return "invalid state for this call";
        default: return "unknown error";
    }
}

const char* seg_last_cuda_error(void) { return g_last_cuda.c_str(); }

}  // extern "C"
