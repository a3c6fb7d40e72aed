// Internal declarations shared by the libseg CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "seg.h"

namespace segk {

// Bounded waits: every device-side wait gives up, and raises SEG_ETIMEOUT, after kWaitNs of
// wall time on the GPU's global timer or kSpinLimit polls, whichever comes first.
constexpr unsigned kSpinLimit = 1u << 26;
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct WaitBound {
    unsigned long long t0 = 0;
    unsigned spins = 0;
    // called once per failed poll; true once the wait has run out
    __device__ __forceinline__ bool expired()
    {
        if (spins++ == 0) {
            t0 = global_ns();
            return false;
        }
        if (spins > kSpinLimit) return true;
        return (spins & 255u) == 0 && global_ns() - t0 > kWaitNs;
    }
};

// region models whose data term uses local means over a ball (the piecewise-smooth ones)
__host__ __device__ __forceinline__ bool is_ps(int model) { return model == SEG_PS || model == SEG_PS_POISSON; }

constexpr unsigned char kFlagFixup = 1, kFlagCand = 2, kFlagAcc = 4, kFlagSplit = 8;
constexpr int kUndecided = 0, kAccepted = 1, kRejected = 2;

// Division by an invariant 32-bit divisor with one multiply-high (Granlund & Montgomery,
// "Division by invariant integers using multiplication", 1994, Fig. 4.1).
struct FastDiv {
    unsigned d, m;
    int s1, s2;
};

inline FastDiv make_fastdiv(unsigned d)
{
    int l = 0;
    while ((1ull << l) < d) l++;
    FastDiv f;
    f.d = d;
    f.m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 1 ? l - 1 : 0;
    return f;
}

__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f)
{
    unsigned t = __umulhi(n, f.m);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

// Per-job counters and optimiser state, device memory, zeroed at seg_init.
struct Counters {
    unsigned n_particles;   // particles of the current iteration
    unsigned need;          // particles required when the capacity was exceeded (sticky until regrown)
    unsigned n_flag;        // particles queued for the FP64 recompute
    unsigned n_cand;        // candidates
    unsigned n_accepted;
    unsigned n_osc;
    unsigned mis_rounds;
    int error;              // SEG_E* raised on the device (sticky)
    unsigned iter_tag;      // grows by one per executed iteration; tags pixel-map and look-back words
    int mode;               // gradient type of the next iteration
    int converged;
    int skip;               // nonzero: this iteration does nothing (converged, error or overflow)
    long long t;            // iterations done
    long long best_A;       // smallest accepted count so far, -1 before the first iteration
    long long t_best;
    long long cum_particles; // particles summed over executed iterations
    long long perim;        // |Gamma|: adjacent pixel pairs with different labels (current labels)
    int n_labels;           // labels in use (grows when regions split)
    unsigned n_split;       // accepted moves of the iteration admitted by the split rule
    unsigned n_newcomp;     // pieces given new labels by the iteration's relabelling
    unsigned n_fpairs;      // fusion: touching label pairs listed in the hash table
    unsigned n_fused;       // fusion: pairs fused by the last fusion pass
    unsigned n_void;        // candidates whose FP64 key turned out >= 0 (dropped before the rounds)
    long long g_lim;        // E = |Gamma| mode: interaction partners have d^2 < g_lim
    seg_status last;        // status of the last executed iteration
};

// Everything a kernel needs about one segmentation job; lives in device memory (the
// tensor maps inside need 64-byte alignment).
struct alignas(64) Job {
    unsigned char tmap_L[128];  // TMA tensor map of the label image (when use_tma)
    unsigned char tmap_I[128];  // ... of the image (2D piecewise smooth with staged image)
    int use_tma;              // tile boxes arrive by tensor copies
    int tma_bx;               // box width in elements (multiple of 8) from an x aligned down to 8
    int ndim, D, H, W;
    long long npix;
    FastDiv fd_W, fd_HW, fd_cell;   // divide by W, by W*H, by the cell edge
    int dtype, model, conn;
    int cell;                 // cell-list edge (all axes in 3D; x and y in 2D)
    int ncx, ncy, ncz;        // cells per axis (ncz = D in 2D)
    int tcx, tcy, tcz;        // cells per tile per axis
    int ntx, nty, ntz, ntiles;
    int halo;                 // label/image halo staged by extraction
    int ps_staged;            // 2D piecewise smooth with the ball inside the staged halo
    int ps_int;               // ball sums exact in int64 fixed point (value = q * 2^e_min)
    int ps_exact64;           // ... and every FP64 partial sum over a ball is exact (order free)
    int ps_q32;               // fixed-point pixel values fit in int32 (staged as int32)
    int e_min;                // exponent of the fixed-point unit
    float unit32;             // 2^e_min as a float
    double unit64;            // 2^e_min as a double
    float maxabs;             // largest |I| of the image
    float mu_floor32;         // Poisson model: local means below this are taken as this
    double mu_floor64;
    float lambda32;           // length-prior weight (0 with the curvature regulariser)
    double lambda64;
    int curv;                 // curvature regulariser: dE += w (A_l - A_c) over the ball cv_off
    int cv_n;
    const int4* cv_off;       // ... ball offsets (dz, dy, dx, d2), row-major
    float curv_w32;           // ... w rounded to float
    double curv_w64;          // ... w
    double cutoff, E;         // E = 2 * cutoff (Eq. 5 length scale)
    int r2max;                // interaction partners: squared distance <= r2max  (< cutoff^2)
    int ps_n;                 // piecewise-smooth ball offsets, row-major (dz, dy, dx, d2)
    const int4* ps_off;
    int nb_n;                 // offsets with d2 <= r2max, row-major (for the FP64 recompute)
    const int4* nb_off;
    const float* klut;        // K(sqrt(d2)) rounded to float, d2 = 0..r2max
    const float* klut_lo;     // ... and the rest, K - klut rounded to float (the pair holds 48 bits)
    const double* klut64;     // K(sqrt(d2)) in FP64, Eq. 5 evaluated in the order written
    int global_E;             // Eq. 6 with E = |Gamma| (all pairs) while in Sobolev mode
    int gd2max;               // ... largest squared distance within the image
    float* gK32;              // ... K(sqrt(d2)) for E = |Gamma| of the iteration, float
    float* gK32l;             // ... and the rest, gK64 - gK32 rounded to float
    double* gK64;             // ... and FP64 (Eq. 5 in the order written); 0 outside the support
    int psf_r;                // deconvolving model: PSF profile radius, -1 until seg_set_psf
    double* psf;              // ... taps k(-r..r) (room for 2 SEG_PSF_MAX_RADIUS + 1)
    double* psf_n;            // ... per axis sum of k(u)^2 over the in-image offsets: x [W], y [H], z [D]
    double* dc_T;             // ... FP64 fields of the separable passes [npix]
    double* dc_T2;            // ... (3D) [npix]
    double* dc_R;             // ... R = I - J [npix]
    double* dc_G;             // ... G = K * R at the particle pixels of the iteration [npix]
    int M;                    // number of labels
    int osc_window;           // L2 fallback window (0 = never)
    const unsigned* simple_tab;   // simple-point decisions, one bit per neighbourhood mask (this job's dimension)
    const unsigned* topo_adjF;    // foreground adjacency of the neighbour positions (26 masks)
    unsigned topo_touch, topo_nF; // 4- (6-) neighbours of the centre; the foreground count's neighbourhood
    int topo_vanish;          // a region's last pixel may leave it (SEG_TOPO_VANISH)
    int topo_split;           // a region may split (SEG_TOPO_SPLIT); M is then the label capacity
    int* cc_parent;           // ... relabelling: union-find parent per pixel [npix]
    int* cc_newl;             // ... new label of each piece, at the piece's root pixel [npix]
    int* cc_first;            // ... smallest pixel index of each label [M]
    int* cc_list;             // ... roots of the pieces that get new labels [M]
    int topo_fuse;            // touching regions may fuse (SEG_TOPO_FUSE)
    double fz_lam64;          // ... length weight of the shared boundary
    unsigned fz_cap;          // ... hash table slots (power of two)
    unsigned long long* fz_key;   // ... (a << 32 | b) per slot, ~0 when empty [fz_cap]
    unsigned* fz_cnt;         // ... adjacent pixel pairs of the slot's labels [fz_cap]
    unsigned* fz_list;        // ... occupied slots, then per listed pair: [fz_cap]
    unsigned long long* fz_ab;    // ... key [fz_cap]
    unsigned long long* fz_u;     // ... dE in unsigned order [fz_cap]
    unsigned* fz_B;           // ... shared pairs [fz_cap]
    int* fz_state;            // ... open / taken / out [fz_cap]
    unsigned long long* fz_best_u;   // ... per label: smallest open dE, then key [M]
    unsigned long long* fz_best_ab;
    int* fz_used;             // ... per label: fused in this pass [M]
    int* fz_to;               // ... per label: the label it fused into, or -1 [M]
    int* fz_done;             // ... labels fused away by the last pass [M]
    int inject;               // test-only fault injection (SEG_INJECT_*)
    int nbr_stride;           // neighbour-list slots per candidate: 8 (2D) | 26 (3D)
    int slot_lo, nS, nQ;      // exact float32 sums: exponent slots [slot_lo, slot_lo + nS)
    const void* I;
    int* L;
    unsigned long long* pmap; // per pixel: (iter_tag << 32) | index of the pixel's first particle
    long long pcap;
    unsigned* p_idx;
    int* p_l;
    int* p_c;
    float* p_dE;              // energy difference: the FP64 value rounded to float ...
    float* p_dEl;             // ... and the rest of it, rounded to float
    float* p_eE;              // ... bound on |p_dE - FP64 value|
    double* p_dE64;           // ... the FP64 value (with the curvature regulariser: the data term until
                              //     the ball term is added)
    float* p_g;
    float* p_eg;
    double* p_key;
    unsigned long long* p_nbm;   // topology masks: neighbours holding l (low word) and c (high word)
    unsigned char* p_flags;
    long long* p_qc;          // piecewise smooth with exact sums: sum of q(I) over the c part of the ball
    long long* p_ql;          //   ... over the own-label part
    int* p_nc;                //   pixel counts of the two parts
    int* p_nl;
    int* pix_cand;            // at a pixel's first particle: its candidate slot or -1
    unsigned* flag_list;
    unsigned* cell_start;
    unsigned* cell_count;
    unsigned long long* tile_word;  // decoupled look-back: (tag << 34) | (status << 32) | value
    unsigned* tile_start;
    unsigned* tile_count;
    long long* st_n;          // [M]
    long long* st_S;          // u16: [M]; f32: [M * nS] mantissa sums per exponent slot
    long long* st_Q;          // u16: [M]; f32: [M * nQ] 24-bit limbs of squared mantissas
    int stats_mode;           // SEG_STATS_*: the sums of I and I^2 above are kept only when exact
    double* sf64;             // SEG_STATS_F64: [2M] S then Q per label
    unsigned long long* sk32; // SEG_STATS_KAHAN32: [2M] (sum | compensation << 32) float pairs, S then Q
    double* S64;
    double* Q64;
    double* mu64;
    double* wp64;             // n / (n + 1)
    double* wm64;             // n / (n - 1), 0 for n <= 1
    float* mu32;
    float* wp32;
    float* wm32;
    int* c_best;              // candidate -> particle
    unsigned long long* c_key;    // the candidate's key as an order-preserving integer (ordered_key)
    unsigned* c_pix;
    float2* c_ge;             // the candidate's gradient as a float and its bound (0: the key is exact)
    int* c_state;
    int* c_nbr;               // smaller-key neighbouring candidates, nbr_stride slots per candidate
    int* c_nnbr;
    Counters* ctr;
};

// A set of jobs of one dimensionality, stepped by one launch per stage.
struct Group {
    const Job* jobs;          // device array of all jobs of the batch
    const int* job_ids;       // jobs of this group
    const unsigned* tile_prefix;   // njobs + 1 exclusive prefix of tiles
    int njobs;
    unsigned total_tiles;
    unsigned* ticket;         // extraction tile ticket
};

struct BatchCtl {
    unsigned ticket[2];       // per group
    int err;
    unsigned rounds_done;     // selection rounds of the last iteration
    unsigned pad[7];
};

// Image value as an exact fixed-point integer: value = q * 2^e_min. For float32 images
// q = +-mantissa * 2^(slot - slot_lo); for uint16 images q is the value itself.
__device__ __forceinline__ long long fixed_of_f32(float f, int slot_lo)
{
    unsigned bits = __float_as_uint(f);
    int eb = (int)((bits >> 23) & 0xffu);
    unsigned long long m = bits & 0x7fffffu;
    if (eb == 0) eb = 1; else m |= 0x800000ull;
    if (m == 0) return 0;
    long long q = (long long)(m << (eb - slot_lo));
    return (bits >> 31) ? -q : q;
}

__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) { return *(const volatile unsigned*)p; }
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p)
{
    return *(const volatile unsigned long long*)p;
}

// pixel coordinates of a linear index
__device__ __forceinline__ void pix_coords(const Job& J, unsigned gi, int& x, int& y, int& z)
{
    unsigned zy = fdiv(gi, J.fd_W);
    x = (int)(gi - zy * (unsigned)J.W);
    if (J.ndim == 3) {
        unsigned zz = fdiv(gi, J.fd_HW);
        z = (int)zz;
        y = (int)(zy - zz * (unsigned)J.H);
    } else {
        z = 0;
        y = (int)zy;
    }
}

// Block-wide exclusive scan of one unsigned per thread.
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* s_warp, unsigned& total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        unsigned a = lane < nw ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, a, o);
            if (lane >= o) a += y;
        }
        if (lane < nw) s_warp[lane] = a;       // inclusive warp totals
    }
    __syncthreads();
    unsigned before = w > 0 ? s_warp[w - 1] : 0u;
    total = s_warp[(blockDim.x >> 5) - 1];
    return before + x - v;
}

// Pixel box and cell range of tile k of a job.
struct TileBox {
    int x0, x1, y0, y1, z0, z1;   // pixel box of the tile
    int cx0, cy0, cz0;            // first cell
    int ccx, ccy, ccz;            // cells in the tile
};

__device__ __forceinline__ TileBox tile_box(const Job& J, unsigned k)
{
    TileBox b;
    int tx = (int)(k % (unsigned)J.ntx);
    int ty = (int)((k / (unsigned)J.ntx) % (unsigned)J.nty);
    int tz = (int)(k / ((unsigned)J.ntx * (unsigned)J.nty));
    int s = J.cell, sz = J.ndim == 3 ? J.cell : 1;
    b.cx0 = tx * J.tcx; b.cy0 = ty * J.tcy; b.cz0 = tz * J.tcz;
    b.ccx = min(J.tcx, J.ncx - b.cx0);
    b.ccy = min(J.tcy, J.ncy - b.cy0);
    b.ccz = min(J.tcz, J.ncz - b.cz0);
    b.x0 = b.cx0 * s; b.x1 = min(J.W, (b.cx0 + b.ccx) * s);
    b.y0 = b.cy0 * s; b.y1 = min(J.H, (b.cy0 + b.ccy) * s);
    b.z0 = b.cz0 * sz; b.z1 = min(J.D, (b.cz0 + b.ccz) * sz);
    return b;
}

// Which job / tile a tile ticket maps to.
__device__ __forceinline__ int group_job_of_tile(const Group& g, unsigned t)
{
    int lo = 0, hi = g.njobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (g.tile_prefix[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Candidate selection helpers shared by the kernels that select (the interaction kernel for the
// local modes, the selection kernel for E = |Gamma|).

// number of components of set S (adjacency adj) that meet `touch` (all if touch == 0); stops at 2
__device__ __forceinline__ int components(unsigned S, const unsigned* adj, unsigned touch)
{
    int count = 0;
    while (S) {
        unsigned comp = S & (0u - S);
        unsigned frontier = comp;
        while (frontier) {
            int a = __ffs(frontier) - 1;
            frontier &= frontier - 1;
            unsigned nb = adj[a] & S & ~comp;
            comp |= nb;
            frontier |= nb;
        }
        S &= ~comp;
        if (!touch || (comp & touch)) {
            if (++count > 1) return count;
        }
    }
    return count;
}

// Topological control: removal from l (foreground) and addition to c (foreground)
// must both be simple, so regions neither split, vanish, merge nor change holes. The
// neighbourhood enters as two bit masks, written by extraction while it held the labels: bit k
// of ml (mc) is set when the k-th neighbour (dz, dy, dx ascending, the centre skipped) holds l
// (c); a neighbour outside the image holds neither. With SEG_TOPO_VANISH the removal of a
// region's last pixel is admissible too: no 4- (6-) neighbour holds l (every foreground label
// being one connected component). With SEG_TOPO_SPLIT a removal whose foreground number is
// >= 2 is admissible too. Returns 0 (not admissible), 1, or 2 (admissible by the split rule).
__device__ __forceinline__ int admissible(const Job& J, int l, int c, unsigned long long masks)
{
    const unsigned ml = (unsigned)masks, mc = (unsigned)(masks >> 32);
    // both table words are loaded before either is tested, so that their latencies overlap
    const unsigned* tab = J.simple_tab;
    const unsigned wc = c != 0 ? __ldg(tab + (mc >> 5)) : 0xffffffffu;
    const unsigned wl = l != 0 ? __ldg(tab + (ml >> 5)) : 0xffffffffu;
    if (!((wc >> (mc & 31u)) & 1u)) return 0;
    if ((wl >> (ml & 31u)) & 1u) return 1;
    if (J.topo_vanish && (ml & J.topo_touch) == 0) return 1;
    if (J.topo_split && components(ml & J.topo_nF, J.topo_adjF, J.topo_touch) >= 2) return 2;
    return 0;
}

// An integer image of a finite double that keeps its order: the sign bit set for x >= 0, all bits
// flipped for x < 0 (-0 maps to the image of +0, as the two compare equal)
__device__ __forceinline__ unsigned long long ordered_key(double k)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(k);
    if (b == 0x8000000000000000ull) b = 0ull;
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// queue candidate slot s of job J for the FP64 recompute
__device__ __forceinline__ void queue_fixup(const Job& J, unsigned s, unsigned p)
{
    J.p_flags[p] |= kFlagFixup;
    const unsigned f = atomicAdd(&J.ctr->n_flag, 1u);
    J.flag_list[f] = s;
}

// Deconvolving model: the last separable pass of G = K * R at pixel gi (along y in 2D, z in
// 3D), over the field the other passes left, taps in ascending offset, fused multiply-adds.
__device__ __forceinline__ double deconv_G(const Job& J, unsigned gi, int y, int z)
{
    const int r = J.psf_r;
    const bool d3 = J.ndim == 3;
    const int t = d3 ? z : y;
    const int extent = d3 ? J.D : J.H;
    const long long stride = d3 ? (long long)J.W * J.H : (long long)J.W;
    const double* f = d3 ? J.dc_T2 : J.dc_T;
    const int lo = max(-r, -t), hi = min(r, extent - 1 - t);
    long long q = (long long)gi + (long long)lo * stride;
    double acc = 0.0;
    for (int u = lo; u <= hi; u++, q += stride) acc = __fma_rn(J.psf[u + r], f[q], acc);
    return acc;
}

// ... and its data-term change for moving the pixel at (x, y, z) from l to c with theta held:
// d^2 |K_x|^2 - 2 d G, d = theta_c - theta_l, |K_x|^2 the product of the per-axis tables;
// every operation rounded separately in the order written.
__device__ __forceinline__ double deconv_data64(const Job& J, double G, int x, int y, int z, int l, int c)
{
    const double d = __dsub_rn(J.mu64[c], J.mu64[l]);
    const double t = __dmul_rn(d, G);
    double np = __dmul_rn(J.psf_n[x], J.psf_n[J.W + y]);
    if (J.ndim == 3) np = __dmul_rn(np, J.psf_n[J.W + J.H + z]);
    const double q = __dmul_rn(__dmul_rn(d, d), np);
    return __dsub_rn(q, __dadd_rn(t, t));
}

// ---------------------------------------------------------------------------
// FP64 evaluation of the energy difference in the order of its definition: every product and
// sum rounded separately (no fused multiply-add), so that it equals the FP64 reference's value
// bit for bit.
__device__ __forceinline__ double image64(const Job& J, long long i)
{
    if (J.dtype == SEG_F32) return (double)((const float*)J.I)[i];
    return (double)((const unsigned short*)J.I)[i];
}

// Natural logarithm by the atanh series after reduction to [sqrt(1/2), sqrt(2)):
// ln x = e ln 2 + 2 (y + y^3/3 + ... + y^23/23), y = (m - 1)/(m + 1), every operation an IEEE
// double operation in a fixed order (the FP64 reference evaluates the same series the same way).
__device__ __forceinline__ double log_series(double x)
{
    int e = 0;
    double m = frexp(x, &e);
    if (m < 0.70710678118654752440) { m = __dmul_rn(2.0, m); e = e - 1; }
    const double y = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
    const double y2 = __dmul_rn(y, y);
    double s = 1.0 / 23.0;
    s = __dadd_rn(1.0 / 21.0, __dmul_rn(y2, s));
    s = __dadd_rn(1.0 / 19.0, __dmul_rn(y2, s));
    s = __dadd_rn(1.0 / 17.0, __dmul_rn(y2, s));
    s = __dadd_rn(1.0 / 15.0, __dmul_rn(y2, s));
    s = __dadd_rn(1.0 / 13.0, __dmul_rn(y2, s));
    s = __dadd_rn(1.0 / 11.0, __dmul_rn(y2, s));
    s = __dadd_rn(1.0 / 9.0, __dmul_rn(y2, s));
    s = __dadd_rn(1.0 / 7.0, __dmul_rn(y2, s));
    s = __dadd_rn(1.0 / 5.0, __dmul_rn(y2, s));
    s = __dadd_rn(1.0 / 3.0, __dmul_rn(y2, s));
    s = __dadd_rn(1.0, __dmul_rn(y2, s));
    return __dadd_rn(__dmul_rn((double)e, 0.69314718055994530942), __dmul_rn(2.0, __dmul_rn(y, s)));
}

// Poisson negative log-likelihood of v under the (floored) mean mu, the log(v!) term dropped
__device__ __forceinline__ double poisson_f64(double v, double mu, double floor)
{
    const double m = mu > floor ? mu : floor;
    return __dsub_rn(m, __dmul_rn(v, log_series(m)));
}

// Piecewise-constant data term (Eq. 11, the exact single-pixel change of the squared deviations
// from the region means): n_c/(n_c+1) (v - mu_c)^2 - n_l/(n_l-1) (v - mu_l)^2, where the second
// weight is 0 for n_l <= 1 (so the term is +0, as the definition's 0)
__device__ __forceinline__ double data_pc64(const Job& J, double v, int l, int c)
{
    const double a = __dsub_rn(v, __ldg(J.mu64 + c));
    const double b = __dsub_rn(v, __ldg(J.mu64 + l));
    const double t1 = __dmul_rn(__ldg(J.wp64 + c), __dmul_rn(a, a));
    const double t2 = __dmul_rn(__ldg(J.wm64 + l), __dmul_rn(b, b));
    return __dsub_rn(t1, t2);
}

// Piecewise-smooth data terms from the FP64 sums sc, sl of the c and l parts of the ball and
// their pixel counts: (v - mu_c)^2 - (v - mu_l)^2, or with Poisson noise f(v, mu_c) - f(v, mu_l)
__device__ __forceinline__ double data_ps64(const Job& J, double v, double sc, long long cc, double sl, long long cl)
{
    const double muc = __ddiv_rn(sc, (double)cc), mul = __ddiv_rn(sl, (double)cl);
    if (J.model == SEG_PS_POISSON)
        return __dsub_rn(poisson_f64(v, muc, J.mu_floor64), poisson_f64(v, mul, J.mu_floor64));
    const double a = __dsub_rn(v, muc);
    const double b = __dsub_rn(v, mul);
    return __dsub_rn(__dmul_rn(a, a), __dmul_rn(b, b));
}

// data term + lambda * (change of unlike neighbour pairs)
__device__ __forceinline__ double with_length64(const Job& J, double data, int dP)
{
    return __dadd_rn(data, __dmul_rn(J.lambda64, (double)dP));
}

// Keep the FP64 energy difference e of particle o (for the FP64 recompute) and as a pair of
// floats, hi = fl(e) and lo = fl(e - hi): |hi + lo - e| <= 2^-48 |e| + 2^-149. The bound stored
// with hi is that of its one rounding, 2^-24 |hi| (+ 2^-149 below the normal range), widened by
// 2^-50 |hi|.
__device__ __forceinline__ void store_dE(const Job& J, unsigned o, double e)
{
    J.p_dE64[o] = e;
    const float hi = __double2float_rn(e);
    J.p_dE[o] = hi;
    J.p_dEl[o] = __double2float_rn(__dsub_rn(e, (double)hi));
    J.p_eE[o] = 5.96047e-8f * fabsf(hi) + 1.4e-45f;
}

// Compensated sum of exact products (Ogita, Rump and Oishi, "Accurate sum and dot product",
// SIAM J. Sci. Comput. 2005: algorithm Dot2, the product's error term taken by a fused
// multiply-add, here with both factors given as float pairs): after n terms s + t equals the sum
// of (Kh + Kl)(dh + dl) within u |sum| + (gamma_n^2 + 2^-46) sum |K dE|, u = 2^-24.
struct DotAcc {
    float s = 0.0f, t = 0.0f;
    __device__ __forceinline__ float add(float Kh, float Kl, float dh, float dl)
    {
        const float p = __fmul_rn(Kh, dh);
        float e = __fmaf_rn(Kh, dh, -p);          // the product's rounding error, exactly
        e = __fmaf_rn(Kh, dl, e);
        e = __fmaf_rn(Kl, dh, e);
        const float x = __fadd_rn(s, p);          // two-sum: x + err = s + p exactly
        const float z = __fsub_rn(x, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(x, z)), __fsub_rn(p, z));
        s = x;
        t = __fadd_rn(t, __fadd_rn(err, e));
        return p;
    }
};

// (s + t) / n as a pair (q, ql): q the rounded quotient of s, whose remainder s - q n is exact
__device__ __forceinline__ void pair_div(float s, float t, int n, float& q, float& ql)
{
    const float fn = (float)n;
    q = __fdiv_rn(s, fn);
    ql = __fdiv_rn(__fadd_rn(__fmaf_rn(-q, fn, s), t), fn);
}

// (a + al) - (b + bl) rounded to one float, through a two-sum of the leading parts
__device__ __forceinline__ float pair_sub(float a, float al, float b, float bl)
{
    const float x = __fsub_rn(a, b);
    const float z = __fsub_rn(x, a);
    const float err = __fsub_rn(__fsub_rn(a, __fsub_rn(x, z)), __fadd_rn(b, z));
    return __fadd_rn(x, __fadd_rn(err, __fsub_rn(al, bl)));
}

// Bound on |g - g_fp64| of a gradient from the compensated Eq. 6 sums of nA and nB terms
// (partial sums of parallel lanes joined count as terms): the final rounding to float, the
// second-order terms of the compensated sums (gamma_2n^2), the float pairs of K and dE with the
// products' rounded cross terms (below 6e-14 of |K dE|), the pair divisions and difference
// (u^2), and the FP64 reference's own rounding (1e-12), each relative to a set's sum of |K dE|
// over its size (TA, TB).
__device__ __forceinline__ float pair_bound(float g, int nA, float TA, int nB, float TB)
{
    auto g2 = [](int n) {
        const float t = (float)(2 * n) * 5.9604645e-8f;
        const float gm = t / (1.0f - t);
        return gm * gm;
    };
    const float cA = nA ? g2(nA) + 6e-14f + 1e-12f : 0.0f;
    const float cB = nB ? g2(nB) + 6e-14f + 1e-12f : 0.0f;
    return (5.9604645e-8f * fabsf(g) + (cA * TA + cB * TB) * 1.01f) * 1.001f + 1.4e-45f;
}

// What seg_init needs to know about its inputs, found on the device in one pass.
struct InputScan {
    int lab_min, lab_max;          // smallest and largest label
    int slot_lo, slot_hi;          // float32: exponent slots of the non-zero values (slot_hi < slot_lo: none)
    unsigned maxabs;               // float32: bits of the largest |I|; uint16: the largest value
    int bad;                       // float32: a NaN or an infinity
    int neg;                       // float32: a value below zero
    unsigned long long particles;  // particles of the initial labels (pixel, neighbouring label) pairs
    unsigned long long pairs;      // adjacent pixel pairs with different labels (|Gamma|)
};

// Programmatic dependent launch: a stage kernel launched with programmatic stream
// serialization may be scheduled while its predecessor finishes. Every stage kernel starts
// with pdl_enter(): it waits until the predecessor grid has completed and its memory is
// visible (a no-op when the kernel was launched without the attribute), then lets its own
// successor be scheduled.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launches of the iteration's stages use programmatic serialization while this is set
// (the stepper sets it while enqueueing an iteration without per-stage events).
extern thread_local bool g_pdl;

// Kernel launch accounting (seg_kernel_launches): every launch site calls count_launch().
// A launch made while a graph is being captured counts towards that graph; each replay of
// the graph then counts its kernels.
void count_launch();

template <typename... KArgs, typename... Args>
inline cudaError_t launch_stage(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = g_pdl ? 1 : 0;
    count_launch();
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// Launch wrappers (one iteration's stages); defined in the kernel translation units.
cudaError_t launch_extract(const Group& g, int ndim, size_t smem, cudaStream_t s);
cudaError_t launch_sobolev(const Group& g, BatchCtl* bc, int ndim, size_t smem, cudaStream_t s);
cudaError_t launch_global_lut(const Job* jobs, int njobs, int sms, cudaStream_t s);
cudaError_t launch_sobolev_global(const Group& g, int ndim, cudaStream_t s);
cudaError_t launch_fixup(const Job* jobs, int njobs, int sms, cudaStream_t s);
cudaError_t launch_gather_counters(const Job* jobs, int njobs, Counters* out, cudaStream_t s);
cudaError_t configure_kernels(size_t smem_x2, size_t smem_x3, size_t smem_s2, size_t smem_s3);
cudaError_t launch_select(const Group& g, BatchCtl* bc, cudaStream_t s);
cudaError_t launch_lists(const Job* jobs, int njobs, int sms, cudaStream_t s);
cudaError_t launch_rounds(const Job* jobs, int njobs, BatchCtl* bc, int grid, int block, cudaStream_t s);
cudaError_t launch_moves(const Job* jobs, int njobs, BatchCtl* bc, int sms, cudaStream_t s);
cudaError_t launch_finish(const Job* jobs, int njobs, BatchCtl* bc, int sms, cudaStream_t s);
cudaError_t launch_stats_init(const Job* jobs, int j, long long npix, cudaStream_t s, bool after_split = false);
cudaError_t launch_stats_zero_after_split(const Job* jobs, int j, const Job& h, cudaStream_t s);
cudaError_t launch_relabel(const Job* jobs, int j, const Job& h, int sms, cudaStream_t s);
cudaError_t launch_curvature(const Job* jobs, int j, int sms, cudaStream_t s);
cudaError_t launch_fuse(const Job* jobs, int j, int sms, cudaStream_t s);
cudaError_t launch_deconv(const Job* jobs, int j, const Job& h, int sms, cudaStream_t s);
cudaError_t launch_psf_norms(const Job* job, const Job& h, cudaStream_t s);
cudaError_t launch_scan_inputs(const void* I, int dtype, const int* L, int ndim, int D, int H, int W, InputScan* out,
                               cudaStream_t s);
cudaError_t launch_stats_finalize(const Job* jobs, int njobs, cudaStream_t s);
cudaError_t topology_tables_init();
void topology_for_job(Job& h);   // the job's pointers to the topology tables (after topology_tables_init)
cudaError_t commit_occupancy(int block, int* blocks_per_sm);
size_t extract_smem_bytes(const Job& h);
size_t sobolev_smem_bytes(const Job& h);
cudaError_t launch_debug_simple(const unsigned* masks, int ndim, int n, unsigned char* out, cudaStream_t s);

}  // namespace segk
