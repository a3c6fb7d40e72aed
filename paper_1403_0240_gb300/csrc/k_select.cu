// Decision kernels of one iteration: the neighbour lists of the candidates with the order
// certificates of their float32 keys, the FP64 recompute of uncertified keys, the candidate
// selection of the E = |Gamma| mode (the other modes select inside the interaction kernel), and
// the commit (ranked conflict-free selection, label update, exact region statistics,
// oscillation fallback).
#include <algorithm>

#include "seg_internal.cuh"

namespace segk {

// ---------------------------------------------------------------------------
// Simple points by topological numbers (Bertrand & Malandain): bitmask flood fills
// over the 8 (2D) or 26 (3D) neighbour positions, row-major order without the centre.
struct TopoTables {
    unsigned adjF[2][26];   // foreground adjacency: 4 (2D) | 6 (3D)
    unsigned adjB[2][26];   // background adjacency: 8 (2D) | 26 (3D)
    unsigned nF[2];         // neighbourhood of the foreground count: N8* (2D) | N18* (3D)
    unsigned touch[2];      // 4- | 6-neighbours of the centre
    unsigned all[2];
    int npos[2];
};
__constant__ TopoTables c_topo;
// Simple-point decisions tabulated for every neighbourhood mask: 2^8 (2D) and 2^26 (3D) bits,
// computed once per process on the device from simple_mask() below.
__constant__ const unsigned* c_simple[2];
// host copies of the same, for the job descriptors
static const unsigned* g_simple[2];
static const unsigned* g_topo_adjF[2];
static unsigned g_topo_touch[2], g_topo_nF[2];

__device__ __forceinline__ bool simple_mask(unsigned X, int d);

__global__ void k_simple_table(unsigned* out, int d, unsigned nwords)
{
    const unsigned w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwords) return;
    unsigned bits = 0;
    for (unsigned b = 0; b < 32; b++)
        if (simple_mask(w * 32u + b, d)) bits |= 1u << b;
    out[w] = bits;
}

cudaError_t simple_tables_init()
{
    unsigned* t2 = nullptr;
    unsigned* t3 = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&t2, 8 * sizeof(unsigned))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&t3, (1u << 21) * sizeof(unsigned))) != cudaSuccess) return e;
    count_launch();
    k_simple_table<<<1, 32>>>(t2, 0, 8);
    count_launch();
    k_simple_table<<<(1u << 21) / 256, 256>>>(t3, 1, 1u << 21);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return e;
    const unsigned* ptrs[2] = {t2, t3};
    g_simple[0] = t2;
    g_simple[1] = t3;
    return cudaMemcpyToSymbol(c_simple, ptrs, sizeof ptrs);
}

cudaError_t topology_tables_init()
{
    TopoTables t;
    memset(&t, 0, sizeof t);
    for (int d = 0; d < 2; d++) {
        int pos[26][3];
        int n = 0;
        for (int dz = (d ? -1 : 0); dz <= (d ? 1 : 0); dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    if (!dz && !dy && !dx) continue;
                    pos[n][0] = dz; pos[n][1] = dy; pos[n][2] = dx;
                    n++;
                }
        t.npos[d] = n;
        t.all[d] = n == 32 ? 0xffffffffu : ((1u << n) - 1u);
        for (int a = 0; a < n; a++) {
            int l1 = abs(pos[a][0]) + abs(pos[a][1]) + abs(pos[a][2]);
            if (l1 == 1) t.touch[d] |= 1u << a;
            if (d == 0 || l1 <= 2) t.nF[d] |= 1u << a;
            for (int b = 0; b < n; b++) {
                if (a == b) continue;
                int dz = abs(pos[a][0] - pos[b][0]), dy = abs(pos[a][1] - pos[b][1]), dx = abs(pos[a][2] - pos[b][2]);
                int m1 = dz + dy + dx, mi = max(dz, max(dy, dx));
                if (m1 == 1) t.adjF[d][a] |= 1u << b;
                if (mi == 1) t.adjB[d][a] |= 1u << b;
            }
        }
    }
    cudaError_t e = cudaMemcpyToSymbol(c_topo, &t, sizeof t);
    if (e != cudaSuccess) return e;
    // the jobs reach the foreground adjacency through a pointer (the selection runs in more
    // than one translation unit)
    unsigned* adj = nullptr;
    if ((e = cudaMalloc(&adj, sizeof t.adjF)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(adj, t.adjF, sizeof t.adjF, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    for (int d = 0; d < 2; d++) {
        g_topo_adjF[d] = adj + 26 * d;
        g_topo_touch[d] = t.touch[d];
        g_topo_nF[d] = t.nF[d];
    }
    return simple_tables_init();
}

void topology_for_job(Job& h)
{
    const int d = h.ndim == 3 ? 1 : 0;
    h.simple_tab = g_simple[d];
    h.topo_adjF = g_topo_adjF[d];
    h.topo_touch = g_topo_touch[d];
    h.topo_nF = g_topo_nF[d];
}

__device__ __forceinline__ bool simple_mask(unsigned X, int d)
{
    const unsigned* aF = c_topo.adjF[d];
    const unsigned* aB = c_topo.adjB[d];
    if (components(X & c_topo.nF[d], aF, c_topo.touch[d]) != 1) return false;
    return components(~X & c_topo.all[d], aB, 0u) == 1;
}

__device__ __forceinline__ bool simple_table(unsigned X, int d)
{
    return (__ldg(c_simple[d] + (X >> 5)) >> (X & 31u)) & 1u;
}

// the tabulated decision, as the selection uses it
__global__ void k_debug_simple(const unsigned* masks, int ndim, int n, unsigned char* out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = simple_table(masks[i], ndim == 3 ? 1 : 0) ? 1 : 0;
}

cudaError_t launch_debug_simple(const unsigned* masks, int ndim, int n, unsigned char* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    count_launch();
    k_debug_simple<<<(n + 255) / 256, 256, 0, s>>>(masks, ndim, n, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ bool job_idle(const Counters* c)
{
    return ld_volatile(&c->skip) != 0 || ld_volatile(&c->need) != 0;
}

__device__ __forceinline__ void coords(const Job& J, unsigned gi, int& x, int& y, int& z)
{
    pix_coords(J, gi, x, y, z);
}

// Certification. A decision takes the float gradient g in place of the FP64 key wherever the
// bound eg (|g - key| <= eg) makes that safe:
//  - candidacy needs key < 0. The best particle of a pixel becomes a candidate when g < eg
//    (possibly negative); when moreover |g| <= eg its sign is uncertain and it is queued for the
//    FP64 recompute, after which a key >= 0 drops it (it enters the rounds rejected);
//  - the rounds need the order of neighbouring candidates. Two candidates whose gradients lie
//    within the sum of their bounds are both queued (each finds the other while listing its
//    neighbours), and their lists are rebuilt once every queued key is exact. Any other pair
//    keeps its order: an exact key stays within its bound of the float it replaces.
// In the Sobolev modes the particles of one pixel share their label, hence both sets of Eq. 6
// and the gradient, so the best particle of a pixel is the one of smallest c, without a
// certificate; in L2 mode the key is the FP64 energy difference itself, exact (bound 0).
//
// The comparisons run in float32: with d = fl(gp - gq) and s = fl(ep + eq), each within one
// rounding, |gp - gq| <= ep + eq implies |d| <= s (1 + 2^-22), so a pair is queued whenever
// the exact test could fail.
__device__ __forceinline__ bool order_uncertain(float gp, float ep, float gq, float eq)
{
    return fabsf(__fsub_rn(gp, gq)) <= __fmul_rn(__fadd_rn(ep, eq), 1.00000024f);
}


// ---------------------------------------------------------------------------
// FP64 recompute in the order of the definition: every product and sum rounded separately (no
// fused multiply-add), neighbours in ascending particle key. The partners' FP64 energy
// differences are those extraction evaluated (the FP64 reference's values, bit for bit).

// ---------------------------------------------------------------------------
// Batches: per-job counts (flagged particles, candidates, labels) turned into one
// flattened index space by a block-parallel exclusive prefix in shared memory; an index is
// mapped back to its job by binary search. Idle jobs count zero.
constexpr int kMaxBatchJobs = 2048;
enum JobCount { kCountFlag = 0, kCountCand = 1, kCountLabels = 2 };

__device__ __forceinline__ unsigned job_count(const Job& J, int kind)
{
    if (kind == kCountLabels) return (unsigned)J.M;
    if (ld_volatile(&J.ctr->skip) || ld_volatile(&J.ctr->need)) return 0;
    return ld_volatile(kind == kCountFlag ? &J.ctr->n_flag : &J.ctr->n_cand);
}

// s_pref[0..njobs]: exclusive prefix; returns the total (all threads)
__device__ unsigned block_job_prefix(const Job* jobs, int njobs, int kind, unsigned* s_pref, unsigned* s_tmp)
{
    const int nt = blockDim.x;
    const int chunk = (njobs + nt - 1) / nt;
    const int j0 = min((int)threadIdx.x * chunk, njobs), j1 = min(j0 + chunk, njobs);
    unsigned sum = 0;
    for (int j = j0; j < j1; j++) sum += job_count(jobs[j], kind);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_tmp[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned a = lane < (nt >> 5) ? s_tmp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, a, o);
            if (lane >= o) a += y;
        }
        if (lane < (nt >> 5)) s_tmp[lane] = a;
    }
    __syncthreads();
    unsigned run = (w > 0 ? s_tmp[w - 1] : 0u) + x - sum;
    for (int j = j0; j < j1; j++) {
        s_pref[j] = run;
        run += job_count(jobs[j], kind);
    }
    const unsigned total = s_tmp[(nt >> 5) - 1];
    if (threadIdx.x == 0) s_pref[njobs] = total;
    __syncthreads();
    return total;
}

// the job holding flattened index i (the last job whose prefix is <= i)
__device__ __forceinline__ int job_of(const unsigned* s_pref, int njobs, unsigned i)
{
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (s_pref[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

constexpr int kFixThreads = 128;             // one block per queued particle
constexpr int kFixTerms = 6 * kFixThreads;     // at most 6 particles per pixel

// Block-wide exclusive prefix of v (kFixThreads threads); the total goes to *total.
__device__ __forceinline__ int block_excl(int v, int* s_w, int* total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    int before = 0, all = 0;
    for (int k = 0; k < kFixThreads / 32; k++) {
        if (k < w) before += s_w[k];
        all += s_w[k];
    }
    *total = all;
    return before + x - v;
}


// The FP64 key of queued candidate slot s (particle p) replaces its float one: exact from now
// on (bound 0); a key >= 0 drops the candidate, which then enters the rounds rejected.
__device__ __forceinline__ void fix_apply(const Job& J, unsigned s, unsigned p, double key)
{
    J.p_key[p] = key;
    J.c_key[s] = ordered_key(key);
    J.c_ge[s] = make_float2(0.0f, 0.0f);
    if (!(key < 0.0)) {
        J.c_state[s] = kRejected;
        J.p_flags[p] &= (unsigned char)~(kFlagCand | kFlagSplit);
        atomicAdd(&J.ctr->n_void, 1u);
    }
}

// E = |Gamma| mode: the FP64 key of particle (gi, lp) over every particle with d^2 < g_lim, in
// ascending key order (the pixels of the support's bounding box in row-major order, particles
// of a pixel in order); one warp walks the box, t_w / a_w hold 192 terms. Lane 0's value counts.
__device__ double fix_global_warp(const Job& J, unsigned gi, int lp, unsigned tag, unsigned np, double* t_w,
                                  unsigned char* a_w)
{
    const int lane = threadIdx.x & 31;
    int x, y, z;
    coords(J, gi, x, y, z);
    const long long lim = J.ctr->g_lim;
    // largest r with r^2 < lim, from the square root corrected by one step
    long long r = (long long)sqrt((double)(lim > 0 ? lim - 1 : 0));
    while (r > 0 && r * r >= lim) r--;
    while ((r + 1) * (r + 1) < lim) r++;
    const long long x0 = max(0LL, x - r), x1 = min((long long)J.W - 1, x + r);
    const long long y0 = max(0LL, y - r), y1 = min((long long)J.H - 1, y + r);
    const long long z0 = J.ndim == 3 ? max(0LL, z - r) : 0, z1 = J.ndim == 3 ? min((long long)J.D - 1, z + r) : 0;
    const long long bw = x1 - x0 + 1, bh = y1 - y0 + 1, nbox = bw * bh * (z1 - z0 + 1);
    double As = 0.0, Bs = 0.0;
    long long nA = 0, nB = 0;
    for (long long base0 = 0; base0 < nbox; base0 += 32) {
        const long long i = base0 + lane;
        unsigned yi = 0, q0 = 0;
        long long d2 = 0;
        bool ok = false;
        if (i < nbox) {
            const long long xx = x0 + i % bw, yy = y0 + (i / bw) % bh, zz = z0 + i / (bw * bh);
            d2 = (xx - x) * (xx - x) + (yy - y) * (yy - y) + (zz - z) * (zz - z);
            if (d2 < lim) {
                yi = (unsigned)((zz * J.H + yy) * J.W + xx);
                const unsigned long long e = J.pmap[yi];
                ok = (unsigned)(e >> 32) == tag;
                q0 = (unsigned)e;
            }
        }
        int nt = 0;
        if (ok)
            for (unsigned q = q0; q < np && J.p_idx[q] == yi; q++)
                nt += (J.p_l[q] == lp || J.p_c[q] == lp) ? 1 : 0;
        if (!__any_sync(0xffffffffu, nt > 0)) continue;
        int incl = nt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        int pos = incl - nt;
        if (ok && nt) {
            const double K = J.gK64[d2];
            for (unsigned q = q0; q < np && J.p_idx[q] == yi; q++) {
                const int lq = J.p_l[q], cq = J.p_c[q];
                if (lq != lp && cq != lp) continue;
                t_w[pos] = __dmul_rn(K, J.p_dE64[q]);
                a_w[pos] = lq == lp ? 1 : 0;
                pos++;
            }
        }
        __syncwarp();
        if (lane == 0) {
            for (int u = 0; u < tot; u++) {
                if (a_w[u]) { As = __dadd_rn(As, t_w[u]); nA++; }
                else { Bs = __dadd_rn(Bs, t_w[u]); nB++; }
            }
        }
        __syncwarp();
    }
    const double A = nA ? __ddiv_rn(As, (double)nA) : 0.0;
    const double B = nB ? __ddiv_rn(Bs, (double)nB) : 0.0;
    return __dsub_rn(A, B);
}

// The same recompute with one queued particle per warp (many queued particles): lanes take
// the interaction offsets 32 at a time, lane 0 sums each group's terms in ascending key order.
__device__ void fixup_warps(const Job* jobs, int njobs, unsigned total, const unsigned* s_pref, double* s_t,
                            unsigned char* s_a)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int kWarps = kFixThreads / 32, kWarpTerms = kFixTerms / kWarps;
    double* t_w = s_t + w * kWarpTerms;
    unsigned char* a_w = s_a + w * kWarpTerms;
    for (unsigned fi = blockIdx.x * kWarps + w; fi < total; fi += gridDim.x * kWarps) {
        const int j = job_of(s_pref, njobs, fi);
        const Job& J = jobs[j];
        Counters* ctr = J.ctr;
        const unsigned tag = ld_volatile(&ctr->iter_tag);
        const unsigned np = ld_volatile(&ctr->n_particles);
        const int mode = ld_volatile(&ctr->mode);
        const unsigned sl = J.flag_list[fi - s_pref[j]];
        const unsigned p = (unsigned)J.c_best[sl];
        const unsigned gi = J.p_idx[p];
        const int lp = J.p_l[p];
        if (mode == SEG_L2) {
            if (lane == 0) fix_apply(J, sl, p, J.p_dE64[p]);
            continue;
        }
        if (mode == SEG_SOBOLEV_GLOBAL) {
            const double gval = fix_global_warp(J, gi, lp, tag, np, t_w, a_w);
            if (lane == 0) fix_apply(J, sl, p, gval);
            continue;
        }
        int x, y, z;
        coords(J, gi, x, y, z);
        double As = 0.0, Bs = 0.0;
        long long nA = 0, nB = 0;
        for (int base = 0; base < J.nb_n; base += 32) {
            const int u = base + lane;
            double tv[6];
            unsigned char ta[6];
            int nt = 0;
            if (u < J.nb_n) {
                const int4 d = J.nb_off[u];
                const int xx = x + d.z, yy = y + d.y, zz = z + d.x;
                if (xx >= 0 && xx < J.W && yy >= 0 && yy < J.H && zz >= 0 && zz < J.D) {
                    const unsigned yi = (unsigned)(((long long)zz * J.H + yy) * J.W + xx);
                    const unsigned long long e = J.pmap[yi];
                    if ((unsigned)(e >> 32) == tag) {
                        const double K = J.klut64[d.w];
                        for (unsigned q = (unsigned)e; q < np && J.p_idx[q] == yi && nt < 6; q++) {
                            const int lq = J.p_l[q], cq = J.p_c[q];
                            if (lq == lp || cq == lp) {
                                tv[nt] = __dmul_rn(K, J.p_dE64[q]);
                                ta[nt] = lq == lp ? 1 : 0;
                                nt++;
                            }
                        }
                    }
                }
            }
            int incl = nt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const int tot = __shfl_sync(0xffffffffu, incl, 31);
            for (int i = 0; i < nt; i++) {
                t_w[incl - nt + i] = tv[i];
                a_w[incl - nt + i] = ta[i];
            }
            __syncwarp();
            if (lane == 0) {
                for (int i = 0; i < tot; i++) {
                    if (a_w[i]) { As = __dadd_rn(As, t_w[i]); nA++; }
                    else { Bs = __dadd_rn(Bs, t_w[i]); nB++; }
                }
            }
            __syncwarp();
        }
        if (lane == 0) {
            const double A = nA ? __ddiv_rn(As, (double)nA) : 0.0;
            const double B = nB ? __ddiv_rn(Bs, (double)nB) : 0.0;
            fix_apply(J, sl, p, __dsub_rn(A, B));
        }
    }
}

__global__ void k_gather_counters(const Job* jobs, int njobs, Counters* out)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < njobs) out[j] = *jobs[j].ctr;
}

cudaError_t launch_gather_counters(const Job* jobs, int njobs, Counters* out, cudaStream_t s)
{
    if (njobs <= 0) return cudaSuccess;
    count_launch();
    k_gather_counters<<<(njobs + 127) / 128, 128, 0, s>>>(jobs, njobs, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Candidates of the E = |Gamma| mode (after the all-pairs interaction kernel): per pixel the
// particle with the smallest (key, c); a candidate when its key could be negative and its move
// passes the topology tests on the masks extraction wrote. The other modes select the same way
// inside the interaction kernel.
__global__ void __launch_bounds__(256) k_select(Group g, BatchCtl* bc)
{
    pdl_enter();
    const unsigned t = blockIdx.x;
    if (t == 0 && threadIdx.x == 0) {
        bc->err = 0;
        bc->rounds_done = 0;
    }
    const int gj = group_job_of_tile(g, t);
    const Job& J = g.jobs[g.job_ids[gj]];
    const unsigned k = t - g.tile_prefix[gj];
    Counters* ctr = J.ctr;
    if (job_idle(ctr) || ld_volatile(&ctr->mode) != SEG_SOBOLEV_GLOBAL) return;   // the others: k_sobolev
    const unsigned pstart = J.tile_start[k], pend = pstart + J.tile_count[k];
    const bool exact_keys = false;
    __shared__ unsigned s_scan[32], s_slot0;
    // the tile's candidates take one contiguous range of slots per pass (a block scan and one
    // counter update), so that candidate indices follow the tiles: the selection rounds give each
    // block a contiguous range of indices and so a compact region of the image
    for (unsigned p0 = pstart; p0 < pend; p0 += blockDim.x) {          // uniform over the block
        const unsigned p = p0 + threadIdx.x;
        unsigned best = 0, gi = 0;
        double bk = 0.0;
        float bg = 0.0f, be = 0.0f;
        int bc_ = 0, adm = 0;
        const bool first = p < pend && (p == pstart || J.p_idx[p - 1] != J.p_idx[p]);
        if (first) {
            gi = J.p_idx[p];
            best = p;
            bk = J.p_key[p];
            bc_ = J.p_c[p];
            for (unsigned q = p + 1; q < pend && J.p_idx[q] == gi; q++) {
                double kq = J.p_key[q];
                int cq = J.p_c[q];
                if (kq < bk || (kq == bk && cq < bc_)) { best = q; bk = kq; bc_ = cq; }
            }
            // the candidate's float gradient and bound (exact keys: bound 0)
            bg = exact_keys ? 0.0f : J.p_g[best];
            be = exact_keys ? 0.0f : J.p_eg[best];
            const bool maybe_neg = exact_keys ? bk < 0.0 : bg < be;
            adm = maybe_neg ? admissible(J, J.p_l[best], bc_, J.p_nbm[best]) : 0;
        }
        unsigned n_adm;
        const unsigned rank = block_excl_scan(adm ? 1u : 0u, s_scan, n_adm);
        if (threadIdx.x == 0) s_slot0 = n_adm ? atomicAdd(&ctr->n_cand, n_adm) : 0u;
        __syncthreads();
        if (first) {
            int slot = -1;
            if (adm) {
                slot = (int)(s_slot0 + rank);
                J.c_best[slot] = (int)best;
                J.c_key[slot] = ordered_key(bk);
                J.c_pix[slot] = gi;
                J.c_ge[slot] = make_float2(bg, be);
                J.p_flags[best] |= adm == 2 ? (kFlagCand | kFlagSplit) : kFlagCand;
                if (!exact_keys && fabsf(bg) <= be) queue_fixup(J, (unsigned)slot, best);   // sign uncertain
            }
            J.pix_cand[p] = slot;
        }
        __syncthreads();                       // s_scan and s_slot0 are reused by the next pass
    }
}

cudaError_t launch_select(const Group& g, BatchCtl* bc, cudaStream_t s)
{
    if (g.total_tiles == 0) return cudaSuccess;
    return launch_stage(k_select, g.total_tiles, 256, 0, s, g, bc);
}

// ---------------------------------------------------------------------------
// Exact region statistics.
__device__ __forceinline__ void f32_parts(float f, int& slot, long long& sm, unsigned long long& m2lo,
                                          unsigned long long& m2hi)
{
    unsigned bits = __float_as_uint(f);
    int eb = (int)((bits >> 23) & 0xffu);
    unsigned long long m = bits & 0x7fffffu;
    if (eb == 0) eb = 1; else m |= 0x800000ull;
    slot = eb;
    sm = (bits >> 31) ? -(long long)m : (long long)m;
    unsigned long long sq = m * m;
    m2lo = sq & 0xffffffull;
    m2hi = sq >> 24;
}

__device__ __forceinline__ void atomic_add_ll(long long* a, long long v)
{
    atomicAdd((unsigned long long*)a, (unsigned long long)v);
}

// Compensated FP32 sums (SEG_STATS_KAHAN32): add a then b to the (sum, compensation) float
// pair at p, each by one Neumaier step (Neumaier 1974: the rounding error of every addition is
// accumulated in the compensation), the pair updated atomically by compare-and-swap. Retries
// happen only when another thread's update landed; they are bounded all the same.
__device__ __forceinline__ unsigned long long neumaier2(unsigned long long pair, float a, float b)
{
    float s = __uint_as_float((unsigned)pair), c = __uint_as_float((unsigned)(pair >> 32));
    for (int k = 0; k < 2; k++) {
        const float v = k ? b : a;
        const float t = __fadd_rn(s, v);
        const float e = fabsf(s) >= fabsf(v) ? __fadd_rn(__fsub_rn(s, t), v) : __fadd_rn(__fsub_rn(v, t), s);
        c = __fadd_rn(c, e);
        s = t;
    }
    return (unsigned long long)__float_as_uint(s) | ((unsigned long long)__float_as_uint(c) << 32);
}

__device__ void kahan_add(unsigned long long* p, float a, float b, Counters* ctr)
{
    unsigned long long old = ld_volatile(p);
    for (unsigned tries = 0; tries < kSpinLimit; tries++) {
        const unsigned long long got = atomicCAS(p, old, neumaier2(old, a, b));
        if (got == old) return;
        old = got;
    }
    atomicExch(&ctr->error, SEG_ETIMEOUT);
}

// the value and its exact square split into float head + tail (two-product by fused multiply-add)
__device__ __forceinline__ void value_parts(const Job& J, long long i, float& v, float& q, float& qe)
{
    v = J.dtype == SEG_U16 ? (float)((const unsigned short*)J.I)[i] : ((const float*)J.I)[i];
    q = __fmul_rn(v, v);
    qe = __fmaf_rn(v, v, -q);
}

// one pixel of value at index i joins (sign +1) or leaves (sign -1) label m
__device__ __forceinline__ void stats_move(const Job& J, long long i, int m, int sign)
{
    atomic_add_ll(J.st_n + m, sign);
    if (J.stats_mode == SEG_STATS_F64) {
        const double v = J.dtype == SEG_U16 ? (double)((const unsigned short*)J.I)[i] : (double)((const float*)J.I)[i];
        atomicAdd(J.sf64 + m, sign * v);
        atomicAdd(J.sf64 + J.M + m, sign * (v * v));       // exact: at most 48 significant bits
        return;
    }
    if (J.stats_mode == SEG_STATS_KAHAN32) {
        float v, q, qe;
        value_parts(J, i, v, q, qe);
        kahan_add(J.sk32 + m, sign * v, 0.0f, J.ctr);
        kahan_add(J.sk32 + J.M + m, sign * q, sign * qe, J.ctr);
        return;
    }
    if (J.dtype == SEG_U16) {
        long long v = ((const unsigned short*)J.I)[i];
        atomic_add_ll(J.st_S + m, sign * v);
        atomic_add_ll(J.st_Q + m, sign * v * v);
    } else {
        int slot;
        long long sm;
        unsigned long long lo, hi;
        f32_parts(((const float*)J.I)[i], slot, sm, lo, hi);
        if (sm == 0) return;
        int k = slot - J.slot_lo;
        atomic_add_ll(J.st_S + (long long)m * J.nS + k, sign * sm);
        atomic_add_ll(J.st_Q + (long long)m * J.nQ + 2 * k, sign * (long long)lo);
        atomic_add_ll(J.st_Q + (long long)m * J.nQ + 2 * k + 24, sign * (long long)hi);
    }
}

// Round sum_k bins[k] * 2^(k + e0) (exactly) to the nearest double, ties to even.
constexpr int kLimbs = 24;
__device__ double round_bins(const long long* bins, int nb, int e0)
{
    long long lim[kLimbs];
    const int nl = min(kLimbs, (nb + 63) / 32 + 3);   // bins span nb bits plus 64 of each value
    for (int i = 0; i < kLimbs; i++) lim[i] = 0;
    for (int k = 0; k < nb; k++) {
        long long b = bins[k];
        if (!b) continue;
        int j = k >> 5, r = k & 31;
        unsigned long long lo = (unsigned long long)(b & 0xffffffffLL) << r;
        lim[j] += (long long)(lo & 0xffffffffull);
        lim[j + 1] += (long long)(lo >> 32);
        long long hs = (b >> 32) * (1LL << r);
        lim[j + 1] += hs & 0xffffffffLL;
        lim[j + 2] += hs >> 32;
    }
    long long carry = 0;
    for (int i = 0; i < nl; i++) {
        long long t = lim[i] + carry;
        lim[i] = t & 0xffffffffLL;
        carry = t >> 32;
    }
    const bool neg = carry < 0;
    if (neg) {
        unsigned long long cy = 1;
        for (int i = 0; i < nl; i++) {
            unsigned long long t = ((~(unsigned long long)lim[i]) & 0xffffffffull) + cy;
            lim[i] = (long long)(t & 0xffffffffull);
            cy = t >> 32;
        }
    }
    int hl = -1;
    for (int i = nl - 1; i >= 0; i--)
        if (lim[i]) { hl = i; break; }
    if (hl < 0) return 0.0;
    const int top = hl * 32 + 31 - __clz((unsigned)lim[hl]);
    // a 96-bit window of limbs hl-2 .. hl holds the 53 mantissa bits and the rounding bit
    const int base = (hl - 2) * 32;
    unsigned __int128 w = ((unsigned __int128)(unsigned long long)lim[hl] << 64) |
                          ((unsigned __int128)(unsigned long long)(hl >= 1 ? lim[hl - 1] : 0) << 32) |
                          (unsigned __int128)(unsigned long long)(hl >= 2 ? lim[hl - 2] : 0);
    unsigned long long mant;
    int shift = 0;
    if (top <= 52) {
        mant = (unsigned long long)(w >> (0 - base));            // base = -64 or -32 here: the whole value
    } else {
        shift = top - 52;
        const int r = shift - base;                              // window position of the lowest mantissa bit
        mant = (unsigned long long)(w >> r) & ((1ull << 53) - 1);
        const unsigned long long rb = (unsigned long long)(w >> (r - 1)) & 1ull;
        bool sticky = r >= 2 && (w & (((unsigned __int128)1 << (r - 1)) - 1)) != 0;
        for (int i = hl - 3; i >= 0 && !sticky; i--) sticky = lim[i] != 0;
        if (rb && (sticky || (mant & 1ull))) {
            mant++;
            if (mant == (1ull << 53)) { mant >>= 1; shift++; }
        }
    }
    double v = ldexp((double)mant, shift + e0);
    return neg ? -v : v;
}

// The per-iteration finish needs the means (S); the sums of squares (Q) are only reported,
// so they are rounded when statistics are read.
__device__ void finalize_label(const Job& J, int m, bool with_Q)
{
    long long n = J.st_n[m];
    double S;
    if (J.stats_mode == SEG_STATS_EXACT && J.dtype == SEG_U16) {
        S = __ll2double_rn(J.st_S[m]);
        if (with_Q) J.Q64[m] = __ll2double_rn(J.st_Q[m]);
    } else if (J.stats_mode == SEG_STATS_EXACT) {
        S = round_bins(J.st_S + (long long)m * J.nS, J.nS, J.slot_lo - 150);
        if (with_Q) J.Q64[m] = round_bins(J.st_Q + (long long)m * J.nQ, J.nQ, 2 * (J.slot_lo - 150));
    } else if (J.stats_mode == SEG_STATS_F64) {
        S = J.sf64[m];
        if (with_Q) J.Q64[m] = J.sf64[J.M + m];
    } else {
        const unsigned long long ps = J.sk32[m];
        S = __dadd_rn((double)__uint_as_float((unsigned)ps), (double)__uint_as_float((unsigned)(ps >> 32)));
        if (with_Q) {
            const unsigned long long pq = J.sk32[J.M + m];
            J.Q64[m] = __dadd_rn((double)__uint_as_float((unsigned)pq), (double)__uint_as_float((unsigned)(pq >> 32)));
        }
    }
    const double dn = (double)n;
    const double mu = n > 0 ? __ddiv_rn(S, dn) : 0.0;
    const double wp = __ddiv_rn(dn, __dadd_rn(dn, 1.0));
    const double wm = n > 1 ? __ddiv_rn(dn, __dsub_rn(dn, 1.0)) : 0.0;
    J.S64[m] = S;
    J.mu64[m] = mu;
    J.wp64[m] = wp;
    J.wm64[m] = wm;
    J.mu32[m] = __double2float_rn(mu);
    J.wp32[m] = __double2float_rn(wp);
    J.wm32[m] = __double2float_rn(wm);
}

// Initial statistics: warp-aggregated atomics keyed by (label, slot).
__device__ __forceinline__ void warp_add(unsigned long long key, bool valid, long long val, long long* addr)
{
    const int lane = threadIdx.x & 31;
    unsigned long long k = valid ? key : ~0ull;
    unsigned peers = __match_any_sync(0xffffffffu, k);
    long long sum = 0;
    for (int i = 0; i < 32; i++) {
        long long v = __shfl_sync(0xffffffffu, val, i);
        if ((peers >> i) & 1u) sum += v;
    }
    if (valid && lane == __ffs(peers) - 1 && sum) atomic_add_ll(addr, sum);
}

__global__ void __launch_bounds__(256) k_stats_init(const Job* jobs, int j, bool after_split)
{
    if (after_split) pdl_enter();
    const Job& J = jobs[j];
    // after the moves: only when regions split (their pieces were relabelled); the tables were
    // zeroed by k_stats_zero
    if (after_split && (ld_volatile(&J.ctr->n_split) == 0 || ld_volatile(&J.ctr->skip))) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n = J.npix;
    const long long rounds = (n + stride - 1) / stride;
    for (long long r = 0; r < rounds; r++) {
        long long i = r * stride + blockIdx.x * (long long)blockDim.x + threadIdx.x;
        bool valid = i < n;
        int m = valid ? J.L[i] : 0;
        warp_add((unsigned long long)m, valid, 1, J.st_n + m);
        if (J.stats_mode != SEG_STATS_EXACT) {
            // inexact modes: the peers of one label add their values lane by lane (FP64, or
            // compensated FP32), the group's first lane applies the result
            const unsigned peers = __match_any_sync(0xffffffffu, valid ? (unsigned)m : 0xffffffffu);
            float v = 0.0f, q = 0.0f, qe = 0.0f;
            if (valid) value_parts(J, i, v, q, qe);
            const int lane = threadIdx.x & 31;
            if (J.stats_mode == SEG_STATS_F64) {
                double s = 0.0, s2 = 0.0;
                for (int k = 0; k < 32; k++) {
                    const double vk = (double)__shfl_sync(0xffffffffu, v, k);
                    if ((peers >> k) & 1u) { s = __dadd_rn(s, vk); s2 = __dadd_rn(s2, __dmul_rn(vk, vk)); }
                }
                if (valid && lane == __ffs(peers) - 1) {
                    atomicAdd(J.sf64 + m, s);
                    atomicAdd(J.sf64 + J.M + m, s2);
                }
            } else {
                unsigned long long ps = 0, pq = 0;
                for (int k = 0; k < 32; k++) {
                    const float vk = __shfl_sync(0xffffffffu, v, k);
                    const float qk = __shfl_sync(0xffffffffu, q, k), ek = __shfl_sync(0xffffffffu, qe, k);
                    if ((peers >> k) & 1u) { ps = neumaier2(ps, vk, 0.0f); pq = neumaier2(pq, qk, ek); }
                }
                if (valid && lane == __ffs(peers) - 1) {
                    kahan_add(J.sk32 + m, __uint_as_float((unsigned)ps), __uint_as_float((unsigned)(ps >> 32)), J.ctr);
                    kahan_add(J.sk32 + J.M + m, __uint_as_float((unsigned)pq), __uint_as_float((unsigned)(pq >> 32)), J.ctr);
                }
            }
            continue;
        }
        if (J.dtype == SEG_U16) {
            long long v = valid ? ((const unsigned short*)J.I)[i] : 0;
            warp_add((unsigned long long)m, valid, v, J.st_S + m);
            warp_add((unsigned long long)m, valid, v * v, J.st_Q + m);
        } else {
            int slot = 0;
            long long sm = 0;
            unsigned long long lo = 0, hi = 0;
            if (valid) f32_parts(((const float*)J.I)[i], slot, sm, lo, hi);
            bool nz = valid && sm != 0;
            int kk = nz ? slot - J.slot_lo : 0;
            unsigned long long key = ((unsigned long long)m << 16) | (unsigned)kk;
            warp_add(key, nz, sm, J.st_S + (long long)m * J.nS + kk);
            warp_add(key, nz, (long long)lo, J.st_Q + (long long)m * J.nQ + 2 * kk);
            warp_add(key, nz, (long long)hi, J.st_Q + (long long)m * J.nQ + 2 * kk + 24);
        }
    }
}

__global__ void k_stats_finalize(const Job* jobs, int njobs)
{
    for (int j = 0; j < njobs; j++) {
        const Job& J = jobs[j];
        for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < J.M; m += gridDim.x * blockDim.x) finalize_label(J, m, true);
    }
}

// zero every statistic table of job j before k_stats_init recomputes them after a split
__global__ void __launch_bounds__(256) k_stats_zero(const Job* jobs, int j)
{
    pdl_enter();
    const Job& J = jobs[j];
    if (ld_volatile(&J.ctr->n_split) == 0 || ld_volatile(&J.ctr->skip)) return;
    const long long M = J.M;
    const long long nS = J.dtype == SEG_F32 ? J.nS : 1, nQ = J.dtype == SEG_F32 ? J.nQ : 1;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M * (1 + nS + nQ); i += stride) {
        if (i < M) J.st_n[i] = 0;
        else if (i < M * (1 + nS)) J.st_S[i - M] = 0;
        else J.st_Q[i - M * (1 + nS)] = 0;
        if (i < 2 * M) {
            if (J.sf64) J.sf64[i] = 0.0;
            if (J.sk32) J.sk32[i] = 0ull;
        }
    }
}

cudaError_t launch_stats_zero_after_split(const Job* jobs, int j, const Job& h, cudaStream_t s)
{
    const long long nS = h.dtype == SEG_F32 ? h.nS : 1, nQ = h.dtype == SEG_F32 ? h.nQ : 1;
    const long long n = (long long)h.M * (1 + nS + nQ);
    const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, 1024);
    return launch_stage(k_stats_zero, grid, 256, 0, s, jobs, j);
}

cudaError_t launch_stats_init(const Job* jobs, int j, long long npix, cudaStream_t s, bool after_split)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = (npix + 255) / 256;
    int grid = (int)(want < (long long)sms * 8 ? want : (long long)sms * 8);
    if (grid < 1) grid = 1;
    if (after_split) return launch_stage(k_stats_init, grid, 256, 0, s, jobs, j, true);
    count_launch();
    k_stats_init<<<grid, 256, 0, s>>>(jobs, j, false);
    return cudaGetLastError();
}

// One pass over the inputs: label range, float32 exponent range and largest magnitude (or the
// largest uint16 value), NaN/infinity, and the number of particles of the initial labels
// (per pixel, the distinct labels among its 4 (2D) or 6 (3D) neighbours that differ from its
// own). out must hold the identities of the reductions on entry.
__global__ void k_scan_inputs(const void* I, int dtype, const int* L, int ndim, int D, int H, int W, InputScan* out)
{
    const long long npix = (long long)D * H * W;
    int lmin = 0x7fffffff, lmax = -0x7fffffff - 1, slo = 0x7fffffff, shi = -1, bad = 0, neg = 0;
    unsigned mabs = 0;
    unsigned long long parts = 0, pairs = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npix; i += (long long)gridDim.x * blockDim.x) {
        const int l = L[i];
        lmin = min(lmin, l);
        lmax = max(lmax, l);
        if (dtype == SEG_F32) {
            const unsigned b = ((const unsigned*)I)[i];
            const int eb = (int)((b >> 23) & 0xffu);
            if (eb == 255) bad = 1;
            else if (b & 0x7fffffffu) {
                if (b >> 31) neg = 1;
                const int slot = eb ? eb : 1;
                slo = min(slo, slot);
                shi = max(shi, slot);
                mabs = max(mabs, b & 0x7fffffffu);
            }
        } else {
            mabs = max(mabs, (unsigned)((const unsigned short*)I)[i]);
        }
        const long long x = i % W, y = (i / W) % H, z = i / ((long long)W * H);
        int nb[6];
        int n = 0;
        if (x > 0) nb[n++] = L[i - 1];
        if (x + 1 < W) nb[n++] = L[i + 1];
        if (y > 0) nb[n++] = L[i - W];
        if (y + 1 < H) nb[n++] = L[i + W];
        if (ndim == 3 && z > 0) nb[n++] = L[i - (long long)W * H];
        if (ndim == 3 && z + 1 < D) nb[n++] = L[i + (long long)W * H];
        pairs += (x + 1 < W && L[i + 1] != l) + (y + 1 < H && L[i + W] != l) +
                 (ndim == 3 && z + 1 < D && L[i + (long long)W * H] != l);
        for (int a = 0; a < n; a++) {
            if (nb[a] == l) continue;
            bool first = true;
            for (int b2 = 0; b2 < a; b2++) first &= nb[b2] != nb[a];
            parts += first ? 1u : 0u;
        }
    }
    lmin = __reduce_min_sync(0xffffffffu, lmin);
    lmax = __reduce_max_sync(0xffffffffu, lmax);
    slo = __reduce_min_sync(0xffffffffu, slo);
    shi = __reduce_max_sync(0xffffffffu, shi);
    bad = __reduce_or_sync(0xffffffffu, (unsigned)bad);
    neg = __reduce_or_sync(0xffffffffu, (unsigned)neg);
    mabs = __reduce_max_sync(0xffffffffu, mabs);
    for (int o = 16; o > 0; o >>= 1) parts += __shfl_down_sync(0xffffffffu, parts, o);
    for (int o = 16; o > 0; o >>= 1) pairs += __shfl_down_sync(0xffffffffu, pairs, o);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&out->lab_min, lmin);
        atomicMax(&out->lab_max, lmax);
        atomicMin(&out->slot_lo, slo);
        atomicMax(&out->slot_hi, shi);
        atomicMax(&out->maxabs, mabs);
        if (bad) atomicOr(&out->bad, 1);
        if (neg) atomicOr(&out->neg, 1);
        if (parts) atomicAdd(&out->particles, parts);
        if (pairs) atomicAdd(&out->pairs, pairs);
    }
}

cudaError_t launch_scan_inputs(const void* I, int dtype, const int* L, int ndim, int D, int H, int W, InputScan* out,
                               cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long npix = (long long)D * H * W;
    long long want = (npix + 255) / 256;
    int grid = (int)(want < (long long)sms * 8 ? want : (long long)sms * 8);
    if (grid < 1) grid = 1;
    count_launch();
    k_scan_inputs<<<grid, 256, 0, s>>>(I, dtype, L, ndim, D, H, W, out);
    return cudaGetLastError();
}

cudaError_t launch_stats_finalize(const Job* jobs, int njobs, cudaStream_t s)
{
    count_launch();
    k_stats_finalize<<<64, 128, 0, s>>>(jobs, njobs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Commit, one co-resident grid with bounded barriers:
//  A. each candidate lists its neighbouring candidates (Chebyshev distance 1) with a
//     smaller (key, pixel);
//  B. rounds: a candidate is accepted once all smaller neighbours are rejected and
//     rejected as soon as one is accepted; this equals the greedy pass in ascending
//     (key, pixel) order, whatever the processing order;
//  C. accepted moves update labels and the exact region sums;
//  D. region tables, oscillation fallback, status, counters for the next iteration.
// The order of two (key, pixel) pairs on the keys' order-preserving integer images, so that the
// neighbour lists compare on the integer pipes (the FP64 pipe is narrow here)
__device__ __forceinline__ bool key_less(unsigned long long ka, unsigned pa, unsigned long long kb, unsigned pb)
{
    return ka < kb || (ka == kb && pa < pb);
}

__device__ __forceinline__ unsigned block_sum(unsigned v, unsigned* s_red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned tot = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) tot += s_red[i];
    return tot;   // valid in thread 0
}

constexpr unsigned kMaxRounds = 1u << 20;
constexpr unsigned kSmallCandidates = 32768;   // at most this many: one block decides alone
constexpr size_t kRoundsDyn = 160 * 1024;      // dynamic shared memory of the rounds kernel

// A: neighbour lists of smaller-key candidates; states reset
// Neighbour positions by compile-time index (dz, dy, dx ascending, the centre skipped), so
// that the per-neighbour arrays stay in registers.
constexpr int kMarked = (int)0x80000000u;    // a list entry whose order the rounds settle

template <int NDIM>
__device__ __forceinline__ void commit_list_nd(const Job& J, unsigned s)
{
    constexpr int K = NDIM == 3 ? 27 : 9;
    const unsigned tag = ld_volatile(&J.ctr->iter_tag);
    const unsigned gi = J.c_pix[s];
    const unsigned long long ks = J.c_key[s];
    int x, y, z;
    coords(J, gi, x, y, z);
    // three dependent levels (pixel map, candidate slot, key), each level's loads for all
    // neighbours issued together
    unsigned long long e[K];
    unsigned in = 0;
#pragma unroll
    for (int t = 0; t < K; t++) {
        const int dz = NDIM == 3 ? t / 9 - 1 : 0, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        const int xx = x + dx, yy = y + dy, zz = z + dz;
        const bool ok = t != K / 2 && xx >= 0 && xx < J.W && yy >= 0 && yy < J.H && zz >= 0 && zz < J.D;
        e[t] = ok ? J.pmap[(unsigned)(((long long)zz * J.H + yy) * J.W + xx)] : 0ull;
        in |= ok ? 1u << t : 0u;
    }
    int slot[K];
#pragma unroll
    for (int t = 0; t < K; t++)
        slot[t] = ((in >> t) & 1u) && (unsigned)(e[t] >> 32) == tag ? J.pix_cand[(unsigned)e[t]] : -1;
    const float2 gs = J.c_ge[s];
    bool uncertain = false;
    int n = 0;
#pragma unroll
    for (int t = 0; t < K; t++) {
        const int o = slot[t];
        if (o < 0) continue;
        // a pair whose gap is not certified enters the list marked, whatever the float order:
        // both keys are recomputed in FP64, and the rounds compare them then
        const bool unc = gs.y > 0.0f && order_uncertain(gs.x, gs.y, J.c_ge[o].x, J.c_ge[o].y);
        uncertain |= unc;
        if (unc) J.c_nbr[(long long)s * J.nbr_stride + n++] = o | kMarked;
        else if (key_less(J.c_key[o], J.c_pix[o], ks, gi)) J.c_nbr[(long long)s * J.nbr_stride + n++] = o;
    }
    J.c_nnbr[s] = n;
    J.c_state[s] = kUndecided;
    if (uncertain) {
        const unsigned p = (unsigned)J.c_best[s];
        if (!(J.p_flags[p] & kFlagFixup)) queue_fixup(J, s, p);   // not already queued for its sign
    }
}

__device__ __forceinline__ void commit_list_one(const Job& J, unsigned s)
{
    if (J.ndim == 3) commit_list_nd<3>(J, s);
    else commit_list_nd<2>(J, s);
}

// A list entry of candidate s: candidate o when it has the smaller (key, pixel), -1 when it
// does not. Unmarked entries are smaller by construction; a marked one is compared on the
// keys, exact by the time the rounds run.
__device__ __forceinline__ int list_entry(const Job& J, unsigned s, int e)
{
    if (!(e & kMarked)) return e;
    const int o = e & ~kMarked;
    return key_less(J.c_key[o], J.c_pix[o], J.c_key[s], J.c_pix[s]) ? o : -1;
}

// B: one decision for candidate s of job J on state array st (offset b); returns the new
// state (kUndecided when it has to wait)
template <class State>
__device__ __forceinline__ int commit_decide(const Job& J, unsigned s, State st, unsigned b)
{
    const int n = J.c_nnbr[s];
    const int* nb = J.c_nbr + (long long)s * J.nbr_stride;
    bool all_rej = true;
    for (int i = 0; i < n; i++) {
        const int o = list_entry(J, s, nb[i]);
        if (o < 0) continue;
        const int v = st[b + o];
        if (v == kAccepted) return kRejected;
        if (v != kRejected) all_rej = false;
    }
    return all_rej ? kAccepted : kUndecided;
}

// C: one accepted move changes the label and the exact region sums
__device__ __forceinline__ void commit_move_one(const Job& J, unsigned s)
{
    const int p = J.c_best[s];
    const unsigned gi = J.c_pix[s];
    const int l = J.p_l[p], c = J.p_c[p];
    if (J.global_E) {
        // |Gamma| changes by the move's change of unlike neighbour pairs; accepted moves are
        // never adjacent, so their changes add up exactly
        int x, y, z;
        pix_coords(J, gi, x, y, z);
        long long dP = 0;
        const long long HW = (long long)J.W * J.H;
        if (x > 0) { const int m = J.L[gi - 1]; dP += (m != c) - (m != l); }
        if (x + 1 < J.W) { const int m = J.L[gi + 1]; dP += (m != c) - (m != l); }
        if (y > 0) { const int m = J.L[gi - J.W]; dP += (m != c) - (m != l); }
        if (y + 1 < J.H) { const int m = J.L[gi + J.W]; dP += (m != c) - (m != l); }
        if (J.ndim == 3 && z > 0) { const int m = J.L[gi - HW]; dP += (m != c) - (m != l); }
        if (J.ndim == 3 && z + 1 < J.D) { const int m = J.L[gi + HW]; dP += (m != c) - (m != l); }
        if (dP) atomicAdd((unsigned long long*)&J.ctr->perim, (unsigned long long)dP);
    }
    J.L[gi] = c;
    J.p_flags[p] |= kFlagAcc;
    if (J.p_flags[p] & kFlagSplit) atomicAdd(&J.ctr->n_split, 1u);   // the iteration relabels
    if (J.stats_mode != SEG_STATS_EXACT) {    // the exact sums are added per warp by the caller
        stats_move(J, gi, l, -1);
        stats_move(J, gi, c, +1);
    }
}

// Exact statistic deltas of the warp's moves (one pixel leaving m, sign -1, or joining it,
// sign +1). Every lane of the warp calls this; `valid` marks the lanes with a move of an
// exact-statistics job. uint16 images: the lanes that hit the same label are summed first (a
// 3D move mostly shares its label with other lanes); float32 images: one atomic per lane and
// exponent slot, as the per-lane sums would spread over many slots.
__device__ __forceinline__ void stats_move_warp(const Job* jobs, int j, bool valid, unsigned gi, int m, int sign)
{
    const bool u16 = valid && jobs[j].dtype == SEG_U16;
    if (valid && !u16) stats_move(jobs[j], gi, m, sign);
    if (!__any_sync(0xffffffffu, u16)) return;
    const Job& J = jobs[u16 ? j : 0];
    const unsigned long long key = u16 ? (((unsigned long long)j << 32) | (unsigned)m) : 0ull;
    const long long v = u16 ? ((const unsigned short*)J.I)[gi] : 0;
    const long long mo = u16 ? m : 0;
    warp_add(key, u16, sign, J.st_n + mo);
    warp_add(key, u16, sign * v, J.st_S + mo);
    warp_add(key, u16, sign * v * v, J.st_Q + mo);
}

// D: per-job oscillation fallback, status and counters for the next iteration
__device__ void commit_job_status(const Job& J, bool ok, unsigned rounds, int err)
{
    Counters* c = J.ctr;
    if (!ok) atomicExch(&c->error, err ? err : SEG_ETIMEOUT);
    if (c->error || c->need) {
        c->skip = 1;
        c->last.error = c->error ? c->error : SEG_ENOMEM;
        return;
    }
    if (c->converged) {
        c->last.iteration = c->t;
        c->last.n_particles = 0;
        c->last.n_candidates = 0;
        c->last.n_accepted = 0;
        c->last.n_osc = 0;
        c->last.n_fixup = 0;
        c->last.mode_used = c->mode;
        c->last.converged = 1;
        c->last.mis_rounds = 0;
        c->last.error = 0;
        c->last.particles_total = c->cum_particles;
        c->t++;
        return;
    }
    const long long A = c->n_accepted;
    const int used = c->mode;
    if (c->best_A < 0 || A < c->best_A) { c->best_A = A; c->t_best = c->t; }
    if (c->mode != SEG_L2 && J.osc_window > 0 && c->t - c->t_best >= J.osc_window) c->mode = SEG_L2;
    if (used == SEG_L2 && A == 0) c->converged = 1;
    c->last.iteration = c->t;
    c->last.n_particles = c->n_particles;
    c->last.n_candidates = c->n_cand - c->n_void;
    c->last.n_accepted = A;
    c->last.n_osc = used != SEG_L2 ? c->n_osc : 0;
    c->last.n_fixup = c->n_flag;
    c->last.mode_used = used;
    c->last.converged = c->converged;
    c->last.mis_rounds = (int)rounds;
    c->last.error = 0;
    c->cum_particles += c->n_particles;
    c->last.particles_total = c->cum_particles;
    c->t++;
    c->iter_tag++;
    c->n_flag = 0;
    c->n_split = 0;
    c->n_newcomp = 0;
    c->n_cand = 0;
    c->n_void = 0;
    c->n_accepted = 0;
    c->n_osc = 0;
    c->skip = c->converged;
}

// FP64 recompute of the queued particles' keys in the order of the definition, one block per
// particle: every thread takes one interaction offset (row-major, i.e. ascending pixel) and
// the particles of that pixel in order, so that the dependent loads of all offsets overlap;
// one thread then sums the terms in ascending key order.
__global__ void __launch_bounds__(kFixThreads) k_fixup(const Job* jobs, int njobs)
{
    pdl_enter();
    __shared__ double s_t[kFixTerms];
    __shared__ unsigned char s_a[kFixTerms];
    __shared__ unsigned s_pref[kMaxBatchJobs + 1];
    __shared__ unsigned s_tmp[32];
    __shared__ int s_w[kFixThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned total = block_job_prefix(jobs, njobs, kCountFlag, s_pref, s_tmp);
    if (total > gridDim.x) {                   // many queued particles: one per warp
        fixup_warps(jobs, njobs, total, s_pref, s_t, s_a);
    } else
    for (unsigned fi = blockIdx.x; fi < total; fi += gridDim.x) {
        const int j = job_of(s_pref, njobs, fi);
        const Job& J = jobs[j];
        Counters* ctr = J.ctr;
        const unsigned f = fi - s_pref[j];
        const unsigned tag = ld_volatile(&ctr->iter_tag);
        const unsigned np = ld_volatile(&ctr->n_particles);
        const int mode = ld_volatile(&ctr->mode);
        const unsigned sl = J.flag_list[f];
        const unsigned p = (unsigned)J.c_best[sl];
        const unsigned gi = J.p_idx[p];
        const int lp = J.p_l[p];
        if (mode == SEG_L2) {
            if (tid == 0) fix_apply(J, sl, p, J.p_dE64[p]);
        } else if (mode == SEG_SOBOLEV_GLOBAL) {
            if (w == 0) {
                const double gval = fix_global_warp(J, gi, lp, tag, np, s_t, s_a);
                if (lane == 0) fix_apply(J, sl, p, gval);
            }
        } else {
            int x, y, z;
            coords(J, gi, x, y, z);
            double As = 0.0, Bs = 0.0;
            long long nA = 0, nB = 0;
            for (int base = 0; base < J.nb_n; base += kFixThreads) {
                const int u = base + tid;
                double tv[6];
                unsigned char ta[6];
                int nt = 0;
                if (u < J.nb_n) {
                    const int4 d = J.nb_off[u];
                    const int xx = x + d.z, yy = y + d.y, zz = z + d.x;
                    if (xx >= 0 && xx < J.W && yy >= 0 && yy < J.H && zz >= 0 && zz < J.D) {
                        const unsigned yi = (unsigned)(((long long)zz * J.H + yy) * J.W + xx);
                        const unsigned long long e = J.pmap[yi];
                        if ((unsigned)(e >> 32) == tag) {
                            const double K = J.klut64[d.w];
                            for (unsigned q = (unsigned)e; q < np && J.p_idx[q] == yi && nt < 6; q++) {
                                const int lq = J.p_l[q], cq = J.p_c[q];
                                if (lq == lp || cq == lp) {
                                    tv[nt] = __dmul_rn(K, J.p_dE64[q]);
                                    ta[nt] = lq == lp ? 1 : 0;
                                    nt++;
                                }
                            }
                        }
                    }
                }
                int tot;
                const int pos = block_excl(nt, s_w, &tot);
                for (int i = 0; i < nt; i++) {
                    s_t[pos + i] = tv[i];
                    s_a[pos + i] = ta[i];
                }
                __syncthreads();
                if (tid == 0) {
                    for (int i = 0; i < tot; i++) {
                        if (s_a[i]) { As = __dadd_rn(As, s_t[i]); nA++; }
                        else { Bs = __dadd_rn(Bs, s_t[i]); nB++; }
                    }
                }
                __syncthreads();
            }
            if (tid == 0) {
                const double A = nA ? __ddiv_rn(As, (double)nA) : 0.0;
                const double B = nB ? __ddiv_rn(Bs, (double)nB) : 0.0;
                fix_apply(J, sl, p, __dsub_rn(A, B));
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_fixup(const Job* jobs, int njobs, int sms, cudaStream_t s)
{
    if (njobs <= 0) return cudaSuccess;
    return launch_stage(k_fixup, sms * 8, kFixThreads, 0, s, jobs, njobs);
}

// A, as its own grid, over the flattened candidates of all jobs
__global__ void __launch_bounds__(256, 4) k_lists(const Job* jobs, int njobs)
{
    pdl_enter();
    __shared__ unsigned s_pref[kMaxBatchJobs + 1];
    __shared__ unsigned s_tmp[32];
    const unsigned total = block_job_prefix(jobs, njobs, kCountCand, s_pref, s_tmp);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int j = job_of(s_pref, njobs, i);
        commit_list_one(jobs[j], i - s_pref[j]);
    }
}

// B: the rounds. With few candidates one block runs them on shared-memory states with
// block barriers; otherwise the whole co-resident grid runs them with bounded grid barriers.
__global__ void __launch_bounds__(1024) k_rounds(const Job* jobs, int njobs, BatchCtl* bc)
{
    pdl_enter();
    __shared__ unsigned s_red[32];
    __shared__ unsigned s_flag;
    __shared__ unsigned s_pref[kMaxBatchJobs + 1];
    __shared__ unsigned char s_state[kSmallCandidates + 1];   // + a sentinel, always rejected
    extern __shared__ __align__(16) unsigned char s_dyn[];
    const unsigned total = block_job_prefix(jobs, njobs, kCountCand, s_pref, s_red);
    if (total <= kSmallCandidates) {
        if (blockIdx.x != 0) return;
        volatile unsigned char* st = s_state;
        // The candidates' neighbour lists (compressed rows of 16-bit flattened indices) and a
        // list of the undecided candidates live in shared memory when they fit; each round then
        // visits only the undecided candidates.
        __shared__ unsigned s_cnt3[3];
        const unsigned chunk = (total + blockDim.x - 1) / blockDim.x;
        const unsigned c0 = min(threadIdx.x * chunk, total), c1 = min(c0 + chunk, total);
        unsigned* s_off = (unsigned*)s_dyn;                                 // [total + 1]
        const size_t off_bytes = ((size_t)(total + 1) * 4 + 15) & ~(size_t)15;
        unsigned short* s_wl0 = (unsigned short*)(s_dyn + off_bytes);      // [total]
        unsigned short* s_wl1 = s_wl0 + total;                              // [total]
        const size_t wl_bytes = ((size_t)total * 4 + 15) & ~(size_t)15;
        unsigned short* s_nb = (unsigned short*)(s_dyn + off_bytes + wl_bytes);
        // counts (coalesced), offsets by a block scan over contiguous chunks, then the rows;
        // nothing is written to the dynamic region unless the offsets and both lists fit
        const bool room = off_bytes + wl_bytes <= kRoundsDyn;
        if (room)
            for (unsigned i = threadIdx.x; i < total; i += blockDim.x) {
                const int j = job_of(s_pref, njobs, i);
                s_wl1[i] = (unsigned short)jobs[j].c_nnbr[i - s_pref[j]];
            }
        __syncthreads();
        unsigned mine = 0;
        if (room)
            for (unsigned i = c0; i < c1; i++) mine += s_wl1[i];
        unsigned all_nb;
        const unsigned nb0 = block_excl_scan(mine, s_red, all_nb);
        const bool cache = room && off_bytes + wl_bytes + (size_t)all_nb * 2 <= kRoundsDyn;   // uniform
        if (cache) {
            unsigned o = nb0;
            for (unsigned i = c0; i < c1; i++) {
                s_off[i] = o;
                o += s_wl1[i];
            }
            if (threadIdx.x == blockDim.x - 1) s_off[total] = all_nb;
        }
        __syncthreads();
        if (cache) {
            for (unsigned i = threadIdx.x; i < total; i += blockDim.x) {
                const int j = job_of(s_pref, njobs, i);
                const Job& J = jobs[j];
                const int* nb = J.c_nbr + (long long)(i - s_pref[j]) * J.nbr_stride;
                const unsigned n = s_wl1[i], o = s_off[i], b = s_pref[j];
#pragma unroll 8
                for (unsigned k = 0; k < n; k++) {
                    const int e = list_entry(J, i - b, nb[k]);
                    s_nb[o + k] = (unsigned short)(e >= 0 ? b + (unsigned)e : total);   // total: the sentinel
                }
            }
        }
        for (unsigned i = threadIdx.x; i < total; i += blockDim.x) {
            const int j = job_of(s_pref, njobs, i);
            st[i] = (unsigned char)jobs[j].c_state[i - s_pref[j]];   // undecided, or dropped by the recompute
            if (cache) s_wl0[i] = (unsigned short)i;
        }
        if (threadIdx.x == 0) st[total] = kRejected;               // the sentinel of settled entries
        if (threadIdx.x == 0) s_cnt3[0] = 0;
        __syncthreads();
        unsigned rounds = 0;
        bool ok = true;
        if (cache) {
            // one barrier per round: round r appends to s_cnt3[r % 3] while thread 0 clears the
            // counter of round r + 1 (last read before the barrier that ended round r - 1)
            unsigned n_cur = total;
            unsigned short* cur = s_wl0;
            unsigned short* nxt = s_wl1;
            const unsigned lane = threadIdx.x & 31;
            for (unsigned r = 0; n_cur > 0; r++) {
                if (r >= kMaxRounds) { ok = false; break; }
                unsigned* cnt = &s_cnt3[r % 3];
                if (threadIdx.x == 0) s_cnt3[(r + 1) % 3] = 0;
                for (unsigned t = threadIdx.x; t < n_cur; t += blockDim.x) {
                    const unsigned i = cur[t];
                    const int v0 = st[i];              // decided already: dropped by the recompute
                    bool all_rej = true, rej = false;
                    if (v0 == kUndecided)
                        for (unsigned k = s_off[i], e = s_off[i + 1]; k < e; k++) {
                            const int u = st[s_nb[k]];
                            if (u == kAccepted) { rej = true; break; }
                            if (u != kRejected) all_rej = false;
                        }
                    const int v = v0 != kUndecided ? v0 : (rej ? kRejected : (all_rej ? kAccepted : kUndecided));
                    if (v0 == kUndecided && v != kUndecided) st[i] = (unsigned char)v;
                    const unsigned act = __activemask();
                    const unsigned m = __ballot_sync(act, v == kUndecided);
                    if (m) {
                        const unsigned leader = __ffs(m) - 1;
                        unsigned base = 0;
                        if (lane == leader) base = atomicAdd(cnt, (unsigned)__popc(m));
                        base = __shfl_sync(act, base, leader);
                        if (v == kUndecided) nxt[base + __popc(m & ((1u << lane) - 1u))] = (unsigned short)i;
                    }
                }
                __syncthreads();
                n_cur = *(volatile unsigned*)cnt;
                unsigned short* tmp = cur;
                cur = nxt;
                nxt = tmp;
                rounds = r + 1;
            }
        } else {
        for (unsigned r = 0;; r++) {
            unsigned und = 0;
            for (unsigned i = threadIdx.x; i < total; i += blockDim.x) {
                if (st[i] != kUndecided) continue;
                const int j = job_of(s_pref, njobs, i);
                const unsigned b = s_pref[j];
                const int v = commit_decide(jobs[j], i - b, st, b);
                if (v == kUndecided) und++;
                else st[i] = (unsigned char)v;
            }
            const unsigned bs = block_sum(und, s_red);
            if (threadIdx.x == 0) s_flag = bs;
            __syncthreads();
            const unsigned rem = s_flag;
            __syncthreads();
            if (rem == 0) { rounds = r + 1; break; }
            if (r + 1 >= kMaxRounds) { ok = false; break; }
        }
        }
        for (unsigned i = threadIdx.x; i < total; i += blockDim.x) {
            const int j = job_of(s_pref, njobs, i);
            jobs[j].c_state[i - s_pref[j]] = st[i];
        }
        if (threadIdx.x == 0) {
            bc->rounds_done = rounds;
            if (!ok) atomicExch(&bc->err, SEG_ETIMEOUT);
        }
        return;
    }

    // The whole co-resident grid. Block b owns the candidate indices [lo, hi); candidates are
    // numbered tile by tile, so that is a compact part of each image. Decisions are final once
    // made and depend only on smaller-key neighbours, so the order in which blocks and sweeps
    // make them does not change them.
    // When they fit, the range's states and rows sit in shared memory: a row entry is the local
    // index of a neighbour inside the range, or (top bit set) the job slot of one outside it, read
    // from global memory. Every decision is also written to global memory as it is made.
    const unsigned nblocks = gridDim.x;
    const unsigned per = (total + nblocks - 1) / nblocks;
    const unsigned lo = min(blockIdx.x * per, total), hi = min(lo + per, total);
    const unsigned n = hi - lo;
    volatile unsigned char* st = s_state;
    unsigned* s_roff = (unsigned*)s_dyn;                                     // [n + 1]
    const size_t roff_bytes = ((size_t)(n + 1) * 4 + 15) & ~(size_t)15;
    unsigned* s_ent = (unsigned*)(s_dyn + roff_bytes);
    bool cache = n <= kSmallCandidates && roff_bytes <= kRoundsDyn;          // uniform over the block
    if (cache) {
        for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
            const int j = job_of(s_pref, njobs, lo + i);
            s_roff[i] = (unsigned)jobs[j].c_nnbr[lo + i - s_pref[j]];
            st[i] = (unsigned char)jobs[j].c_state[lo + i - s_pref[j]];
        }
        if (threadIdx.x == 0) st[n] = kRejected;                   // the sentinel of settled entries
        __syncthreads();
        const unsigned chunk = (n + blockDim.x - 1) / blockDim.x;
        const unsigned c0 = min(threadIdx.x * chunk, n), c1 = min(c0 + chunk, n);
        unsigned mine = 0;
        for (unsigned i = c0; i < c1; i++) mine += s_roff[i];
        unsigned all_nb;
        unsigned o = block_excl_scan(mine, s_red, all_nb);
        cache = roff_bytes + (size_t)all_nb * 4 <= kRoundsDyn;
        if (cache) {
            for (unsigned i = c0; i < c1; i++) {
                const unsigned c = s_roff[i];
                s_roff[i] = o;
                o += c;
            }
            if (threadIdx.x == 0) s_roff[n] = all_nb;
        }
        __syncthreads();
        if (cache)
            for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
                const int j = job_of(s_pref, njobs, lo + i);
                const Job& J = jobs[j];
                const int* nb = J.c_nbr + (long long)(lo + i - s_pref[j]) * J.nbr_stride;
                const unsigned e0 = s_roff[i], e1 = s_roff[i + 1];
                for (unsigned k = e0; k < e1; k++) {
                    const int e = list_entry(J, lo + i - s_pref[j], nb[k - e0]);
                    const unsigned slot = (unsigned)e;
                    const unsigned loc = s_pref[j] + slot - lo;
                    s_ent[k] = e < 0 ? n : (loc < n ? loc : (slot | 0x80000000u));   // n: the sentinel
                }
            }
        __syncthreads();
    }
    // No grid-wide rounds: each block sweeps its range until all of it is decided. A sweep that
    // decides nothing while some of the range is left waits (bounded) for the other blocks'
    // decisions, which arrive through global memory; the smallest undecided candidate of the whole
    // grid can always be decided, so some block always progresses. A block leaves as soon as its
    // range is done.
    __shared__ int s_stop;
    if (threadIdx.x == 0) s_stop = 0;
    unsigned sweeps = 0;
    WaitBound wb;
    while (true) {
        int changed = 0, left = 0;
        for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
            int v;
            if (cache) {
                if (st[i] != kUndecided) continue;
                bool all_rej = true, rej = false;
                for (unsigned k = s_roff[i], e = s_roff[i + 1]; k < e; k++) {
                    const unsigned en = s_ent[k];
                    int u;
                    if (en & 0x80000000u) {
                        const Job& J = jobs[job_of(s_pref, njobs, lo + i)];
                        u = ld_volatile(J.c_state + (en & 0x7fffffffu));
                    } else {
                        u = st[en];
                    }
                    if (u == kAccepted) { rej = true; break; }
                    if (u != kRejected) all_rej = false;
                }
                v = rej ? kRejected : (all_rej ? kAccepted : kUndecided);
                if (v != kUndecided) st[i] = (unsigned char)v;
            } else {
                const int j = job_of(s_pref, njobs, lo + i);
                if (ld_volatile(jobs[j].c_state + (lo + i - s_pref[j])) != kUndecided) continue;
                v = commit_decide(jobs[j], lo + i - s_pref[j], (const volatile int*)jobs[j].c_state, 0u);
            }
            if (v == kUndecided) {
                left = 1;
            } else {
                const int j = job_of(s_pref, njobs, lo + i);
                *(volatile int*)(jobs[j].c_state + (lo + i - s_pref[j])) = v;
                changed = 1;
            }
        }
        ++sweeps;
        if (!__syncthreads_or(left)) break;
        if (__syncthreads_or(changed)) {
            if (threadIdx.x == 0) wb = WaitBound();
            continue;
        }
        if (threadIdx.x == 0 && (wb.expired() || sweeps >= kMaxRounds)) {
            s_stop = 1;
            atomicExch(&bc->err, SEG_ETIMEOUT);
        }
        __syncthreads();
        if (s_stop) break;
        __nanosleep(128);
    }
    if (threadIdx.x == 0) atomicMax(&bc->rounds_done, sweeps);
}

// C, as its own grid: accepted moves; accepted counts aggregated per warp and job
__global__ void __launch_bounds__(256) k_moves(const Job* jobs, int njobs, const BatchCtl* bc)
{
    pdl_enter();
    __shared__ unsigned s_pref[kMaxBatchJobs + 1];
    __shared__ unsigned s_tmp[32];
    if (ld_volatile(&bc->err)) return;
    const unsigned total = block_job_prefix(jobs, njobs, kCountCand, s_pref, s_tmp);
    const unsigned stride = gridDim.x * blockDim.x;
    const unsigned rounds = (total + stride - 1) / stride;
    for (unsigned r = 0; r < rounds; r++) {
        const unsigned i = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
        int j = -1;
        bool acc = false;
        unsigned gi = 0;
        int l = 0, c = 0;
        if (i < total) {
            j = job_of(s_pref, njobs, i);
            const Job& J = jobs[j];
            const unsigned s = i - s_pref[j];
            if (J.c_state[s] == kAccepted) {
                const int p = J.c_best[s];
                gi = J.c_pix[s];
                l = J.p_l[p];
                c = J.p_c[p];
                commit_move_one(J, s);
                acc = true;
            }
        }
        const bool exact = acc && jobs[j].stats_mode == SEG_STATS_EXACT;
        stats_move_warp(jobs, j, exact, gi, l, -1);
        stats_move_warp(jobs, j, exact, gi, c, +1);
        const unsigned peers = __match_any_sync(0xffffffffu, acc ? j : -1);
        if (acc && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&jobs[j].ctr->n_accepted, (unsigned)__popc(peers));
    }
}

// D, as its own grid: exact region tables of every label of every job, then per-job status
__global__ void __launch_bounds__(256) k_finish(const Job* jobs, int njobs, BatchCtl* bc)
{
    pdl_enter();
    __shared__ unsigned s_pref[kMaxBatchJobs + 1];
    __shared__ unsigned s_tmp[32];
    const int err = ld_volatile(&bc->err);
    const bool ok = err == 0;
    const unsigned total = block_job_prefix(jobs, njobs, kCountLabels, s_pref, s_tmp);
    // labels go to block-leading threads first, so that their serial work spreads over SMs
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned k = threadIdx.x * gridDim.x + blockIdx.x; k < total; k += stride) {
        const int j = job_of(s_pref, njobs, k);
        const Job& J = jobs[j];
        if (ok && !job_idle(J.ctr)) finalize_label(J, (int)(k - s_pref[j]), false);
    }
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < njobs; j += stride)
        commit_job_status(jobs[j], ok, ld_volatile(&bc->rounds_done), err);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bc->ticket[0] = 0;
        bc->ticket[1] = 0;
    }
}

cudaError_t commit_occupancy(int block, int* blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(k_rounds, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRoundsDyn);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_rounds, block, kRoundsDyn);
}

cudaError_t launch_lists(const Job* jobs, int njobs, int sms, cudaStream_t s)
{
    return launch_stage(k_lists, sms * 4, 256, 0, s, jobs, njobs);
}

// the rounds kernel is cooperative: every block co-resident
cudaError_t launch_rounds(const Job* jobs, int njobs, BatchCtl* bc, int grid, int block, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = kRoundsDyn;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launch();
    return cudaLaunchKernelEx(&cfg, k_rounds, jobs, njobs, bc);
}

cudaError_t launch_moves(const Job* jobs, int njobs, BatchCtl* bc, int sms, cudaStream_t s)
{
    return launch_stage(k_moves, sms * 4, 256, 0, s, jobs, njobs, (const BatchCtl*)bc);
}

cudaError_t launch_finish(const Job* jobs, int njobs, BatchCtl* bc, int sms, cudaStream_t s)
{
    return launch_stage(k_finish, sms, 256, 0, s, jobs, njobs, bc);
}


// ---------------------------------------------------------------------------
// Fusion (SEG_TOPO_FUSE, piecewise-constant model, exact statistics): after the moves (and the
// relabelling of split pieces), touching foreground regions a < b fuse when
//     dE = w (d d) - lambda B_ab,  w = (n_a n_b) / (n_a + n_b),  d = S_a / n_a - S_b / n_b
// is negative (the exact change of the sum of squared deviations about the joint mean, minus
// the B_ab adjacent pixel pairs between them that leave the contour), greedily in ascending
// (dE, a, b), each label at most once per iteration; b's pixels then take label a.
//
//  1. k_fuse_pairs: every pixel adds its forward-neighbour pairs of different foreground
//     labels to a hash table keyed by (a << 32 | b) (warp-aggregated counts, bounded probing;
//     a full table raises SEG_ENOMEM); new keys are listed.
//  2. k_fuse_match (one block): dE per listed pair from the exact sums after the moves, the
//     table cleared; then rounds of the greedy matching: a pair is accepted when it holds the
//     smallest (dE, a, b) among the undecided pairs of both its labels (the lexicographically
//     first maximal matching, as the ranked candidate selection); accepted pairs merge their
//     exact statistics into a.
//  3. k_fuse_relabel: b -> a over the label image.
constexpr unsigned long long kFuseEmpty = ~0ull;
constexpr int kFuseBlock = 1024;
enum { kFuseOpen = 0, kFuseTaken = 1, kFuseOut = 2 };

__device__ __forceinline__ unsigned long long fuse_order(double v)
{
    // IEEE order as unsigned order
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ bool fuse_idle(const Job& J)
{
    return !J.topo_fuse || ld_volatile(&J.ctr->skip) != 0 || ld_volatile(&J.ctr->need) != 0 ||
           ld_volatile(&J.ctr->error) != 0;
}

__device__ void fuse_insert(const Job& J, unsigned long long key, bool valid)
{
    const unsigned peers = __match_any_sync(0xffffffffu, valid ? key : kFuseEmpty);
    const int lane = threadIdx.x & 31;
    if (!valid || lane != __ffs(peers) - 1) return;
    const unsigned cap = J.fz_cap;
    unsigned h = (unsigned)((key * 0x9E3779B97F4A7C15ull) >> 40) & (cap - 1);
    for (unsigned probe = 0; probe < cap; probe++, h = (h + 1) & (cap - 1)) {
        const unsigned long long prev = atomicCAS(J.fz_key + h, kFuseEmpty, key);
        if (prev == kFuseEmpty || prev == key) {
            atomicAdd(J.fz_cnt + h, (unsigned)__popc(peers));
            if (prev == kFuseEmpty) J.fz_list[atomicAdd(&J.ctr->n_fpairs, 1u)] = h;
            return;
        }
    }
    atomicExch(&J.ctr->error, SEG_ENOMEM);
}

__global__ void __launch_bounds__(256) k_fuse_pairs(const Job* jobs, int j)
{
    pdl_enter();
    const Job& J = jobs[j];
    if (fuse_idle(J)) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n = J.npix;
    const long long rounds = (n + stride - 1) / stride;
    for (long long r = 0; r < rounds; r++) {
        const long long i = r * stride + blockIdx.x * (long long)blockDim.x + threadIdx.x;
        const bool in = i < n;
        int x = 0, y = 0, z = 0, m = 0;
        if (in) {
            pix_coords(J, (unsigned)i, x, y, z);
            m = J.L[i];
        }
        for (int axis = 0; axis < 3; axis++) {
            bool ok = in && m != 0;
            long long q = 0;
            if (axis == 0) { ok = ok && x + 1 < J.W; q = i + 1; }
            else if (axis == 1) { ok = ok && y + 1 < J.H; q = i + J.W; }
            else { ok = ok && J.ndim == 3 && z + 1 < J.D; q = i + (long long)J.W * J.H; }
            const int m2 = ok ? J.L[q] : 0;
            ok = ok && m2 != 0 && m2 != m;
            const unsigned a = (unsigned)min(m, m2), b = (unsigned)max(m, m2);
            fuse_insert(J, ((unsigned long long)a << 32) | b, ok);
        }
    }
}

// the region sum of label m as the finish rounds it (exact statistics)
__device__ __forceinline__ double fuse_sum64(const Job& J, int m)
{
    if (J.dtype == SEG_U16) return __ll2double_rn(J.st_S[m]);
    return round_bins(J.st_S + (long long)m * J.nS, J.nS, J.slot_lo - 150);
}

__global__ void __launch_bounds__(kFuseBlock) k_fuse_match(const Job* jobs, int j)
{
    pdl_enter();
    __shared__ int s_open, s_fused;
    const Job& J = jobs[j];
    if (fuse_idle(J)) return;
    Counters* ctr = J.ctr;
    // labels retired by the previous fusion pass map to themselves again
    const unsigned prev = ld_volatile(&ctr->n_fused);
    for (unsigned k = threadIdx.x; k < prev; k += kFuseBlock) J.fz_to[J.fz_done[k]] = -1;
    const unsigned np = min(ld_volatile(&ctr->n_fpairs), J.fz_cap);
    for (unsigned k = threadIdx.x; k < np; k += kFuseBlock) {
        const unsigned h = J.fz_list[k];
        const unsigned long long key = J.fz_key[h];
        const int a = (int)(key >> 32), b = (int)(key & 0xffffffffu);
        const double na = (double)J.st_n[a], nb = (double)J.st_n[b];
        const double w = __ddiv_rn(__dmul_rn(na, nb), __dadd_rn(na, nb));
        const double d = __dsub_rn(__ddiv_rn(fuse_sum64(J, a), na), __ddiv_rn(fuse_sum64(J, b), nb));
        const double dE = __dsub_rn(__dmul_rn(w, __dmul_rn(d, d)), __dmul_rn(J.fz_lam64, (double)J.fz_cnt[h]));
        J.fz_ab[k] = key;
        J.fz_u[k] = fuse_order(dE);
        J.fz_B[k] = J.fz_cnt[h];
        J.fz_state[k] = dE < 0.0 ? kFuseOpen : kFuseOut;
        J.fz_key[h] = kFuseEmpty;                   // the table is empty again for the next iteration
        J.fz_cnt[h] = 0;
        J.fz_used[a] = 0;
        J.fz_used[b] = 0;
    }
    if (threadIdx.x == 0) {
        s_fused = 0;
        ctr->n_fpairs = 0;
    }
    __syncthreads();
    // greedy matching in rounds; every round takes at least the smallest open pair
    for (unsigned round = 0; round <= np; round++) {
        if (threadIdx.x == 0) s_open = 0;
        for (unsigned k = threadIdx.x; k < np; k += kFuseBlock)
            if (J.fz_state[k] == kFuseOpen) {
                const int a = (int)(J.fz_ab[k] >> 32), b = (int)(J.fz_ab[k] & 0xffffffffu);
                J.fz_best_u[a] = J.fz_best_u[b] = kFuseEmpty;
                J.fz_best_ab[a] = J.fz_best_ab[b] = kFuseEmpty;
            }
        __syncthreads();
        for (unsigned k = threadIdx.x; k < np; k += kFuseBlock)
            if (J.fz_state[k] == kFuseOpen) {
                const int a = (int)(J.fz_ab[k] >> 32), b = (int)(J.fz_ab[k] & 0xffffffffu);
                atomicMin(J.fz_best_u + a, J.fz_u[k]);
                atomicMin(J.fz_best_u + b, J.fz_u[k]);
            }
        __syncthreads();
        for (unsigned k = threadIdx.x; k < np; k += kFuseBlock)
            if (J.fz_state[k] == kFuseOpen) {
                const int a = (int)(J.fz_ab[k] >> 32), b = (int)(J.fz_ab[k] & 0xffffffffu);
                if (J.fz_best_u[a] == J.fz_u[k]) atomicMin(J.fz_best_ab + a, J.fz_ab[k]);
                if (J.fz_best_u[b] == J.fz_u[k]) atomicMin(J.fz_best_ab + b, J.fz_ab[k]);
            }
        __syncthreads();
        for (unsigned k = threadIdx.x; k < np; k += kFuseBlock)
            if (J.fz_state[k] == kFuseOpen) {
                const unsigned long long ab = J.fz_ab[k];
                const int a = (int)(ab >> 32), b = (int)(ab & 0xffffffffu);
                if (J.fz_best_u[a] == J.fz_u[k] && J.fz_best_ab[a] == ab && J.fz_best_u[b] == J.fz_u[k] &&
                    J.fz_best_ab[b] == ab) {
                    J.fz_state[k] = kFuseTaken;
                    J.fz_used[a] = 1;
                    J.fz_used[b] = 1;
                }
            }
        __syncthreads();
        for (unsigned k = threadIdx.x; k < np; k += kFuseBlock)
            if (J.fz_state[k] == kFuseOpen) {
                const int a = (int)(J.fz_ab[k] >> 32), b = (int)(J.fz_ab[k] & 0xffffffffu);
                if (J.fz_used[a] || J.fz_used[b]) J.fz_state[k] = kFuseOut;
                else s_open = 1;
            }
        __syncthreads();
        if (!s_open) break;
        __syncthreads();
    }
    // merge the statistics of each accepted pair into a; b is left empty
    const long long nS = J.dtype == SEG_F32 ? J.nS : 1, nQ = J.dtype == SEG_F32 ? J.nQ : 1;
    for (unsigned k = threadIdx.x; k < np; k += kFuseBlock)
        if (J.fz_state[k] == kFuseTaken) {
            const int a = (int)(J.fz_ab[k] >> 32), b = (int)(J.fz_ab[k] & 0xffffffffu);
            J.st_n[a] += J.st_n[b];
            J.st_n[b] = 0;
            for (long long s = 0; s < nS; s++) {
                J.st_S[a * nS + s] += J.st_S[b * nS + s];
                J.st_S[b * nS + s] = 0;
            }
            for (long long s = 0; s < nQ; s++) {
                J.st_Q[a * nQ + s] += J.st_Q[b * nQ + s];
                J.st_Q[b * nQ + s] = 0;
            }
            J.fz_to[b] = a;
            J.fz_done[atomicAdd(&s_fused, 1)] = b;
            atomicAdd((unsigned long long*)&ctr->perim, (unsigned long long)(-(long long)J.fz_B[k]));
        }
    __syncthreads();
    if (threadIdx.x == 0) ctr->n_fused = (unsigned)s_fused;
}

__global__ void __launch_bounds__(256) k_fuse_relabel(const Job* jobs, int j)
{
    pdl_enter();
    const Job& J = jobs[j];
    if (fuse_idle(J) || ld_volatile(&J.ctr->n_fused) == 0) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < J.npix; i += stride) {
        const int m = J.L[i];
        const int t = J.fz_to[m];
        if (t >= 0) J.L[i] = t;
    }
}

cudaError_t launch_fuse(const Job* jobs, int j, int sms, cudaStream_t s)
{
    cudaError_t e;
    if ((e = launch_stage(k_fuse_pairs, (unsigned)sms * 8, 256, 0, s, jobs, j)) != cudaSuccess) return e;
    if ((e = launch_stage(k_fuse_match, 1u, kFuseBlock, 0, s, jobs, j)) != cudaSuccess) return e;
    return launch_stage(k_fuse_relabel, (unsigned)sms * 8, 256, 0, s, jobs, j);
}

}  // namespace segk
