// Tile kernels of one iteration: particle extraction fused with the energy difference and
// the topology masks, and the Sobolev interaction of Eq. 6 over a cell tile fused with the
// candidate selection.
#include <algorithm>
#include <mutex>

#include "seg_internal.cuh"

namespace segk {

constexpr int kBlock = 256;
constexpr int kLocalCap = 512;               // particles a piecewise-constant tile keeps in shared memory

__device__ __forceinline__ float image_at(const Job& J, long long i)
{
    if (J.dtype == SEG_F32) return __ldg((const float*)J.I + i);
    return (float)__ldg((const unsigned short*)J.I + i);
}

// the image value as an exact fixed-point integer (see fixed_of_f32)
__device__ __forceinline__ long long image_q(const Job& J, long long i)
{
    if (J.dtype == SEG_F32) return fixed_of_f32(__ldg((const float*)J.I + i), J.slot_lo);
    return (long long)__ldg((const unsigned short*)J.I + i);
}

// --------------------------------------------------------------------------
// Tensor-memory-access copies of a tile box into shared memory, completed on an mbarrier.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned phase)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int x, int y, int z, unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// wait for phase 0 of bar, bounded in time and polls; false when it gave up
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar)
{
    WaitBound wb;
    while (true) {
        if (mbar_try_wait(bar, 0)) return true;
        if (wb.expired()) return false;
    }
}

__host__ __device__ __forceinline__ size_t align128(size_t b) { return (b + 127) & ~(size_t)127; }

// Box of a tile as staged in shared memory: origin (ox, oy, oz) and extent (bx, by, bz).
struct StageBox {
    int ox, oy, oz, bx, by, bz;
};

__device__ __forceinline__ StageBox stage_box(const Job& J, const TileBox& b, int h, int hz)
{
    StageBox r;
    const int s = J.cell, sz = J.ndim == 3 ? J.cell : 1;
    r.oy = b.y0 - h;
    r.oz = b.z0 - hz;
    if (J.use_tma) {
        r.ox = (b.x0 - h) & ~7;
        r.bx = J.tma_bx;
        r.by = J.tcy * s + 2 * h;
        r.bz = J.tcz * sz + 2 * hz;
    } else {
        r.ox = b.x0 - h;
        r.bx = b.x1 - b.x0 + 2 * h;
        r.by = b.y1 - b.y0 + 2 * h;
        r.bz = b.z1 - b.z0 + 2 * hz;
    }
    return r;
}

// --------------------------------------------------------------------------
// Extraction: one block per tile of cells, tiles taken in ticket order so that the
// decoupled look-back only waits on tiles that have already started.
template <int NDIM>
__global__ void __launch_bounds__(kBlock, 5) k_extract(Group g)
{
    pdl_enter();
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned s_ticket, s_base;
    __shared__ unsigned s_warp[32];
    const int tid = threadIdx.x;
    if (tid == 0) s_ticket = atomicAdd(g.ticket, 1u);
    __syncthreads();
    const unsigned t = s_ticket;
    const int gj = group_job_of_tile(g, t);
    const Job& J = g.jobs[g.job_ids[gj]];
    const unsigned k = t - g.tile_prefix[gj];
    Counters* ctr = J.ctr;
    if (ld_volatile(&ctr->skip)) return;
    const unsigned tag = ld_volatile(&ctr->iter_tag);

    const TileBox b = tile_box(J, k);
    const int h = J.halo, hz = NDIM == 3 ? J.halo : 0;
    const StageBox sb = stage_box(J, b, h, hz);
    const int bx = sb.bx, by = sb.by, bz = sb.bz;
    const int nbox = bx * by * bz;
    // shared layout (128-byte aligned regions): [fixed-point image (int64)] [image as stored
    // (float32 | uint16)] [labels] [cell starts] [ball deltas]
    const bool stage_img = J.ps_staged != 0;
    const bool use_int = J.ps_int != 0;
    const size_t esz = J.dtype == SEG_F32 ? 4 : 2;
    const bool q32 = J.ps_q32 != 0;
    size_t off_b = 0;
    long long* sQ = (long long*)(smem + off_b);
    if (stage_img && use_int && !q32) off_b = align128(off_b + (size_t)nbox * 8);
    unsigned char* sRaw = smem + off_b;
    float* sI = (float*)sRaw;
    int* sQ32 = (int*)sRaw;   // int32 fixed point, converted in place over the staged image
    if (stage_img) off_b = align128(off_b + (size_t)nbox * (q32 ? 4 : esz));
    int* sL = (int*)(smem + off_b);
    off_b = align128(off_b + (size_t)nbox * 4);
    unsigned* s_cstart = (unsigned*)(smem + off_b);
    // piecewise constant: the tile's particles at tile-local positions (kLocalCap at most)
    const size_t off_loc = align128(off_b + ((size_t)b.ccx * b.ccy * b.ccz + 1) * 4);
    double* s_le = (double*)(smem + off_loc);
    unsigned* s_lidx = (unsigned*)(s_le + kLocalCap);
    int* s_ll = (int*)(s_lidx + kLocalCap);
    int* s_lc = s_ll + kLocalCap;
    __shared__ unsigned s_w1;
    __shared__ __align__(8) unsigned long long s_bar, s_bar_img;
    __shared__ int s_img_fail;
    const bool outside_box = sb.ox < 0 || sb.oy < 0 || sb.oz < 0 || sb.ox + bx > J.W || sb.oy + by > J.H ||
                             sb.oz + bz > J.D;
    // the image copy (2D piecewise smooth) completes on its own mbarrier: counting and the
    // look-back need only the labels, so the image arrives while they run
    const bool img_tma = J.use_tma && stage_img;
    if (tid == 0) s_img_fail = 0;
    if (J.use_tma) {
        // one tensor copy per array; -1 for labels outside the image
        if (tid == 0) {
            mbar_init(&s_bar, 1);
            mbar_expect_tx(&s_bar, (unsigned)nbox * 4u);
            if (img_tma) {
                mbar_init(&s_bar_img, 1);
                mbar_expect_tx(&s_bar_img, (unsigned)(nbox * esz));
            }
            // (fault injection for tests: the first tile's copy is withheld)
            const bool withhold = J.inject == SEG_INJECT_WITHHELD_COPY && k == 0;
            if (NDIM == 3 && !withhold) tma_load_3d(sL, J.tmap_L, sb.ox, sb.oy, sb.oz, &s_bar);
            else if (!withhold) tma_load_2d(sL, J.tmap_L, sb.ox, sb.oy, &s_bar);
        }
        __syncthreads();
        const bool arrived = mbar_wait_bounded(&s_bar);
        // the image only once the labels are in: every tile's labels (which gate the counts
        // and so every tile's look-back) do not share the DRAM burst with the images
        if (tid == 0 && img_tma && arrived) tma_load_2d(sRaw, J.tmap_I, sb.ox, sb.oy, &s_bar_img);
        if (__syncthreads_or(!arrived)) {   // the whole block leaves together, its tile empty
            if (tid == 0) {
                atomicExch(&ctr->error, SEG_ETIMEOUT);
                atomicExch(&ctr->skip, 1);       // the later stages of the iteration do nothing
                J.tile_start[k] = 0;
                J.tile_count[k] = 0;
            }
            mbar_wait_bounded(&s_bar);       // a second bounded wait for the copies in flight
            if (tid == 0 && img_tma && arrived) mbar_wait_bounded(&s_bar_img);
            return;
        }
        if (outside_box) {
            for (int row = tid >> 5; row < by * bz; row += blockDim.x >> 5)
            for (int lx = tid & 31; lx < bx; lx += 32) {
                const int ly = row % by, lz = row / by;
                const int x = sb.ox + lx, y = sb.oy + ly, z = sb.oz + lz;
                if (!(x >= 0 && x < J.W && y >= 0 && y < J.H && z >= 0 && z < J.D)) sL[row * bx + lx] = -1;
            }
        }
        __syncthreads();
    }

    // row-by-row staging when the rows cannot be copied by tensor copies: labels (and, for the
    // 2D piecewise-smooth model, the image) with halo; -1 outside; one warp per row of the box
    const int nrows = J.use_tma ? 0 : by * bz;
    for (int row = tid >> 5; row < nrows; row += blockDim.x >> 5)
    for (int lx = tid & 31; lx < bx; lx += 32) {
        const int ly = row % by, lz = row / by;
        const int i = row * bx + lx;
        int x = sb.ox + lx, y = sb.oy + ly, z = sb.oz + lz;
        int lab = -1;
        float val = 0.0f;
        long long qval = 0;
        if (x >= 0 && x < J.W && y >= 0 && y < J.H && z >= 0 && z < J.D) {
            long long gi = ((long long)z * J.H + y) * J.W + x;
            lab = __ldg(J.L + gi);
            if (stage_img) {
                if (use_int) qval = image_q(J, gi);
                else val = image_at(J, gi);
            }
        }
        sL[i] = lab;
        if (stage_img) {
            if (use_int && q32) sQ32[i] = (int)qval;
            else if (use_int) sQ[i] = qval;
            else sI[i] = val;
        }
    }
    __syncthreads();

    const int s = J.cell, sz = NDIM == 3 ? J.cell : 1;
    const int cellvol = s * s * sz;
    const int ncell = b.ccx * b.ccy * b.ccz;
    const int tile_q = ncell * cellvol;
    const int chunk = (tile_q + blockDim.x - 1) / blockDim.x;
    const int q0 = min(tid * chunk, tile_q), q1 = min(q0 + chunk, tile_q);

    // cell-major walk: (cell lx, ly, lz of the tile; pixel rx, ry, rz of the cell), the
    // start decoded once per thread, then advanced like an odometer
    struct Walk { int lx, ly, lz, rx, ry, rz; };
    auto walk_start = [&](int q) -> Walk {
        Walk w;
        int kc = q / cellvol, r = q - kc * cellvol;
        w.lx = kc % b.ccx; w.ly = (kc / b.ccx) % b.ccy; w.lz = kc / (b.ccx * b.ccy);
        w.rx = r % s; w.ry = (r / s) % s; w.rz = r / (s * s);
        return w;
    };
    auto walk_next = [&](Walk& w) {
        if (++w.rx < s) return;
        w.rx = 0;
        if (++w.ry < s) return;
        w.ry = 0;
        if (++w.rz < sz) return;
        w.rz = 0;
        if (++w.lx < b.ccx) return;
        w.lx = 0;
        if (++w.ly < b.ccy) return;
        w.ly = 0;
        ++w.lz;
    };
    auto walk_pixel = [&](const Walk& w, int& x, int& y, int& z) -> bool {
        x = (b.cx0 + w.lx) * s + w.rx;
        y = (b.cy0 + w.ly) * s + w.ry;
        z = (b.cz0 + w.lz) * sz + w.rz;
        return x < J.W && y < J.H && z < J.D;
    };
    auto sidx = [&](int x, int y, int z) -> int {
        return ((z - sb.oz) * by + (y - sb.oy)) * bx + (x - sb.ox);
    };
    // distinct neighbour labels different from the own label, ascending: the neighbours are
    // sorted in registers by an odd-even transposition network, then repeats are dropped;
    // labs[j] is INT_MAX for j >= n
    constexpr int NN = NDIM == 3 ? 6 : 4;
    auto particles_at = [&](int x, int y, int z, int (&labs)[NN]) -> int {
        const int si = sidx(x, y, z);
        const int own = sL[si];
        int v[NN];
        v[0] = sL[si - 1];
        v[1] = sL[si + 1];
        v[2] = sL[si - bx];
        v[3] = sL[si + bx];
        if (NDIM == 3) { v[NDIM == 3 ? 4 : 0] = sL[si - bx * by]; v[NDIM == 3 ? 5 : 1] = sL[si + bx * by]; }
        // interior pixels (every neighbour holds the own label or lies outside) hold no particle
        bool any = false;
#pragma unroll
        for (int j = 0; j < NN; j++) {
            if (v[j] < 0 || v[j] == own) v[j] = 0x7fffffff;
            any |= v[j] != 0x7fffffff;
        }
        if (!any) return 0;
#pragma unroll
        for (int r = 0; r < NN; r++)
#pragma unroll
            for (int j = r & 1; j + 1 < NN; j += 2) {
                const int a = min(v[j], v[j + 1]), b = max(v[j], v[j + 1]);
                v[j] = a;
                v[j + 1] = b;
            }
        int n = 0;
#pragma unroll
        for (int j = 0; j < NN; j++) {
            const bool keep = v[j] != 0x7fffffff && (j == 0 || v[j] != v[j > 0 ? j - 1 : 0]);
            labs[j] = 0x7fffffff;
            if (keep) n++;
        }
        // compact the kept values to the front (static indices only)
        int w = 0;
#pragma unroll
        for (int j = 0; j < NN; j++) {
            const bool keep = v[j] != 0x7fffffff && (j == 0 || v[j] != v[j > 0 ? j - 1 : 0]);
#pragma unroll
            for (int t = 0; t < NN; t++)
                if (keep && t == w) labs[t] = v[j];
            if (keep) w++;
        }
        return n;
    };
    // the topology masks of a particle: bit k of the low (high) word is set when the k-th of the
    // 8 (26) neighbours, (dz, dy, dx) ascending without the centre, holds own (c); -1 outside
    auto nb_masks = [&](int si, int own, int c) -> unsigned long long {
        unsigned ml = 0, mc = 0;
        int kb = 0;
#pragma unroll
        for (int dz = -(NDIM == 3 ? 1 : 0); dz <= (NDIM == 3 ? 1 : 0); dz++)
#pragma unroll
            for (int dy = -1; dy <= 1; dy++)
#pragma unroll
                for (int dx = -1; dx <= 1; dx++) {
                    if (dz == 0 && dy == 0 && dx == 0) continue;
                    const int v = sL[si + (dz * by + dy) * bx + dx];
                    ml |= (unsigned)(v == own) << kb;
                    mc |= (unsigned)(v == c) << kb;
                    kb++;
                }
        return (unsigned long long)ml | ((unsigned long long)mc << 32);
    };
    // change of the number of unlike neighbour pairs when the pixel goes from own to c
    auto delta_p = [&](int si, int own, int c) -> int {
        int nb[NN];
        nb[0] = sL[si - 1]; nb[1] = sL[si + 1]; nb[2] = sL[si - bx]; nb[3] = sL[si + bx];
        if (NDIM == 3) { nb[NDIM == 3 ? 4 : 0] = sL[si - bx * by]; nb[NDIM == 3 ? 5 : 1] = sL[si + bx * by]; }
        int dP = 0;
#pragma unroll
        for (int u = 0; u < NN; u++) {
            const int m = nb[u];
            if (m >= 0) dP += (int)(m != c) - (int)(m != own);
        }
        return dP;
    };

    // count; a thread whose chunk has at most 32 pixels remembers which of them hold particles
    unsigned cnt = 0, busy = 0;
    const bool use_mask = q1 - q0 <= 32;
    {
        Walk w = walk_start(q0);
        for (int q = q0; q < q1; q++, walk_next(w)) {
            int x, y, z, labs[NN];
            if (!walk_pixel(w, x, y, z)) continue;
            const int n = particles_at(x, y, z, labs);
            cnt += n;
            if (n) busy |= 1u << ((q - q0) & 31);
        }
    }
    unsigned total;
    unsigned off = block_excl_scan(cnt, s_warp, total);

    // Piecewise-constant tiles of at most kLocalCap particles: the particles are emitted into
    // shared memory at their tile-local positions and their FP64 energy differences formed there
    // while warp 0 resolves the tile's offset (the look-back below); warps 1.. do so for their
    // pixels at once, warp 0 for its own after the look-back. Cell starts are tile-local anyway.
    const bool local = J.model == SEG_PC && total <= (unsigned)kLocalCap;
    auto emit_local = [&]() {
        unsigned ol = off;
        Walk wl = walk_start(q0);
        for (int q = q0; q < q1; q++, walk_next(wl)) {
            int x, y, z, labs[NN];
            if (wl.rx == 0 && wl.ry == 0 && wl.rz == 0) s_cstart[(wl.lz * b.ccy + wl.ly) * b.ccx + wl.lx] = ol;
            if (use_mask && !((busy >> ((q - q0) & 31)) & 1u)) continue;
            if (!walk_pixel(wl, x, y, z)) continue;
            const int n = particles_at(x, y, z, labs);
            if (n == 0) continue;
            const unsigned gi = (unsigned)(((long long)z * J.H + y) * J.W + x);
            const int own = sL[sidx(x, y, z)];
#pragma unroll
            for (int j = 0; j < NN; j++) {
                if (j >= n) break;
                s_lidx[ol] = gi;
                s_ll[ol] = own;
                s_lc[ol] = labs[j];
                ol++;
            }
        }
    };
    auto energy_local = [&](unsigned i) {
        const unsigned gi = s_lidx[i];
        const int own = s_ll[i], c = s_lc[i];
        int x, y, z;
        pix_coords(J, gi, x, y, z);
        s_le[i] = with_length64(J, data_pc64(J, (double)image_at(J, gi), own, c), delta_p(sidx(x, y, z), own, c));
    };

    // decoupled look-back over the tiles of this job: warp 0 inspects 32 predecessors per
    // round trip, nearest first, and stops at the first one that knows its inclusive prefix
    if (tid < 32) {
        const int lane = tid;
        const unsigned long long ep = (unsigned long long)(tag & 0x3fffffffu) << 34;
        const unsigned long long emask = ~((1ull << 34) - 1);
        unsigned excl = 0;
        if (lane == 0) atomicExch(J.tile_word + k, ep | ((k == 0 ? 2ull : 1ull) << 32) | total);
        if (k > 0) {
            // each lane reads 8 consecutive predecessors (lane 0 the nearest), 256 per round
            // trip. The ready run nearest to the tile is consumed up to the first inclusive
            // prefix; a predecessor that has published nothing yet stops the run, and the next
            // round starts there (progress without waiting for the whole window).
            constexpr int kPer = 8;
            long long win_end = (long long)k - 1;
            WaitBound wb;
            while (true) {
                unsigned st[kPer], val[kPer];
#pragma unroll
                for (int j = 0; j < kPer; j++) {
                    const long long i = win_end - (long long)lane * kPer - j;
                    st[j] = 2;                      // before tile 0: an inclusive prefix of 0
                    val[j] = 0;
                    if (i >= 0) {
                        const unsigned long long w = ld_volatile(J.tile_word + i);
                        st[j] = (w & emask) == ep ? (unsigned)((w >> 32) & 3u) : 0u;
                        val[j] = (unsigned)w;
                    }
                }
                int f2 = kPer, f0 = kPer;           // first inclusive, first unpublished in the lane
#pragma unroll
                for (int j = kPer - 1; j >= 0; j--) {
                    if (st[j] == 2) f2 = j;
                    if (st[j] == 0) f0 = j;
                }
                const unsigned m2 = __ballot_sync(0xffffffffu, f2 < kPer);
                const unsigned m0 = __ballot_sync(0xffffffffu, f0 < kPer);
                const int l2 = m2 ? __ffs(m2) - 1 : 32, l0 = m0 ? __ffs(m0) - 1 : 32;
                const int A = l2 < 32 ? l2 * kPer + __shfl_sync(0xffffffffu, f2, l2 & 31) : 32 * kPer;
                const int B = l0 < 32 ? l0 * kPer + __shfl_sync(0xffffffffu, f0, l0 & 31) : 32 * kPer;
                const bool done = A < B;            // an inclusive prefix before any gap
                const int limit = done ? A + 1 : B; // entries [0, limit) are summed this round
                unsigned part = 0;
#pragma unroll
                for (int j = 0; j < kPer; j++)
                    if (lane * kPer + j < limit) part += val[j];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                excl += part;
                if (done) break;
                win_end -= limit;
                if (limit == 0) {                   // the nearest remaining predecessor is not ready
                    // lane 0 decides for the warp, so that its lanes leave together
                    if (__shfl_sync(0xffffffffu, (int)wb.expired(), 0)) {
                        if (lane == 0) {
                            atomicExch(&ctr->error, SEG_ETIMEOUT);
                            atomicExch(&ctr->skip, 1);
                        }
                        break;
                    }
                    __nanosleep(32);
                }
            }
            __threadfence();
            if (lane == 0) atomicExch(J.tile_word + k, ep | (2ull << 32) | (excl + total));
        }
        if (lane == 0) {
            s_base = excl;
            J.tile_start[k] = excl;
            J.tile_count[k] = total;
            if (k == (unsigned)J.ntiles - 1) {
                ctr->n_particles = excl + total;
                if ((long long)excl + total > J.pcap) atomicMax(&ctr->need, excl + total);
            }
        }
    } else if (local) {
        // meanwhile warps 1.. emit their pixels' particles and form their energies locally
        emit_local();
        if (tid == 32) s_w1 = off;                 // warp 1's first local position
        asm volatile("bar.sync 1, %0;" ::"r"((int)blockDim.x - 32) : "memory");
        for (unsigned i = s_w1 + (tid - 32); i < total; i += blockDim.x - 32) energy_local(i);
    } else if (img_tma) {
        // meanwhile the other warps turn the staged image (once its copy has landed) into exact
        // fixed-point values for the piecewise-smooth ball sums
        const bool landed = mbar_wait_bounded(&s_bar_img);
        if (!landed) s_img_fail = 1;
        if (landed && use_int) {
            const int nw = (blockDim.x >> 5) - 1;
            for (int row = (tid >> 5) - 1; row < by * bz; row += nw)
            for (int lx = tid & 31; lx < bx; lx += 32) {
                const int ly = row % by, lz = row / by;
                const int i = row * bx + lx;
                const int x = sb.ox + lx, y = sb.oy + ly, z = sb.oz + lz;
                const bool in = x >= 0 && x < J.W && y >= 0 && y < J.H && z >= 0 && z < J.D;
                long long q = 0;
                if (in) q = J.dtype == SEG_F32 ? fixed_of_f32(sI[i], J.slot_lo)
                                               : (long long)((const unsigned short*)sRaw)[i];
                if (q32) {
                    if (J.dtype == SEG_F32) sQ32[i] = (int)q;   // same element, same size: in place
                } else {
                    sQ[i] = q;
                }
            }
        }
    }
    __syncthreads();
    if (s_img_fail) {                            // the image copy did not land in time
        if (tid == 0) {
            atomicExch(&ctr->error, SEG_ETIMEOUT);
            atomicExch(&ctr->skip, 1);
            J.tile_count[k] = 0;
        }
        mbar_wait_bounded(&s_bar_img);
        return;
    }
    const unsigned base = s_base;
    const bool fits = (long long)base + total <= J.pcap;

    if (local) {
        // warp 0's own particles, then every particle to global memory at base + its position
        if (tid < 32) {
            emit_local();
            __syncwarp();
            const unsigned w1 = blockDim.x > 32 ? s_w1 : total;
            for (unsigned i = tid; i < w1; i += 32) energy_local(i);
        }
        if (tid == 0) s_cstart[ncell] = total;
        __syncthreads();
        if (fits) {
            for (unsigned i = tid; i < total; i += blockDim.x) {
                const unsigned o2 = base + i, gi = s_lidx[i];
                if (i == 0 || s_lidx[i - 1] != gi) J.pmap[gi] = ((unsigned long long)tag << 32) | o2;
                J.p_idx[o2] = gi;
                J.p_l[o2] = s_ll[i];
                J.p_c[o2] = s_lc[i];
                J.p_flags[o2] = 0;
                store_dE(J, o2, s_le[i]);
                int x, y, z;
                pix_coords(J, gi, x, y, z);
                J.p_nbm[o2] = nb_masks(sidx(x, y, z), s_ll[i], s_lc[i]);
            }
        }
        for (int kc = tid; kc < ncell; kc += blockDim.x) {
            int lx = kc % b.ccx, ly = (kc / b.ccx) % b.ccy, lz = kc / (b.ccx * b.ccy);
            long long cid = ((long long)(b.cz0 + lz) * J.ncy + (b.cy0 + ly)) * J.ncx + (b.cx0 + lx);
            J.cell_start[cid] = base + s_cstart[kc];
            J.cell_count[cid] = s_cstart[kc + 1] - s_cstart[kc];
        }
        return;
    }

    // emit particles
    unsigned o = base + off;
    Walk wk = walk_start(q0);
    for (int q = q0; q < q1; q++, walk_next(wk)) {
        int x, y, z, labs[NN];
        if (wk.rx == 0 && wk.ry == 0 && wk.rz == 0) s_cstart[(wk.lz * b.ccy + wk.ly) * b.ccx + wk.lx] = o - base;
        if (use_mask && !((busy >> ((q - q0) & 31)) & 1u)) continue;
        if (!walk_pixel(wk, x, y, z)) continue;
        int n = particles_at(x, y, z, labs);
        if (n == 0) continue;
        const long long gi = ((long long)z * J.H + y) * J.W + x;
        const int si = sidx(x, y, z);
        const int own = sL[si];
        if (fits) J.pmap[gi] = ((unsigned long long)tag << 32) | o;
#pragma unroll
        for (int j = 0; j < NN; j++) {
            if (j >= n) break;
            const int c = labs[j];
            if (fits) {
                J.p_idx[o] = (unsigned)gi;
                J.p_l[o] = own;
                J.p_c[o] = c;
                J.p_flags[o] = 0;
            }
            o++;
        }
    }
    __syncthreads();
    if (tid == 0) s_cstart[ncell] = total;
    __syncthreads();
    for (int kc = tid; kc < ncell; kc += blockDim.x) {
        int lx = kc % b.ccx, ly = (kc / b.ccx) % b.ccy, lz = kc / (b.ccx * b.ccy);
        long long cid = ((long long)(b.cz0 + lz) * J.ncy + (b.cy0 + ly)) * J.ncx + (b.cx0 + lx);
        J.cell_start[cid] = base + s_cstart[kc];
        J.cell_count[cid] = s_cstart[kc + 1] - s_cstart[kc];
    }
    if (J.model == SEG_PC && fits) {
        // piecewise constant: the FP64 energy difference in the order of its definition, one
        // particle per thread over the tile's dense range (the FP64 pipe is occupied per warp
        // instruction, so the emitting threads' uneven particle counts would waste it)
        for (unsigned o2 = base + tid; o2 < base + total; o2 += blockDim.x) {
            const unsigned gi = J.p_idx[o2];
            const int own = J.p_l[o2], c = J.p_c[o2];
            int x, y, z;
            pix_coords(J, gi, x, y, z);
            const int si = sidx(x, y, z);
            J.p_nbm[o2] = nb_masks(si, own, c);
            const double data = data_pc64(J, (double)image_at(J, gi), own, c);
            store_dE(J, o2, with_length64(J, data, delta_p(si, own, c)));
        }
        return;
    }
    // the other models: the topology masks in a pass of their own, one particle per thread
    if (fits)
        for (unsigned o2 = base + tid; o2 < base + total; o2 += blockDim.x) {
            int x, y, z;
            pix_coords(J, J.p_idx[o2], x, y, z);
            J.p_nbm[o2] = nb_masks(sidx(x, y, z), J.p_l[o2], J.p_c[o2]);
        }
    if (J.model == SEG_PC_DECONV && fits) {
        // deconvolving model: one particle per thread; G at the pixel (the last separable pass,
        // FP64), then the FP64 energy difference
        for (unsigned o2 = base + tid; o2 < base + total; o2 += blockDim.x) {
            const unsigned gi = J.p_idx[o2];
            const int own = J.p_l[o2], c = J.p_c[o2];
            int x, y, z;
            pix_coords(J, gi, x, y, z);
            const double G = deconv_G(J, gi, y, z);
            J.dc_G[gi] = G;                         // for the FP64 recompute (same value per particle)
            const double data = deconv_data64(J, G, x, y, z, own, c);
            store_dE(J, o2, with_length64(J, data, delta_p(sidx(x, y, z), own, c)));
        }
        return;
    }
    if (!is_ps(J.model) || !fits) return;

    // piecewise-smooth energy: one particle per thread over the dense range of this tile's
    // particles, so every thread runs the same ball loop
    int* s_delta = (int*)(s_cstart + ncell + 1);   // ball offsets as staged-box index deltas
    if (stage_img) {
        for (int u = tid; u < J.ps_n; u += blockDim.x) {
            const int4 d = __ldg(J.ps_off + u);
            s_delta[u] = d.y * bx + d.z;
        }
    }
    __syncthreads();
    if (stage_img && use_int) {
        // a quad of lanes per particle, each lane every fourth ball offset; the loads of an
        // offset do not depend on the label test, so consecutive offsets overlap
        auto quad_pass = [&](const auto* Q) {
            const int lane4 = tid & 3;
            const unsigned nquad = blockDim.x >> 2;
            for (unsigned lp0 = 0; lp0 < total; lp0 += nquad) {
                const unsigned lp = lp0 + (tid >> 2);
                const bool act = lp < total;
                const unsigned o2 = base + (act ? lp : 0);
                int own = -2, c = -2, si = 0;
                if (act) {
                    const unsigned gi = J.p_idx[o2];
                    own = J.p_l[o2];
                    c = J.p_c[o2];
                    int x, y, z;
                    pix_coords(J, gi, x, y, z);
                    si = sidx(x, y, z);
                }
                long long isc = 0, isl = 0;
                int cc = 0, cl = 0;
                if (act) {
#pragma unroll 4
                    for (int u = lane4; u < J.ps_n; u += 4) {
                        const int sj = si + s_delta[u];
                        const int m = sL[sj];
                        const long long q = Q[sj];
                        const bool inc = m == c, inl = m == own;
                        isc += inc ? q : 0;
                        isl += inl ? q : 0;
                        cc += inc;
                        cl += inl;
                    }
                }
#pragma unroll
                for (int w2 = 1; w2 < 4; w2 <<= 1) {
                    isc += __shfl_xor_sync(0xffffffffu, isc, w2);
                    isl += __shfl_xor_sync(0xffffffffu, isl, w2);
                    cc += __shfl_xor_sync(0xffffffffu, cc, w2);
                    cl += __shfl_xor_sync(0xffffffffu, cl, w2);
                }
                if (act && lane4 == 0) {
                    J.p_qc[o2] = isc;
                    J.p_ql[o2] = isl;
                    J.p_nc[o2] = cc;
                    J.p_nl[o2] = cl;
                }
            }
            // the FP64 energy differences from the exact sums, one particle per thread (the FP64
            // pipe is occupied per warp instruction, so the quads' single lanes would waste it)
            __syncthreads();
            for (unsigned o2 = base + tid; o2 < base + total; o2 += blockDim.x) {
                const unsigned gi = J.p_idx[o2];
                const int own = J.p_l[o2], c = J.p_c[o2];
                int x, y, z;
                pix_coords(J, gi, x, y, z);
                const int si = sidx(x, y, z);
                const double v = __dmul_rn((double)Q[si], J.unit64);   // the pixel value, exactly
                const int cc = J.p_nc[o2], cl = J.p_nl[o2];
                double sc = 0.0, sl = 0.0;
                if (J.ps_exact64) {
                    // every partial sum of the FP64 ball loop is exact: the integer sums are its sums
                    sc = __dmul_rn((double)J.p_qc[o2], J.unit64);
                    sl = __dmul_rn((double)J.p_ql[o2], J.unit64);
                } else {
                    // the FP64 loop over the ball in row-major order
                    for (int u = 0; u < J.ps_n; u++) {
                        const int sj = si + s_delta[u];
                        const int m = sL[sj];
                        if (m == c) sc = __dadd_rn(sc, __dmul_rn((double)Q[sj], J.unit64));
                        else if (m == own) sl = __dadd_rn(sl, __dmul_rn((double)Q[sj], J.unit64));
                    }
                }
                const double data = data_ps64(J, v, sc, cc, sl, cl);
                store_dE(J, o2, with_length64(J, data, delta_p(si, own, c)));
            }
        };
        if (q32) quad_pass(sQ32);
        else quad_pass(sQ);
        return;
    }
    // one particle per thread: exact fixed-point ball sums where they are exact in FP64, the FP64
    // row-major ball loop where they are not
    for (unsigned o2 = base + tid; o2 < base + total; o2 += blockDim.x) {
        const unsigned gi = J.p_idx[o2];
        const int own = J.p_l[o2], c = J.p_c[o2];
        int x, y, z;
        pix_coords(J, gi, x, y, z);
        const int si = sidx(x, y, z);
        const double v = image64(J, gi);
        long long isc = 0, isl = 0;
        double fsc = 0.0, fsl = 0.0;
        int cc = 0, cl = 0;
        for (int u = 0; u < J.ps_n; u++) {
            int m;
            double f = 0.0;
            long long qy = 0;
            if (stage_img) {
                const int sj = si + s_delta[u];     // staged float32 image (no fixed point here)
                m = sL[sj];
                if (m != c && m != own) continue;
                f = (double)sI[sj];
            } else {
                const int4 d = __ldg(J.ps_off + u);
                const int yx = x + d.z, yy = y + d.y, yz = z + d.x;
                if (yx < 0 || yx >= J.W || yy < 0 || yy >= J.H || yz < 0 || yz >= J.D) continue;
                const long long gj2 = ((long long)yz * J.H + yy) * J.W + yx;
                m = __ldg(J.L + gj2);
                if (m != c && m != own) continue;
                if (use_int) qy = image_q(J, gj2);
                if (!J.ps_exact64) f = image64(J, gj2);
            }
            if (m == c) {
                isc += qy;
                fsc = __dadd_rn(fsc, f);
                cc++;
            } else {
                isl += qy;
                fsl = __dadd_rn(fsl, f);
                cl++;
            }
        }
        double sc = fsc, sl = fsl;
        if (J.ps_exact64) {
            sc = __dmul_rn((double)isc, J.unit64);
            sl = __dmul_rn((double)isl, J.unit64);
        }
        const double data = data_ps64(J, v, sc, cc, sl, cl);
        store_dE(J, o2, with_length64(J, data, delta_p(si, own, c)));
    }
}

size_t extract_smem_bytes(const Job& J)
{
    int s = J.cell, sz = J.ndim == 3 ? J.cell : 1;
    int h = J.halo, hz = J.ndim == 3 ? J.halo : 0;
    long long bx = J.use_tma ? J.tma_bx : (long long)J.tcx * s + 2 * h;
    long long by = (long long)J.tcy * s + 2 * h, bz = (long long)J.tcz * sz + 2 * hz;
    long long nbox = bx * by * bz;
    size_t esz = J.dtype == SEG_F32 ? 4 : 2;
    size_t b = 0;
    if (J.ps_staged && J.ps_int && !J.ps_q32) b = align128(b + nbox * 8);
    if (J.ps_staged) b = align128(b + nbox * (J.ps_q32 ? 4 : esz));
    b = align128(b + nbox * 4);
    long long ncell = (long long)J.tcx * J.tcy * J.tcz;
    long long deltas = J.ps_staged ? J.ps_n : 0;
    size_t local = 0;
    if (J.model == SEG_PC) {        // the tile-local particles: energy f64, pixel u32, l, c i32
        b = align128(b + (size_t)(ncell + 1) * 4);
        local = (size_t)kLocalCap * 20;
        return b + local + 128;
    }
    return b + (size_t)((ncell + 1) * 4 + deltas * 4) + 128;
}

cudaError_t launch_extract(const Group& g, int ndim, size_t smem, cudaStream_t st)
{
    if (g.total_tiles == 0) return cudaSuccess;
    if (ndim == 2) return launch_stage(k_extract<2>, g.total_tiles, kBlock, smem, st, g);
    return launch_stage(k_extract<3>, g.total_tiles, kBlock, smem, st, g);
}

// --------------------------------------------------------------------------
// Sobolev interaction, Eq. 6: g_p = (1/|Q_p|) sum_{Q_p} K(d) dE_q - (1/|Q'_p|) sum_{Q'_p} K(d) dE_q,
// Q_p = {q : d < E/2, l_q = l_p}, Q'_p = {q : d < E/2, c_q = l_p}; empty sets give 0.
//
// One block per tile. The particles within rr = floor(sqrt(r2max)) pixels of the tile (found
// through the tile's cells and one ring of cells around them, one warp per cell) are staged
// in shared memory sorted by pixel, with a per-pixel offset table over the box "tile grown
// by rr" (not clipped to the image: pixels outside hold no particles). A particle then visits
// only the rows of its interaction ball: for every (dy, dz) with dy^2 + dz^2 <= r2max the
// particles of the pixel run [x - rx, x + rx], rx = floor(sqrt(r2max - dy^2 - dz^2)), are one
// contiguous range of the staged arrays, and every one of them is a partner by construction.
// Tiles whose box or particle count does not fit read global memory instead.
constexpr int kRecCap = 2048;      // staged particles per tile
constexpr int kBoxCap = 16384;     // staged pixel box per tile
constexpr int kMaxRows = 256;      // (dy, dz) rows of the interaction ball
constexpr int kMaxRing = 4096;     // ring cells per tile

struct Rec {
    float dh, dl;                  // the energy difference as a float pair
    int l, c;
};

__host__ __device__ __forceinline__ int isqrt_floor(int v)
{
    int r = 0;
    while ((r + 1) * (r + 1) <= v) r++;
    return r;
}

// staged pixel box of a full tile (an upper bound for every tile of the job)
__host__ __device__ __forceinline__ long long sob_box_cap(const Job& J)
{
    const int rr = isqrt_floor(J.r2max);
    long long bx = (long long)J.tcx * J.cell + 2 * rr, by = (long long)J.tcy * J.cell + 2 * rr;
    long long bz = J.ndim == 3 ? (long long)J.tcz * J.cell + 2 * rr : 1;
    return bx * by * bz;
}

__host__ __device__ __forceinline__ long long sob_ring_cells(const Job& J)
{
    return (long long)(J.tcx + 2) * (J.tcy + 2) * (J.ndim == 3 ? J.tcz + 2 : J.tcz);
}

__host__ __device__ __forceinline__ bool sob_can_stage(const Job& J)
{
    const int rr = isqrt_floor(J.r2max);
    const int w = 2 * rr + 1;
    return J.r2max < 256 && (J.ndim == 3 ? w * w : w) <= kMaxRows && sob_box_cap(J) <= kBoxCap &&
           sob_ring_cells(J) <= kMaxRing;
}

// shared-memory layout: records | x | pixel offsets (u16) | ring-cell starts, counts, prefix
struct SobLayout {
    size_t x, off, cs, cn, eoff, total;
};

__host__ __device__ __forceinline__ SobLayout sob_layout(const Job& J)
{
    SobLayout L;
    const bool st = sob_can_stage(J);
    const size_t ring = st ? (size_t)((sob_ring_cells(J) + 4) & ~3LL) * 4 : 0;
    L.x = st ? (size_t)kRecCap * sizeof(Rec) : 0;
    L.off = L.x + (st ? (size_t)kRecCap * 2 : 0);
    L.cs = L.off + (st ? (size_t)((sob_box_cap(J) + 8) & ~7LL) * 2 : 0);
    L.cn = L.cs + ring;
    L.eoff = L.cn + ring;
    L.total = L.eoff + ring;
    return L;
}

// the ring cell holding ring particle i (the last cell whose prefix is <= i)
__device__ __forceinline__ int ring_cell_of(const unsigned* s_eoff, int ne, unsigned i)
{
    int lo = 0, hi = ne - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_eoff[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The sums of Eq. 6 for particle (x, y, z; label lp) from global memory (tiles that are not
// staged): compensated sums of exact products, and sum |K dE| per set for the bound
template <int NDIM>
__device__ __forceinline__ void sobolev_sums(const Job& J, int lp, int x, int y, int z, int r2max, DotAcc& A,
                                             DotAcc& B, float& aA, float& aB, int& nA, int& nB)
{
    const int pcx = (int)fdiv((unsigned)x, J.fd_cell), pcy = (int)fdiv((unsigned)y, J.fd_cell);
    const int pcz = NDIM == 3 ? (int)fdiv((unsigned)z, J.fd_cell) : z;
    for (int cz = max(pcz - (NDIM == 3), 0); cz <= min(pcz + (NDIM == 3), J.ncz - 1); cz++)
        for (int cy = max(pcy - 1, 0); cy <= min(pcy + 1, J.ncy - 1); cy++)
            for (int cx = max(pcx - 1, 0); cx <= min(pcx + 1, J.ncx - 1); cx++) {
                const long long cid = ((long long)cz * J.ncy + cy) * J.ncx + cx;
                const unsigned c0 = J.cell_start[cid], c1 = c0 + J.cell_count[cid];
                for (unsigned j = c0; j < c1; j++) {
                    int qx, qy, qz;
                    pix_coords(J, J.p_idx[j], qx, qy, qz);
                    const int d2 = (qx - x) * (qx - x) + (qy - y) * (qy - y) + (qz - z) * (qz - z);
                    if (d2 > r2max) continue;
                    const int ql = J.p_l[j], qc = J.p_c[j];
                    if (ql != lp && qc != lp) continue;
                    const float Kh = __ldg(J.klut + d2), Kl = __ldg(J.klut_lo + d2);
                    if (ql == lp) {
                        aA += fabsf(A.add(Kh, Kl, J.p_dE[j], J.p_dEl[j]));
                        nA++;
                    } else {
                        aB += fabsf(B.add(Kh, Kl, J.p_dE[j], J.p_dEl[j]));
                        nB++;
                    }
                }
            }
}

template <int NDIM>
__global__ void __launch_bounds__(kBlock, NDIM == 2 ? 4 : 3) k_sobolev(Group g, BatchCtl* bc)
{
    pdl_enter();
    if (blockIdx.x == 0 && threadIdx.x == 0) {       // the selection's control words
        bc->err = 0;
        bc->rounds_done = 0;
    }
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned s_warp[32];
    __shared__ float2 s_klut[256];               // K(sqrt(d2)) as a float pair
    __shared__ unsigned s_dmax;                  // largest |dE| staged (float bits)
    __shared__ int s_rdelta[kMaxRows];           // row offset in the pixel box
    __shared__ unsigned short s_rinfo[kMaxRows]; // rx | dy^2 + dz^2 << 8
    __shared__ int s_nrows;
    __shared__ unsigned s_osc;
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned t = blockIdx.x;
    const int gj = group_job_of_tile(g, t);
    const Job& J = g.jobs[g.job_ids[gj]];
    const unsigned k = t - g.tile_prefix[gj];
    Counters* ctr = J.ctr;
    const unsigned skip = ld_volatile(&ctr->skip) | ld_volatile(&ctr->need);
    const unsigned pstart = J.tile_start[k], pcount = J.tile_count[k];
    const int mode = ld_volatile(&ctr->mode);
    if (skip || pcount == 0 || mode == SEG_SOBOLEV_GLOBAL) return;   // E = |Gamma|: k_sobolev_global
    __shared__ unsigned s_slot0;
    // Candidates (Region Competition's selection): the best particle of a pixel (smallest key,
    // then c) is a candidate when its key could be negative and the move is admissible. The
    // pixel's first particle decides for the pixel; the block's candidates of one pass take one
    // contiguous range of slots (a block scan, one counter update), so that candidate indices
    // follow the tiles. Every thread of the block calls this once per pass.
    auto select_append = [&](bool first, int adm, unsigned pfirst, unsigned best, unsigned gi, double bk, float bg,
                             float be, bool exact) {
        unsigned n_adm;
        const unsigned rank = block_excl_scan(adm ? 1u : 0u, s_warp, n_adm);
        if (tid == 0) s_slot0 = n_adm ? atomicAdd(&ctr->n_cand, n_adm) : 0u;
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
                if (!exact && fabsf(bg) <= be) queue_fixup(J, (unsigned)slot, best);   // sign uncertain
            }
            J.pix_cand[pfirst] = slot;
        }
        __syncthreads();                       // s_warp and s_slot0 are reused by the next pass
    };
    if (mode == SEG_L2) {
        // L2: the gradient is the energy difference, the key its FP64 value (exact)
        for (unsigned i0 = 0; i0 < pcount; i0 += blockDim.x) {       // uniform over the block
            const unsigned i = i0 + tid;
            const unsigned p = pstart + i;
            bool first = false;
            int adm = 0, bc_ = 0;
            unsigned best = p, gi = 0;
            double bk = 0.0;
            if (i < pcount) {
                J.p_g[p] = J.p_dE[p];
                J.p_eg[p] = J.p_eE[p];
                bk = J.p_dE64[p];
                J.p_key[p] = bk;
                gi = J.p_idx[p];
                first = i == 0 || J.p_idx[p - 1] != gi;
                if (first) {
                    bc_ = J.p_c[p];
                    for (unsigned q = p + 1; q < pstart + pcount && J.p_idx[q] == gi; q++) {
                        const double kq = J.p_dE64[q];
                        const int cq = J.p_c[q];
                        if (kq < bk || (kq == bk && cq < bc_)) { best = q; bk = kq; bc_ = cq; }
                    }
                    adm = bk < 0.0 ? admissible(J, J.p_l[best], bc_, J.p_nbm[best]) : 0;
                }
            }
            select_append(first, adm, p, best, gi, bk, 0.0f, 0.0f, true);
        }
        return;
    }
    // the first own particle of the thread's lane group, fetched while the neighbourhood is staged
    constexpr int kSplit = 2;                        // lanes per particle (4 measured no faster in 3D)
    const unsigned my_i = (unsigned)tid / kSplit;
    const unsigned my_gi = my_i < pcount ? J.p_idx[pstart + my_i] : 0u;
    const int my_l = my_i < pcount ? J.p_l[pstart + my_i] : 0;
    const TileBox b = tile_box(J, k);
    const int r2max = J.r2max;
    const int rr = isqrt_floor(r2max);
    const bool can_stage = sob_can_stage(J);
    const SobLayout lay = sob_layout(J);
    Rec* s_rec = (Rec*)smem;
    unsigned short* s_x = (unsigned short*)(smem + lay.x);
    unsigned short* s_off = (unsigned short*)(smem + lay.off);
    unsigned* s_off32 = (unsigned*)s_off;
    unsigned* s_cs = (unsigned*)(smem + lay.cs);
    unsigned* s_cn = (unsigned*)(smem + lay.cn);
    unsigned* s_eoff = (unsigned*)(smem + lay.eoff);

    if (tid == 0) s_osc = 0;
    for (int d2 = tid; d2 <= r2max && d2 < 256; d2 += blockDim.x) {
        s_klut[d2] = make_float2(__ldg(J.klut + d2), __ldg(J.klut_lo + d2));
    }

    // staged pixel box: an x-slab [sx0, sx1) of the tile grown by rr (2D: z is the tile's single
    // plane); the whole tile first, halved while its particles do not fit
    const int by0 = b.y0 - rr, bz0 = NDIM == 3 ? b.z0 - rr : b.z0;
    const int bny = b.y1 - b.y0 + 2 * rr, bnz = NDIM == 3 ? b.z1 - b.z0 + 2 * rr : 1;
    int row_dy = 0, row_dz = 0, row_slot = -1;
    unsigned ring_total = 0;
    int ne = 0;
    if (can_stage) {
        // rows of the ball, (dz, dy) ascending, compacted in thread order
        const int w = 2 * rr + 1, nr = NDIM == 3 ? w * w : w;
        bool ok = false;
        int info = 0;
        if (tid < nr) {
            row_dy = tid % w - rr;
            row_dz = NDIM == 3 ? tid / w - rr : 0;
            const int dyz2 = row_dy * row_dy + row_dz * row_dz;
            ok = dyz2 <= r2max;
            info = isqrt_floor(r2max - (ok ? dyz2 : 0)) | (dyz2 << 8);
        }
        unsigned tot_rows;
        const unsigned slot = block_excl_scan(ok ? 1u : 0u, s_warp, tot_rows);
        if (ok) { s_rinfo[slot] = (unsigned short)info; row_slot = (int)slot; }
        if (tid == 0) s_nrows = (int)tot_rows;
        // ring cells: the tile's cells plus one ring, clipped to the image; their particle
        // ranges and an exclusive prefix of their counts (ring index of a cell's first particle)
        const int ex0 = max(b.cx0 - 1, 0), ex1 = min(b.cx0 + b.ccx + 1, J.ncx);
        const int ey0 = max(b.cy0 - 1, 0), ey1 = min(b.cy0 + b.ccy + 1, J.ncy);
        const int ez0 = NDIM == 3 ? max(b.cz0 - 1, 0) : b.cz0;
        const int ez1 = NDIM == 3 ? min(b.cz0 + b.ccz + 1, J.ncz) : b.cz0 + b.ccz;
        const int enx = ex1 - ex0, eny = ey1 - ey0;
        ne = enx * eny * (ez1 - ez0);
        const int chunk = (ne + blockDim.x - 1) / blockDim.x;
        const int e0 = min(tid * chunk, ne), e1 = min(e0 + chunk, ne);
        unsigned cnt = 0;
        for (int e = e0; e < e1; e++) {
            const int lx = e % enx, ly = (e / enx) % eny, lz = e / (enx * eny);
            const long long cid = ((long long)(ez0 + lz) * J.ncy + (ey0 + ly)) * J.ncx + (ex0 + lx);
            const unsigned cs = J.cell_start[cid], cn = J.cell_count[cid];
            s_cs[e] = cs;
            s_cn[e] = cn;
            cnt += cn;
        }
        __syncthreads();                               // s_warp reuse
        unsigned off = block_excl_scan(cnt, s_warp, ring_total);
        for (int e = e0; e < e1; e++) {
            s_eoff[e] = off;
            off += s_cn[e];
        }
    }

    unsigned osc = 0;
    int sx0 = b.x0, width = b.x1 - b.x0;
    while (sx0 < b.x1) {                                 // block-uniform
        const int sx1 = min(sx0 + width, b.x1);
        const int bx0 = sx0 - rr, bnx = sx1 - sx0 + 2 * rr;
        const int nbox = bnx * bny * bnz;
        bool staged = false;
        if (can_stage) {
            if (row_slot >= 0) s_rdelta[row_slot] = (row_dz * bny + row_dy) * bnx;
            for (int i = tid; i < (nbox + 2) / 2; i += blockDim.x) s_off32[i] = 0u;
            __syncthreads();
            // pass 1: particles per box pixel, one thread per ring particle
            for (unsigned i = tid; i < ring_total; i += blockDim.x) {
                const int e = ring_cell_of(s_eoff, ne, i);
                int x, y, z;
                pix_coords(J, J.p_idx[s_cs[e] + (i - s_eoff[e])], x, y, z);
                x -= bx0; y -= by0; z -= bz0;
                if ((unsigned)x < (unsigned)bnx && (unsigned)y < (unsigned)bny && (unsigned)z < (unsigned)bnz) {
                    const int bp = (z * bny + y) * bnx + x;
                    atomicAdd(&s_off32[bp >> 1], 1u << (16 * (bp & 1)));
                }
            }
            __syncthreads();
            // exclusive prefix over the box pixels (chunk per thread)
            const int pc = (nbox + blockDim.x - 1) / blockDim.x;
            const int q0 = min(tid * pc, nbox), q1 = min(q0 + pc, nbox);
            unsigned sum = 0;
            for (int q = q0; q < q1; q++) sum += s_off[q];
            unsigned staged_total;
            unsigned run = block_excl_scan(sum, s_warp, staged_total);
            if (staged_total > (unsigned)kRecCap && sx1 - sx0 > 1) {
                width = (sx1 - sx0 + 1) / 2;                  // too many: a narrower slab
                __syncthreads();
                continue;
            }
            for (int q = q0; q < q1; q++) {
                const unsigned c = s_off[q];
                s_off[q] = (unsigned short)run;
                run += c;
            }
            if (tid == 0) s_off[nbox] = (unsigned short)min(staged_total, 65535u);
            staged = staged_total <= (unsigned)kRecCap;
            if (tid == 0) s_dmax = 0u;
            __syncthreads();
            if (staged) {
                // pass 2: scatter. Particles of one pixel are adjacent in their cell, hence in
                // ring order; a particle's rank among them is the run of equal pixel indices
                // before it (found with warp ballots, global loads only across warp chunks).
                for (unsigned base = 0; base < ring_total; base += blockDim.x) {
                    const unsigned i = base + tid;
                    const bool v = i < ring_total;
                    unsigned p = 0, gi = 0xffffffffu, within = 0;
                    if (v) {
                        const int e = ring_cell_of(s_eoff, ne, i);
                        within = i - s_eoff[e];
                        p = s_cs[e] + within;
                        gi = J.p_idx[p];
                    }
                    const unsigned dbits = v ? __float_as_uint(fabsf(J.p_dE[p])) : 0u;
                    const unsigned wmax = __reduce_max_sync(0xffffffffu, dbits);
                    if (lane == 0 && wmax) atomicMax(&s_dmax, wmax);
                    unsigned prev = __shfl_up_sync(0xffffffffu, gi, 1);
                    if (lane == 0 && v && within > 0) prev = J.p_idx[p - 1];
                    const bool eq = v && within > 0 && prev == gi;
                    const unsigned m = __ballot_sync(0xffffffffu, eq);
                    int x, y, z;
                    pix_coords(J, v ? gi : 0u, x, y, z);
                    x -= bx0; y -= by0; z -= bz0;
                    if (v && (unsigned)x < (unsigned)bnx && (unsigned)y < (unsigned)bny && (unsigned)z < (unsigned)bnz) {
                        unsigned rank = 0;
                        if (eq) {
                            const unsigned zeros = ~m & ((2u << lane) - 1u);   // lanes <= lane not equal
                            if (zeros) {
                                rank = (unsigned)lane - (31u - __clz(zeros));
                            } else {
                                rank = (unsigned)lane + 1;                   // the run reaches lane 0
                                while (rank < within && J.p_idx[p - rank - 1] == gi) rank++;
                            }
                        }
                        const unsigned pos = s_off[(z * bny + y) * bnx + x] + rank;
                        Rec r;
                        r.dh = J.p_dE[p];
                        r.dl = J.p_dEl[p];
                        r.l = J.p_l[p];
                        r.c = J.p_c[p];
                        s_rec[pos] = r;
                        s_x[pos] = (unsigned short)x;
                    }
                }
            }
        }
        __syncthreads();

        const int nrows = staged ? s_nrows : 0;
        // kSplit lanes per particle, each taking every kSplit-th row of the ball; their partial
        // sums are added at the end (the bound below covers any order of the additions)
        const int h = tid % kSplit;
        const unsigned half = blockDim.x / kSplit;
        for (unsigned i0 = 0; i0 < pcount; i0 += half) {
            const unsigned i = i0 + my_i;
            const bool own = i < pcount;
            const unsigned p = pstart + (own ? i : 0u);
            const unsigned gi = i == my_i ? my_gi : J.p_idx[p];
            int x, y, z;
            pix_coords(J, gi, x, y, z);
            const bool act = own && x >= sx0 && x < sx1;
            const int lp = i == my_i ? my_l : J.p_l[p];
            // the particles of a pixel share g here, so its first particle (smallest c) is its
            // best. Whether its move is admissible does not depend on g: the test (and its table
            // loads) is issued now, so that its latency passes while Eq. 6 is summed.
            const bool first = act && h == 0 && (i == 0 || J.p_idx[p - 1] != gi);
            const int adm_pre = first ? admissible(J, lp, J.p_c[p], J.p_nbm[p]) : 0;
            DotAcc A, B;
            float aA = 0.f, aB = 0.f;
            int nA = 0, nB = 0;
            if (act && staged) {
                // the particle lies in the slab, so every row of its ball lies in the box
                const int lx = x - bx0;
                const int cbase = ((z - bz0) * bny + (y - by0)) * bnx + lx;
                for (int r = h; r < nrows; r += kSplit) {
                    const int info = s_rinfo[r];
                    const int rx = info & 255, dyz2 = info >> 8;
                    const int base = cbase + s_rdelta[r];
                    const unsigned j1 = s_off[base + rx + 1];
                    for (unsigned j = s_off[base - rx]; j < j1; j++) {
                        const int dx = (int)s_x[j] - lx;
                        const float2 K = s_klut[dyz2 + dx * dx];
                        const Rec q = s_rec[j];
                        // branch-free: the term goes to A (q in Q), to B (q in Q'; never both, as
                        // l_q != c_q) or nowhere (a zero term); the lanes of a warp stay together
                        const bool inA = q.l == lp, inB = q.c == lp;
                        DotAcc T;
                        T.s = inA ? A.s : B.s;
                        T.t = inA ? A.t : B.t;
                        T.add(K.x, K.y, (inA || inB) ? q.dh : 0.0f, (inA || inB) ? q.dl : 0.0f);
                        A.s = inA ? T.s : A.s;
                        A.t = inA ? T.t : A.t;
                        B.s = inA ? B.s : T.s;
                        B.t = inA ? B.t : T.t;
                        nA += inA;
                        nB += inB;
                    }
                }
                // the bound's sums of |K dE|: every term is at most K(0) times the largest staged
                // |dE| (K falls with the distance; |dl| <= 2^-24 |dh|)
                const float t_max = __fmul_rn(__fadd_rn(s_klut[0].x, s_klut[0].y),
                                              __uint_as_float(s_dmax)) * 1.0001f;
                aA = (float)nA * t_max;
                aB = (float)nB * t_max;
            } else if (act && h == 0) {
                sobolev_sums<NDIM>(J, lp, x, y, z, r2max, A, B, aA, aB, nA, nB);
            }
#pragma unroll
            for (int o = 1; o < kSplit; o <<= 1) {
                // the partner lanes' compensated sums joined by a two-sum of their leading parts
                const float As2 = __shfl_xor_sync(0xffffffffu, A.s, o), At2 = __shfl_xor_sync(0xffffffffu, A.t, o);
                const float Bs2 = __shfl_xor_sync(0xffffffffu, B.s, o), Bt2 = __shfl_xor_sync(0xffffffffu, B.t, o);
                A.add(1.0f, 0.0f, As2, At2);
                B.add(1.0f, 0.0f, Bs2, Bt2);
                aA += __shfl_xor_sync(0xffffffffu, aA, o);
                aB += __shfl_xor_sync(0xffffffffu, aB, o);
                nA += __shfl_xor_sync(0xffffffffu, nA, o);
                nB += __shfl_xor_sync(0xffffffffu, nB, o);
            }
            if (act && h == 0) {
                float gp, ep;
                float Aq = 0.f, Al = 0.f, Bq = 0.f, Bl = 0.f;
                if (nA) pair_div(A.s, A.t, nA, Aq, Al);
                if (nB) pair_div(B.s, B.t, nB, Bq, Bl);
                gp = pair_sub(Aq, Al, Bq, Bl);
                const float TA = nA ? aA / (float)nA : 0.f, TB = nB ? aB / (float)nB : 0.f;
                ep = pair_bound(gp, nA ? nA + kSplit : 0, TA, nB ? nB + kSplit : 0, TB);
                J.p_g[p] = gp;
                J.p_eg[p] = ep;
                J.p_key[p] = (double)gp;
                const float Af = __fadd_rn(Aq, Al), Bf = __fadd_rn(Bq, Bl);
                osc += (Af != 0.f && Bf != 0.f && ((Af > 0.f) == (Bf > 0.f))) ? 1u : 0u;
                // possibly negative (g < eg) and admissible makes the pixel's best a candidate;
                // its slot is taken after the last pass (no block barrier between passes)
                if (gp < ep && adm_pre) J.p_flags[p] |= adm_pre == 2 ? (kFlagCand | kFlagSplit) : kFlagCand;
            }
        }
        sx0 = sx1;
        __syncthreads();                                 // the next slab reuses shared memory
    }
    // the tile's candidates, marked above at their pixels' first particles, take their slots
    for (unsigned i0 = 0; i0 < pcount; i0 += blockDim.x) {           // uniform over the block
        const unsigned i = i0 + tid;
        const unsigned p = pstart + i;
        bool first = false;
        int adm = 0;
        unsigned gi = 0;
        float gp = 0.0f, ep = 0.0f;
        if (i < pcount) {
            gi = J.p_idx[p];
            first = i == 0 || J.p_idx[p - 1] != gi;
            const unsigned char f = first ? J.p_flags[p] : (unsigned char)0;
            adm = (f & kFlagCand) ? ((f & kFlagSplit) ? 2 : 1) : 0;
            if (adm) {
                gp = J.p_g[p];
                ep = J.p_eg[p];
            }
        }
        select_append(first, adm, p, p, gi, (double)gp, gp, ep, false);
    }
    if (osc) atomicAdd(&s_osc, osc);
    __syncthreads();
    if (tid == 0 && s_osc) atomicAdd(&ctr->n_osc, s_osc);
}

size_t sobolev_smem_bytes(const Job& J)
{
    return sob_layout(J).total;
}

cudaError_t launch_sobolev(const Group& g, BatchCtl* bc, int ndim, size_t smem, cudaStream_t st)
{
    if (g.total_tiles == 0) return cudaSuccess;
    if (ndim == 2) return launch_stage(k_sobolev<2>, g.total_tiles, kBlock, smem, st, g, bc);
    return launch_stage(k_sobolev<3>, g.total_tiles, kBlock, smem, st, g, bc);
}

// Dynamic shared memory limits, set outside any stream capture. The limits only grow (per
// device), so that a context built later with smaller tiles does not lower the limit below
// what the graphs of earlier contexts launch with.
cudaError_t configure_kernels(size_t x2, size_t x3, size_t s2, size_t s3)
{
    static std::mutex mu;
    static size_t cur[64][4];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    const size_t want[4] = {std::max<size_t>(x2, 1), std::max<size_t>(x3, 1), std::max<size_t>(s2, 1),
                            std::max<size_t>(s3, 1)};
    const void* fn[4] = {(const void*)k_extract<2>, (const void*)k_extract<3>, (const void*)k_sobolev<2>,
                         (const void*)k_sobolev<3>};
    for (int i = 0; i < 4; i++) {
        if (want[i] <= cur[dev][i]) continue;
        if ((e = cudaFuncSetAttribute(fn[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)want[i])) != cudaSuccess)
            return e;
        cur[dev][i] = want[i];
    }
    return cudaSuccess;
}

}  // namespace segk
