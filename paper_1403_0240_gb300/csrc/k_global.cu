// Eq. 6 with the length scale of the inner product set to the contour length, E = |Gamma|
// (Length scale section of the paper: the scale-invariant choice it leaves to future work
// because every particle pair then interacts). |Gamma| is the number of connectivity-adjacent
// pixel pairs with different labels, kept exact from iteration to iteration by the moves.
#include <cuda_runtime.h>

#include "seg_internal.cuh"

namespace segk {

namespace {

constexpr int kBlock = 256;
constexpr int kChunk = 512;          // partner particles staged per round

// Eq. 5, evaluated in the order written (FP64, no fused multiply-add)
__device__ __forceinline__ double kernel_eq5_fp64(double r, double E)
{
    const double eps = 1.0 / 24.0;
    const double x = __ddiv_rn(r, E);
    const double num = __dadd_rn(__dsub_rn(__dmul_rn(x, x), x), 1.0 / 6.0);
    return __dmul_rn(__ddiv_rn(1.0, E), __dadd_rn(1.0, __ddiv_rn(num, 2.0 * eps)));
}


}  // namespace

// Per iteration and job in E = |Gamma| mode: the support bound and the kernel table over
// every squared distance that occurs in the image.
__global__ void k_global_lut(const Job* jobs, int njobs)
{
    pdl_enter();
    for (int j = 0; j < njobs; j++) {
        const Job& J = jobs[j];
        if (!J.global_E) continue;
        Counters* ctr = J.ctr;
        if (ld_volatile(&ctr->skip) || ld_volatile(&ctr->mode) != SEG_SOBOLEV_GLOBAL) continue;
        const long long P = *(volatile long long*)&ctr->perim;
        const long long lim = (P * P + 3) / 4;        // d^2 < (E/2)^2  <=>  d^2 < ceil(P^2 / 4)
        if (blockIdx.x == 0 && threadIdx.x == 0) ctr->g_lim = lim;
        const double E = (double)P;
        for (long long d2 = blockIdx.x * (long long)blockDim.x + threadIdx.x; d2 <= J.gd2max;
             d2 += (long long)gridDim.x * blockDim.x) {
            const double K = d2 < lim ? kernel_eq5_fp64(__dsqrt_rn((double)d2), E) : 0.0;
            const float Kh = __double2float_rn(K);
            J.gK64[d2] = K;
            J.gK32[d2] = Kh;
            J.gK32l[d2] = __double2float_rn(__dsub_rn(K, (double)Kh));
        }
    }
}

// One block per tile: the tile's particles against every particle of the job, staged in
// shared memory kChunk at a time; compensated sums of exact products as in the local kernel.
template <int NDIM>
__global__ void __launch_bounds__(kBlock) k_sobolev_global(Group g)
{
    pdl_enter();
    __shared__ int s_x[kChunk], s_y[kChunk], s_z[kChunk], s_l[kChunk], s_c[kChunk];
    __shared__ float s_dh[kChunk], s_dl[kChunk];
    __shared__ unsigned s_osc;
    const int tid = threadIdx.x;
    const unsigned t = blockIdx.x;
    const int gj = group_job_of_tile(g, t);
    const Job& J = g.jobs[g.job_ids[gj]];
    const unsigned k = t - g.tile_prefix[gj];
    Counters* ctr = J.ctr;
    if (!J.global_E || ld_volatile(&ctr->skip) || ld_volatile(&ctr->need)) return;
    if (ld_volatile(&ctr->mode) != SEG_SOBOLEV_GLOBAL) return;
    const unsigned pstart = J.tile_start[k], pcount = J.tile_count[k];
    if (pcount == 0) return;
    const unsigned np = ld_volatile(&ctr->n_particles);
    const long long lim = *(volatile long long*)&ctr->g_lim;
    if (tid == 0) s_osc = 0;
    unsigned osc = 0;
    for (unsigned i0 = 0; i0 < pcount; i0 += blockDim.x) {
        const unsigned i = i0 + tid;
        const bool own = i < pcount;
        const unsigned p = pstart + (own ? i : 0);
        int x = 0, y = 0, z = 0;
        pix_coords(J, J.p_idx[p], x, y, z);
        const int lp = J.p_l[p];
        DotAcc A, B;
        float aA = 0.f, aB = 0.f;
        int nA = 0, nB = 0;
        for (unsigned q0 = 0; q0 < np; q0 += kChunk) {
            const unsigned nq = min((unsigned)kChunk, np - q0);
            __syncthreads();
            for (unsigned jj = tid; jj < nq; jj += blockDim.x) {
                const unsigned q = q0 + jj;
                int qx, qy, qz;
                pix_coords(J, J.p_idx[q], qx, qy, qz);
                s_x[jj] = qx;
                s_y[jj] = qy;
                s_z[jj] = qz;
                s_l[jj] = J.p_l[q];
                s_c[jj] = J.p_c[q];
                s_dh[jj] = J.p_dE[q];
                s_dl[jj] = J.p_dEl[q];
            }
            __syncthreads();
            if (!own) continue;
            for (unsigned jj = 0; jj < nq; jj++) {
                const long long dx = s_x[jj] - x, dy = s_y[jj] - y, dz = NDIM == 3 ? s_z[jj] - z : 0;
                const long long d2 = dx * dx + dy * dy + dz * dz;
                if (d2 >= lim) continue;
                const int ql = s_l[jj], qc = s_c[jj];
                if (ql != lp && qc != lp) continue;
                const float Kh = __ldg(J.gK32 + d2), Kl = __ldg(J.gK32l + d2);
                if (ql == lp) { aA += fabsf(A.add(Kh, Kl, s_dh[jj], s_dl[jj])); nA++; }
                else { aB += fabsf(B.add(Kh, Kl, s_dh[jj], s_dl[jj])); nB++; }
            }
        }
        if (own) {
            float Aq = 0.f, Al = 0.f, Bq = 0.f, Bl = 0.f;
            if (nA) pair_div(A.s, A.t, nA, Aq, Al);
            if (nB) pair_div(B.s, B.t, nB, Bq, Bl);
            const float gp = pair_sub(Aq, Al, Bq, Bl);
            J.p_g[p] = gp;
            J.p_eg[p] = pair_bound(gp, nA, nA ? aA / (float)nA : 0.f, nB, nB ? aB / (float)nB : 0.f);
            J.p_key[p] = (double)gp;
            const float Af = __fadd_rn(Aq, Al), Bf = __fadd_rn(Bq, Bl);
            osc += (Af != 0.f && Bf != 0.f && ((Af > 0.f) == (Bf > 0.f))) ? 1u : 0u;
        }
    }
    if (osc) atomicAdd(&s_osc, osc);
    __syncthreads();
    if (tid == 0 && s_osc) atomicAdd(&ctr->n_osc, s_osc);
}

cudaError_t launch_global_lut(const Job* jobs, int njobs, int sms, cudaStream_t s)
{
    return launch_stage(k_global_lut, sms * 2, 256, 0, s, jobs, njobs);
}

cudaError_t launch_sobolev_global(const Group& g, int ndim, cudaStream_t s)
{
    if (g.total_tiles == 0) return cudaSuccess;
    if (ndim == 2) return launch_stage(k_sobolev_global<2>, g.total_tiles, kBlock, 0, s, g);
    return launch_stage(k_sobolev_global<3>, g.total_tiles, kBlock, 0, s, g);
}

}  // namespace segk
