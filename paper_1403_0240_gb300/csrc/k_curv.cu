// Curvature regulariser (SEG_REG_CURVATURE): after extraction, every particle (x: l -> c) adds
// w (A_l(x) - A_c(x)) to its energy difference, A_m(x) the pixels of label m in the ball of
// radius rho around x (x counted in l, pixels outside the image in neither). The integral
// invariants of a ball centred on a region's boundary give that region's curvature from its
// share of the ball; the first variation of |Gamma| under the move leaves this difference of
// counts, with w = lambda 3 / (2 rho^3) in 2D and lambda 4 / (pi rho^4) in 3D (host side).
//
// One warp per particle, the lanes over the ball offsets (consecutive dx of a row in
// consecutive lanes, so the label loads of a row coalesce). The energy difference is completed in
// FP64 from the data term extraction left, in the order of the definition.
#include <cuda_runtime.h>

#include <algorithm>

#include "seg_internal.cuh"

namespace segk {

namespace {

constexpr int kBlock = 256;
constexpr int kStaged = 2048;                 // offsets kept in shared memory

__global__ void __launch_bounds__(kBlock) k_curvature(const Job* jobs, int j)
{
    pdl_enter();
    __shared__ int4 s_off[kStaged];
    const Job& J = jobs[j];
    const Counters* ctr = J.ctr;
    if (ld_volatile(&ctr->skip) != 0 || ld_volatile(&ctr->need) != 0) return;
    const int n_off = J.cv_n;
    const int staged = min(n_off, kStaged);
    for (int u = threadIdx.x; u < staged; u += kBlock) s_off[u] = J.cv_off[u];
    __syncthreads();
    const unsigned np = ld_volatile(&ctr->n_particles);
    const int lane = threadIdx.x & 31;
    const unsigned warps = gridDim.x * (kBlock / 32);
    for (unsigned p = blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5); p < np; p += warps) {
        const unsigned gi = J.p_idx[p];
        const int l = J.p_l[p], c = J.p_c[p];
        int x, y, z;
        pix_coords(J, gi, x, y, z);
        int bal = 0;
        for (int u = lane; u < n_off; u += 32) {
            const int4 d = u < kStaged ? s_off[u] : __ldg(J.cv_off + u);
            const int xx = x + d.z, yy = y + d.y, zz = z + d.x;
            if (xx < 0 || xx >= J.W || yy < 0 || yy >= J.H || zz < 0 || zz >= J.D) continue;
            const int m = __ldg(J.L + ((long long)zz * J.H + yy) * J.W + xx);
            bal += (int)(m == l) - (int)(m == c);
        }
        bal = __reduce_add_sync(0xffffffffu, bal);
        // the FP64 data term from extraction plus w times the count, in the order of the definition
        if (lane == 0) store_dE(J, p, __dadd_rn(J.p_dE64[p], __dmul_rn(J.curv_w64, (double)bal)));
    }
}

}  // namespace

cudaError_t launch_curvature(const Job* jobs, int j, int sms, cudaStream_t s)
{
    return launch_stage(k_curvature, (unsigned)sms * 4, kBlock, 0, s, jobs, j);
}

}  // namespace segk
