// Region splitting (SEG_TOPO_SPLIT). A removal that locally disconnects its region is
// admissible; after the moves of an iteration in which such a move was made, every foreground
// label's connectivity components but the one holding its smallest pixel index get new labels,
// numbered upward from the label count in ascending order of the components' smallest pixel
// indices (foreground regions stay connected sets, Particle-based image segmentation).
//
// Components by a lock-free union-find over the pixels (each root the smallest pixel index of
// its component: a union hangs the larger root under the smaller), then the statistics of
// every label are recomputed exactly. Every kernel returns at once unless the iteration made a
// split move; the retry loops are bounded.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "seg_internal.cuh"

namespace segk {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ bool split_pending(const Job& J)
{
    return ld_volatile(&J.ctr->n_split) != 0 && !ld_volatile(&J.ctr->skip) && !ld_volatile(&J.ctr->error);
}

__device__ __forceinline__ int cc_parent(const int* parent, int x) { return *(const volatile int*)(parent + x); }

// root of x; false when the walk did not end within the bound
__device__ __forceinline__ bool cc_find(const int* parent, int x, int& root)
{
    for (unsigned it = 0; it < kSpinLimit; it++) {
        const int p = cc_parent(parent, x);
        if (p == x) { root = x; return true; }
        x = p;
    }
    return false;
}

__device__ __forceinline__ bool cc_unite(int* parent, int a, int b)
{
    for (unsigned it = 0; it < kSpinLimit; it++) {
        int ra, rb;
        if (!cc_find(parent, a, ra) || !cc_find(parent, b, rb)) return false;
        if (ra == rb) return true;
        if (ra > rb) { const int t = ra; ra = rb; rb = t; }
        if (atomicCAS(parent + rb, rb, ra) == rb) return true;   // else rb got a parent meanwhile
        a = ra;
        b = rb;
    }
    return false;
}

__global__ void __launch_bounds__(kBlock) k_cc_init(const Job* jobs, int j)
{
    pdl_enter();
    const Job& J = jobs[j];
    if (!split_pending(J)) return;
    const long long stride = (long long)gridDim.x * kBlock;
    for (long long i = blockIdx.x * (long long)kBlock + threadIdx.x; i < J.npix; i += stride) {
        J.cc_parent[i] = (int)i;
        if (i < J.M) J.cc_first[i] = INT_MAX;
    }
}

// unions along the forward neighbours (x+1, y+1, z+1) of equal foreground label
__global__ void __launch_bounds__(kBlock) k_cc_union(const Job* jobs, int j)
{
    pdl_enter();
    const Job& J = jobs[j];
    if (!split_pending(J)) return;
    const long long stride = (long long)gridDim.x * kBlock;
    const long long HW = (long long)J.W * J.H;
    bool ok = true;
    for (long long i = blockIdx.x * (long long)kBlock + threadIdx.x; i < J.npix; i += stride) {
        const int m = J.L[i];
        if (m == 0) continue;
        int x, y, z;
        pix_coords(J, (unsigned)i, x, y, z);
        if (x + 1 < J.W && J.L[i + 1] == m) ok = cc_unite(J.cc_parent, (int)i, (int)(i + 1)) && ok;
        if (y + 1 < J.H && J.L[i + J.W] == m) ok = cc_unite(J.cc_parent, (int)i, (int)(i + J.W)) && ok;
        if (J.ndim == 3 && z + 1 < J.D && J.L[i + HW] == m) ok = cc_unite(J.cc_parent, (int)i, (int)(i + HW)) && ok;
    }
    if (!ok) atomicExch(&J.ctr->error, SEG_ETIMEOUT);
}

// every pixel points to its root; each label's smallest pixel index (its smallest root)
__global__ void __launch_bounds__(kBlock) k_cc_roots(const Job* jobs, int j)
{
    pdl_enter();
    const Job& J = jobs[j];
    if (!split_pending(J)) return;
    const long long stride = (long long)gridDim.x * kBlock;
    bool ok = true;
    for (long long i = blockIdx.x * (long long)kBlock + threadIdx.x; i < J.npix; i += stride) {
        const int m = J.L[i];
        if (m == 0) continue;
        int r = (int)i;
        ok = cc_find(J.cc_parent, (int)i, r) && ok;
        J.cc_parent[i] = r;
        if (r == (int)i) atomicMin(J.cc_first + m, (int)i);
    }
    if (!ok) atomicExch(&J.ctr->error, SEG_ETIMEOUT);
}

// the roots of the pieces that get new labels
__global__ void __launch_bounds__(kBlock) k_cc_collect(const Job* jobs, int j)
{
    pdl_enter();
    const Job& J = jobs[j];
    if (!split_pending(J)) return;
    const long long stride = (long long)gridDim.x * kBlock;
    for (long long i = blockIdx.x * (long long)kBlock + threadIdx.x; i < J.npix; i += stride) {
        const int m = J.L[i];
        if (m == 0 || J.cc_parent[i] != (int)i || J.cc_first[m] == (int)i) continue;
        const unsigned slot = atomicAdd(&J.ctr->n_newcomp, 1u);
        if (slot < (unsigned)J.M) J.cc_list[slot] = (int)i;
    }
}

// new labels in ascending order of the pieces' smallest pixel indices (one block)
__global__ void __launch_bounds__(1024) k_cc_assign(const Job* jobs, int j)
{
    pdl_enter();
    const Job& J = jobs[j];
    if (!split_pending(J)) return;
    const unsigned n = ld_volatile(&J.ctr->n_newcomp);
    const int base = J.ctr->n_labels;
    if ((long long)base + n > J.M) {                // beyond the label capacity
        if (threadIdx.x == 0) {
            atomicExch(&J.ctr->error, SEG_ENOMEM);
            atomicExch(&J.ctr->skip, 1);
        }
        return;
    }
    for (unsigned k = threadIdx.x; k < n; k += blockDim.x) {
        const int r = J.cc_list[k];
        unsigned rank = 0;
        for (unsigned q = 0; q < n; q++) rank += J.cc_list[q] < r ? 1u : 0u;
        J.cc_newl[r] = base + (int)rank;
    }
    __syncthreads();
    if (threadIdx.x == 0) J.ctr->n_labels = base + (int)n;
}

__global__ void __launch_bounds__(kBlock) k_cc_relabel(const Job* jobs, int j)
{
    pdl_enter();
    const Job& J = jobs[j];
    if (!split_pending(J)) return;
    const long long stride = (long long)gridDim.x * kBlock;
    for (long long i = blockIdx.x * (long long)kBlock + threadIdx.x; i < J.npix; i += stride) {
        const int m = J.L[i];
        if (m == 0) continue;
        const int r = J.cc_parent[i];
        if (r != J.cc_first[m]) J.L[i] = J.cc_newl[r];
    }
}

}  // namespace

cudaError_t launch_relabel(const Job* jobs, int j, const Job& h, int sms, cudaStream_t s)
{
    const unsigned grid = (unsigned)std::min<long long>((h.npix + kBlock - 1) / kBlock, (long long)sms * 8);
    cudaError_t e;
    if ((e = launch_stage(k_cc_init, grid, kBlock, 0, s, jobs, j)) != cudaSuccess) return e;
    if ((e = launch_stage(k_cc_union, grid, kBlock, 0, s, jobs, j)) != cudaSuccess) return e;
    if ((e = launch_stage(k_cc_roots, grid, kBlock, 0, s, jobs, j)) != cudaSuccess) return e;
    if ((e = launch_stage(k_cc_collect, grid, kBlock, 0, s, jobs, j)) != cudaSuccess) return e;
    if ((e = launch_stage(k_cc_assign, 1u, 1024u, 0, s, jobs, j)) != cudaSuccess) return e;
    if ((e = launch_stage(k_cc_relabel, grid, kBlock, 0, s, jobs, j)) != cudaSuccess) return e;
    if ((e = launch_stats_zero_after_split(jobs, j, h, s)) != cudaSuccess) return e;
    return launch_stats_init(jobs, j, h.npix, s, true);
}

}  // namespace segk
