// Deconvolving piecewise-constant model (Methods, Eq. 8): the expected image is
// J = s_theta(Gamma) * K, K the point-spread function K(x) = k(x) k(y) [k(z)] with a symmetric
// profile k(-r..r), s_theta the region means painted on the label image, zero outside the
// image. A move of pixel x from l to c, theta held, changes the data term sum (I - J)^2 by
// d^2 |K_x|^2 - 2 d G(x) with d = theta_c - theta_l and G = K * (I - J).
//
// Every iteration recomputes J, R = I - J and the passes of K * R in FP64 before extraction,
// by separable passes along x, then y, then z. Each output of a pass is the fused multiply-add
// chain acc = fma(k(u), f(. + u e_axis), acc) over ascending u starting from +0; taps outside
// the image are skipped, which is exact (they would add k(u) * 0 to a partial sum that is
// never -0). The last pass of G (y in 2D, z in 3D) is only needed at particle pixels and is
// taken there by extraction (deconv_G below, shared with the FP64 recompute).
//
// The passes are bound by the FP64 pipe: 2r + 1 fused multiply-adds per pixel and pass
// against 16 bytes of memory traffic.
#include <cuda_runtime.h>

#include <algorithm>

#include "seg_internal.cuh"

namespace segk {

namespace {

constexpr int kBlock = 256;
constexpr int kMaxTaps = 2 * SEG_PSF_MAX_RADIUS + 1;

enum { kSrcTheta = 0, kSrcField = 1 };

__device__ __forceinline__ double image_value(const Job& J, long long i)
{
    if (J.dtype == SEG_F32) return (double)((const float*)J.I)[i];
    return (double)((const unsigned short*)J.I)[i];
}

// One pass along `axis` of job j: dst = k (x) src along the axis (src = theta_L for
// kSrcTheta); with RESID the output is I - (that sum). One output per thread.
template <int SRC, bool RESID>
__global__ void __launch_bounds__(kBlock) k_psf_pass(const Job* jobs, int j, int axis, const double* __restrict__ src,
                                                     double* __restrict__ dst)
{
    pdl_enter();
    __shared__ double s_k[kMaxTaps];
    const Job& J = jobs[j];
    if (ld_volatile(&J.ctr->skip)) return;
    const int r = J.psf_r;
    for (int u = threadIdx.x; u <= 2 * r; u += kBlock) s_k[u] = J.psf[u];
    __syncthreads();
    const long long stride = axis == 0 ? 1LL : (axis == 1 ? (long long)J.W : (long long)J.W * J.H);
    const int extent = axis == 0 ? J.W : (axis == 1 ? J.H : J.D);
    const unsigned npix = (unsigned)J.npix;
    const double* kk = s_k + r;
    for (unsigned i = blockIdx.x * kBlock + threadIdx.x; i < npix; i += gridDim.x * kBlock) {
        int x, y, z;
        pix_coords(J, i, x, y, z);
        const int t = axis == 0 ? x : (axis == 1 ? y : z);
        const int lo = max(-r, -t), hi = min(r, extent - 1 - t);
        long long q = (long long)i + (long long)lo * stride;
        double acc = 0.0;
        for (int u = lo; u <= hi; u++, q += stride) {
            const double f = SRC == kSrcTheta ? __ldg(J.mu64 + __ldg(J.L + q)) : __ldg(src + q);
            acc = __fma_rn(kk[u], f, acc);
        }
        if (RESID) acc = __dsub_rn(image_value(J, i), acc);
        dst[i] = acc;
    }
}

// Per axis a and position t: sum of k(u)^2 over the u with t + u inside the image.
__global__ void k_psf_norms(const Job* job)
{
    const Job& J = *job;
    const int r = J.psf_r;
    const int total = J.W + J.H + (J.ndim == 3 ? J.D : 0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        int t = i, extent = J.W;
        if (t >= J.W) {
            t -= J.W;
            extent = J.H;
            if (t >= J.H) { t -= J.H; extent = J.D; }
        }
        const int lo = max(-r, -t), hi = min(r, extent - 1 - t);
        double acc = 0.0;
        for (int u = lo; u <= hi; u++) acc = __fma_rn(J.psf[u + r], J.psf[u + r], acc);
        J.psf_n[i] = acc;
    }
}

}  // namespace

// Resident blocks per SM of each pass kernel, found before any graph capture.
// J (passes along x, y[, z], the last one leaving R = I - J), then every pass of K * R but the
// last: 2D x; 3D x, y. The field the last pass reads is J.dc_T (2D) or J.dc_T2 (3D).
cudaError_t launch_deconv(const Job* jobs, int j, const Job& h, int sms, cudaStream_t s)
{
    const unsigned grid = (unsigned)std::min<long long>((h.npix + kBlock - 1) / kBlock, (long long)sms * 8);
    const double* none = nullptr;
    cudaError_t e;
    if ((e = launch_stage(k_psf_pass<kSrcTheta, false>, grid, kBlock, 0, s, jobs, j, 0, none, h.dc_T)) != cudaSuccess)
        return e;
    if (h.ndim == 2) {
        if ((e = launch_stage(k_psf_pass<kSrcField, true>, grid, kBlock, 0, s, jobs, j, 1, (const double*)h.dc_T,
                              h.dc_R)) != cudaSuccess) return e;
        return launch_stage(k_psf_pass<kSrcField, false>, grid, kBlock, 0, s, jobs, j, 0, (const double*)h.dc_R, h.dc_T);
    }
    if ((e = launch_stage(k_psf_pass<kSrcField, false>, grid, kBlock, 0, s, jobs, j, 1, (const double*)h.dc_T,
                          h.dc_T2)) != cudaSuccess) return e;
    if ((e = launch_stage(k_psf_pass<kSrcField, true>, grid, kBlock, 0, s, jobs, j, 2, (const double*)h.dc_T2,
                          h.dc_R)) != cudaSuccess) return e;
    if ((e = launch_stage(k_psf_pass<kSrcField, false>, grid, kBlock, 0, s, jobs, j, 0, (const double*)h.dc_R,
                          h.dc_T)) != cudaSuccess) return e;
    return launch_stage(k_psf_pass<kSrcField, false>, grid, kBlock, 0, s, jobs, j, 1, (const double*)h.dc_T, h.dc_T2);
}

cudaError_t launch_psf_norms(const Job* job, const Job& h, cudaStream_t s)
{
    const int total = h.W + h.H + (h.ndim == 3 ? h.D : 0);
    count_launch();
    k_psf_norms<<<(total + kBlock - 1) / kBlock, kBlock, 0, s>>>(job);
    return cudaGetLastError();
}

}  // namespace segk
