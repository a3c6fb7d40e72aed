// Region statistics without device allocation: the same exact reduction seg_init runs,
// with its accumulators in a fixed file-scope device array instead of cudaMalloc'd memory.
//
// For callers that must not allocate device memory, e.g. code running inside a memory
// pool or allocator of their own (where an unplanned cudaMalloc would break the pool's
// accounting or fragment it), code that may not synchronise the device (cudaMalloc and
// cudaFree can), or a framework that hands libseg only the buffers it owns.
#include <cuda_runtime.h>

#include <mutex>

#include "seg_internal.cuh"

using namespace segk;

namespace {

constexpr int kMaxLabels = 1024;          // labels 0..1023
constexpr int kSlots = 255;               // every float32 exponent slot, so any input stays in bounds
constexpr int kQSlots = 2 * (kSlots - 1) + 25;
constexpr size_t kScratchBytes = (size_t)kMaxLabels * (1 + kSlots + kQSlots) * 8   // n, S and Q accumulators
                                 + (size_t)kMaxLabels * (3 * 8 + 3 * 4)             // derived tables
                                 + 256;                                              // label check flag
constexpr int kMaxDevices = 64;

// Every GPU that loads libseg holds these until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static __device__ __align__(256) Job g_job;

std::mutex g_setup_lock;
unsigned char* g_scratch_ptr[kMaxDevices];
Job* g_job_ptr[kMaxDevices];

__global__ void k_check_labels(const int* labels, long long npix, int nlabels, int* bad)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npix; i += (long long)gridDim.x * blockDim.x) {
        int m = labels[i];
        if (m < 0 || m >= nlabels) {
            *bad = 1;
            return;
        }
    }
}

bool device_pointer(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice;
}

}  // namespace

extern "C" int seg_region_stats_noalloc(int32_t dtype, int64_t npix, const void* image, const int32_t* labels,
                                        int32_t nlabels, int64_t* n, double* S, double* Q, void* cuda_stream)
{
    if (dtype != SEG_F32 && dtype != SEG_U16) return SEG_EINVAL;
    if (npix < 1 || npix >= 2147483647LL) return SEG_EINVAL;
    if (nlabels < 1 || nlabels > kMaxLabels) return SEG_EINVAL;
    if (!image || !labels || !n || !S || !Q) return SEG_EINVAL;
    if (!device_pointer(image) || !device_pointer(labels) || !device_pointer(n) || !device_pointer(S) ||
        !device_pointer(Q))
        return SEG_EINVAL;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SEG_ECUDA;
    }
    unsigned char* base;
    Job* job;
    {
        // once per device, with that device current: the device addresses of the arrays
        std::lock_guard<std::mutex> lock(g_setup_lock);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            void* q = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || cudaGetSymbolAddress(&q, g_job) != cudaSuccess) {
                cudaGetLastError();
                return SEG_ECUDA;
            }
            g_scratch_ptr[dev] = (unsigned char*)p;
            g_job_ptr[dev] = (Job*)q;
        }
        base = g_scratch_ptr[dev];
        job = g_job_ptr[dev];
    }
    const int M = nlabels;
    Job h{};
    h.ndim = 2;
    h.npix = npix;
    h.dtype = dtype;
    h.M = M;
    h.slot_lo = 1;
    h.nS = kSlots;
    h.nQ = kQSlots;
    h.I = image;
    h.L = (int*)labels;
    unsigned char* at = base;
    h.st_n = (long long*)at;
    at += (size_t)M * 8;
    h.st_S = (long long*)at;
    at += (size_t)M * (dtype == SEG_F32 ? kSlots : 1) * 8;
    h.st_Q = (long long*)at;
    at += (size_t)M * (dtype == SEG_F32 ? kQSlots : 1) * 8;
    const size_t zero_bytes = (size_t)(at - base);
    h.mu64 = (double*)at;
    at += (size_t)M * 8;
    h.wp64 = (double*)at;
    at += (size_t)M * 8;
    h.wm64 = (double*)at;
    at += (size_t)M * 8;
    h.mu32 = (float*)at;
    at += (size_t)M * 4;
    h.wp32 = (float*)at;
    at += (size_t)M * 4;
    h.wm32 = (float*)at;
    at += (size_t)M * 4;
    int* bad = (int*)(base + kScratchBytes - 256);
    h.S64 = S;
    h.Q64 = Q;

    // labels outside 0..nlabels-1 would index past the accumulators: check first
    int hbad = 0;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), stream);
    if (e == cudaSuccess) {
        count_launch();
        k_check_labels<<<256, 256, 0, stream>>>(labels, npix, M, bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SEG_ECUDA;
    }
    if (hbad) return SEG_EINVAL;

    // the accumulators start at zero on every call (the array keeps the previous call's contents)
    e = cudaMemcpyToSymbolAsync(g_job, &h, sizeof(Job), 0, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base, 0, zero_bytes, stream);
    if (e == cudaSuccess) e = launch_stats_init(job, 0, npix, stream);
    if (e == cudaSuccess) e = launch_stats_finalize(job, 1, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(n, h.st_n, (size_t)M * 8, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SEG_ECUDA;
    }
    return SEG_OK;
}
