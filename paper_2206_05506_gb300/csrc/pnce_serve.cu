// Row gather / scatter for batched serving.  A serving batch packs the antennas of several
// requests, each with its own received block and result buffer, into one contiguous
// estimate.  These kernels move rows between per-antenna addresses (typically page-locked
// host memory, read and written by the GPU directly over the host link) and the batch's
// contiguous device buffers, so a whole batch needs no per-request copy calls and its
// launch sequence can be captured once and replayed.  The contiguous copy-out kernel serves
// pnce_estimate_host: stores from the SMs into page-locked host memory share the host link
// with a concurrent host-to-device DMA better than a device-to-host DMA does (measured on
// GB300: 2.15 GB in and 1.07 GB out together in 10.6 ms against 11.3 ms with two DMAs; the
// inbound copy alone takes 10.15 ms).
#include "pnce_internal.h"

namespace {

constexpr int THREADS = 256;

// dst[r][0 .. nelem) = src_rows[r][0 .. nelem) (8-byte elements); one block per row
__global__ void __launch_bounds__(THREADS)
gather_rows_kernel(const uint64_t* __restrict__ src_rows, int rows, int nelem,
                   float2* __restrict__ dst, long long dst_pitch) {
    const int r = blockIdx.x;
    if (r >= rows) return;
    const float2* src = reinterpret_cast<const float2*>(src_rows[r]);
    float2* d = dst + (long long)r * dst_pitch;
    if (!src) return;
    for (int i = threadIdx.x; i < nelem; i += THREADS) d[i] = src[i];
}

// dst_rows[r][0 .. counts[r]) = src[r][0 .. counts[r]), counts[r] <= src_pitch
__global__ void __launch_bounds__(THREADS)
scatter_rows_kernel(const float2* __restrict__ src, long long src_pitch,
                    const uint64_t* __restrict__ dst_rows, const int* __restrict__ counts,
                    int rows) {
    const int r = blockIdx.x;
    if (r >= rows) return;
    float2* d = reinterpret_cast<float2*>(dst_rows[r]);
    int n = counts[r];
    if (!d || n <= 0) return;
    if (n > src_pitch) n = (int)src_pitch;
    const float2* s = src + (long long)r * src_pitch;
    for (int i = threadIdx.x; i < n; i += THREADS) d[i] = s[i];
}

// dst[0 .. n) = src[0 .. n) (8-byte elements), grid-stride; dst is page-locked host memory
__global__ void __launch_bounds__(THREADS)
copy_out_kernel(const float2* __restrict__ src, float2* dst, long long n) {
    const long long stride = (long long)gridDim.x * THREADS;
    for (long long i = blockIdx.x * (long long)THREADS + threadIdx.x; i < n; i += stride)
        dst[i] = __ldcs(src + i);
}

}  // namespace

namespace pnce {

cudaError_t launch_copy_to_host(const void* src_dev, void* dst_host_mapped, size_t bytes,
                                int num_sms, cudaStream_t s) {
    const long long n = (long long)(bytes / sizeof(float2));
    if (n <= 0) return cudaSuccess;
    long long grid = (n + THREADS - 1) / THREADS;
    if (grid > num_sms) grid = num_sms;
    copy_out_kernel<<<(unsigned)grid, THREADS, 0, s>>>(static_cast<const float2*>(src_dev),
                                                       static_cast<float2*>(dst_host_mapped), n);
    return cudaGetLastError();
}

}  // namespace pnce

extern "C" {

pnce_status pnce_gather_rows(const uint64_t* src_rows, int rows, int nelem, void* dst_dev,
                             long long dst_pitch, void* stream) {
    if (!src_rows || !dst_dev || rows < 0 || nelem < 0 || dst_pitch < nelem) return PNCE_EINVAL;
    if (((uintptr_t)dst_dev & 7u) || ((uintptr_t)src_rows & 7u)) return PNCE_EINVAL;
    if (rows == 0 || nelem == 0) return PNCE_OK;
    gather_rows_kernel<<<rows, THREADS, 0, static_cast<cudaStream_t>(stream)>>>(
        src_rows, rows, nelem, static_cast<float2*>(dst_dev), dst_pitch);
    return cudaGetLastError() == cudaSuccess ? PNCE_OK : PNCE_ECUDA;
}

pnce_status pnce_scatter_rows(const void* src_dev, long long src_pitch, const uint64_t* dst_rows,
                              const int* counts, int rows, void* stream) {
    if (!src_dev || !dst_rows || !counts || rows < 0 || src_pitch < 0) return PNCE_EINVAL;
    if (((uintptr_t)src_dev & 7u) || ((uintptr_t)dst_rows & 7u) || ((uintptr_t)counts & 3u))
        return PNCE_EINVAL;
    if (rows == 0) return PNCE_OK;
    scatter_rows_kernel<<<rows, THREADS, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const float2*>(src_dev), src_pitch, dst_rows, counts, rows);
    return cudaGetLastError() == cudaSuccess ? PNCE_OK : PNCE_ECUDA;
}

}  // extern "C"
