// Row gather / scatter for batched serving.  A serving batch packs the antennas of several
// requests, each with its own received block and result buffer, into one contiguous
// estimate.  These kernels move rows between per-antenna addresses (typically page-locked
// host memory, read and written by the GPU directly over the host link) and the batch's
// contiguous device buffers, so a whole batch needs no per-request copy calls and its
// launch sequence can be captured once and replayed.  pnce_estimate_grouped does the whole
// batch in one call from a table of request descriptors (gather, estimate, scatter).  The
// contiguous copy-out kernel serves
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

// Grouped estimate: request b's rows m < M go to batch rows row_offset + m.  A descriptor
// that does not fit the batch (rows, kl_max) or has null buffers is skipped and latches
// PNCE_EINVAL; M = 0 marks an empty slot.  The rows are spread over the blocks one batch
// row per block (as many blocks as rows, like the row gather), through a row -> request
// map built on the device.
__device__ __forceinline__ bool desc_ok(const pnce_req_desc& q, int rows, int kl_max) {
    return q.M > 0 && q.row_offset >= 0 && (long long)q.row_offset + q.M <= rows && q.K >= 1 &&
           q.L >= 1 && (long long)q.K * q.L <= kl_max && q.Y != nullptr && q.H != nullptr;
}

// row_req[r] = the request that owns batch row r (-1 already written for every row)
__global__ void __launch_bounds__(THREADS)
grouped_map_kernel(const pnce_req_desc* __restrict__ d, int nreq, int rows, int kl_max,
                   int* __restrict__ row_req, int* err) {
    for (int b = blockIdx.x; b < nreq; b += gridDim.x) {
        const pnce_req_desc q = d[b];
        if (q.M <= 0) continue;
        if (!desc_ok(q, rows, kl_max)) {
            if (threadIdx.x == 0) atomicCAS(err, 0, (int)PNCE_EINVAL);
            continue;
        }
        for (int m = threadIdx.x; m < q.M; m += THREADS) row_req[q.row_offset + m] = b;
    }
}

__global__ void __launch_bounds__(THREADS)
grouped_gather_kernel(const pnce_req_desc* __restrict__ d, const int* __restrict__ row_req,
                      int N, float2* __restrict__ Yb) {
    const int r = blockIdx.x;
    const int b = row_req[r];
    if (b < 0) return;
    const pnce_req_desc& q = d[b];
    const float2* src = static_cast<const float2*>(q.Y) + (long long)(r - q.row_offset) * N;
    float2* dst = Yb + (long long)r * N;
    for (int n = threadIdx.x; n < N; n += THREADS) dst[n] = src[n];
}

__global__ void __launch_bounds__(THREADS)
grouped_scatter_kernel(const pnce_req_desc* __restrict__ d, const int* __restrict__ row_req,
                       int kl_max, const float2* __restrict__ Hb) {
    const int r = blockIdx.x;
    const int b = row_req[r];
    if (b < 0) return;
    const pnce_req_desc& q = d[b];
    const int kl = q.K * q.L;
    const float2* src = Hb + (long long)r * kl_max;
    float2* dst = static_cast<float2*>(q.H) + (long long)(r - q.row_offset) * kl;
    for (int j = threadIdx.x; j < kl; j += THREADS) dst[j] = src[j];
}

struct GroupedLayout {
    size_t d_off, m_off, y_off, h_off, q_off, total;
};

GroupedLayout grouped_layout(int rows, int N, int kl_max, int dtype) {
    GroupedLayout l{};
    l.d_off = 0;                                   // device copy of up to `rows` descriptors
    l.m_off = pnce::round_up((size_t)rows * sizeof(pnce_req_desc), 256);   // row -> request
    l.y_off = l.m_off + pnce::round_up((size_t)rows * sizeof(int), 256);
    l.h_off = l.y_off + pnce::round_up((size_t)rows * N * sizeof(float2), 256);
    l.q_off = l.h_off + pnce::round_up((size_t)rows * kl_max * sizeof(float2), 256);
    l.total = l.q_off;
    if (dtype != PNCE_FP32_SIMT) l.total += pnce::quant_layout(rows, N, dtype).total;
    return l;
}

bool grouped_shape_ok(int rows, int N, int kl_max, int dtype) {
    if (rows < 1 || N < 2 || kl_max < 1 || kl_max > N) return false;
    if ((long long)rows * N > (1LL << 36)) return false;
    return dtype == PNCE_FP32_SIMT || dtype == PNCE_TF32 || dtype == PNCE_FP16 ||
           dtype == PNCE_BF16 || dtype == PNCE_FP8E4M3;
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

size_t pnce_grouped_workspace_size(int rows, int N, int kl_max, int dtype) {
    if (!grouped_shape_ok(rows, N, kl_max, dtype)) return 0;
    return grouped_layout(rows, N, kl_max, dtype).total;
}

pnce_status pnce_estimate_grouped(pnce_handle* h, const pnce_pilot* pilot,
                                  const pnce_req_desc* descs, int nreq, int rows, int kl_max,
                                  int dtype, void* workspace_dev, size_t workspace_bytes,
                                  void* stream) {
    if (!h || !pilot || !workspace_dev || nreq < 0 || (nreq > 0 && !descs)) return PNCE_EINVAL;
    if (!grouped_shape_ok(rows, pilot->N, kl_max, dtype) || nreq > rows) return PNCE_EINVAL;
    if ((uintptr_t)workspace_dev & 255u) return PNCE_EINVAL;
    const GroupedLayout lay = grouped_layout(rows, pilot->N, kl_max, dtype);
    if (workspace_bytes < lay.total) return PNCE_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return PNCE_ECUDA;
    if (dev != h->device || pilot->device != h->device) return PNCE_ESTATE;
    if (dtype != PNCE_FP32_SIMT && !(h->cc_major == 10 && h->cc_minor == 3))
        return PNCE_EUNSUPPORTED;
    if (nreq == 0) return PNCE_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int N = pilot->N;
    unsigned char* ws = static_cast<unsigned char*>(workspace_dev);
    float2* Yb = reinterpret_cast<float2*>(ws + lay.y_off);
    float2* Hb = reinterpret_cast<float2*>(ws + lay.h_off);
    // the table comes over once (one copy; from page-locked host memory it is a graph
    // node like any other), so that the blocks read their descriptors from device memory
    pnce_req_desc* dd = reinterpret_cast<pnce_req_desc*>(ws + lay.d_off);
    if (cudaMemcpyAsync(dd, descs, sizeof(pnce_req_desc) * (size_t)nreq, cudaMemcpyDefault,
                        s) != cudaSuccess)
        return PNCE_ECUDA;
    int* row_req = reinterpret_cast<int*>(ws + lay.m_off);
    if (cudaMemsetAsync(row_req, 0xff, sizeof(int) * (size_t)rows, s) != cudaSuccess)
        return PNCE_ECUDA;
    const int gm = nreq < 2 * h->num_sms ? nreq : 2 * h->num_sms;
    grouped_map_kernel<<<gm, THREADS, 0, s>>>(dd, nreq, rows, kl_max, row_req, h->status_dev);
    grouped_gather_kernel<<<rows, THREADS, 0, s>>>(dd, row_req, N, Yb);
    if (cudaGetLastError() != cudaSuccess) return PNCE_ECUDA;
    if (dtype == PNCE_FP32_SIMT) {
        pnce::TraceScope tr(h, s, pnce::TRACE_SIMT);
        if (pnce::launch_simt_bits(pilot, Yb, rows, N, kl_max, Hb, s) != cudaSuccess)
            return PNCE_ECUDA;
    } else {
        const pnce::QuantLayout ql = pnce::quant_layout(rows, N, dtype);
        void* q = ws + lay.q_off;
        {
            pnce::TraceScope tr(h, s, pnce::TRACE_QUANTIZE);
            if (pnce::launch_quantize(Yb, rows, N, dtype, pnce::ws_operand(q, ql),
                                      pnce::ws_factors(q, ql), nullptr, nullptr, s) != cudaSuccess)
                return PNCE_ECUDA;
        }
        pnce::TraceScope tr(h, s, pnce::TRACE_CORRELATE);
        const pnce_status st = pnce::launch_tc(h, pilot, rows, N, kl_max, dtype,
                                               pnce::ws_operand(q, ql), pnce::ws_factors(q, ql),
                                               Hb, s);
        if (st != PNCE_OK) return st;
    }
    grouped_scatter_kernel<<<rows, THREADS, 0, s>>>(dd, row_req, kl_max, Hb);
    return cudaGetLastError() == cudaSuccess ? PNCE_OK : PNCE_ECUDA;
}

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
