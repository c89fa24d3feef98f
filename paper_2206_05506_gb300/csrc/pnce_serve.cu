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
           q.L >= 1 && (long long)q.K * q.L <= kl_max && q.Y != nullptr && q.H != nullptr &&
           ((uintptr_t)q.Y & 7u) == 0 && ((uintptr_t)q.H & 7u) == 0;
}

constexpr int PREP_THREADS = 1024;

// One block: copies the descriptor table (device or page-locked host memory) into the
// workspace, clears the row -> request map, then lets each valid request claim its rows.
// A row claimed twice (overlapping row ranges) latches PNCE_EINVAL; the first claim keeps
// it.  One kernel in place of a table copy, a memset and a map kernel: fewer graph nodes
// on the latency path of a serving batch.
__global__ void __launch_bounds__(PREP_THREADS)
grouped_prep_kernel(const pnce_req_desc* __restrict__ src, int nreq, int rows, int kl_max,
                    pnce_req_desc* __restrict__ dd, int* __restrict__ row_req, int* err) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    for (int b = threadIdx.x; b < nreq; b += PREP_THREADS) dd[b] = src[b];
    for (int r = threadIdx.x; r < rows; r += PREP_THREADS) row_req[r] = -1;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = warp; b < nreq; b += PREP_THREADS / 32) {
        const pnce_req_desc q = dd[b];
        if (q.M <= 0) continue;
        if (!desc_ok(q, rows, kl_max)) {
            if (lane == 0) atomicCAS(err, 0, (int)PNCE_EINVAL);
            continue;
        }
        bool clash = false;
        for (int m = lane; m < q.M; m += 32)
            clash |= atomicCAS(&row_req[q.row_offset + m], -1, b) != -1;
        if (__any_sync(0xffffffffu, clash) && lane == 0) atomicCAS(err, 0, (int)PNCE_EINVAL);
    }
}

// FP32 path: the rows move into the batch buffer first (the SIMT kernel reads rows at a
// fixed pitch).  A programmatic dependent of the prep kernel.
__global__ void __launch_bounds__(THREADS)
grouped_gather_kernel(const pnce_req_desc* __restrict__ d, const int* __restrict__ row_req,
                      int N, float2* __restrict__ Yb) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int r = blockIdx.x;
    const int b = row_req[r];
    if (b < 0) return;
    const pnce_req_desc& q = d[b];
    const float2* src = static_cast<const float2*>(q.Y) + (long long)(r - q.row_offset) * N;
    float2* dst = Yb + (long long)r * N;
    for (int n = threadIdx.x; n < N; n += THREADS) dst[n] = src[n];
}

// A programmatic dependent of the correlation: waits for it, then moves every row's first
// K*L lags into its request's result.
__global__ void __launch_bounds__(THREADS)
grouped_scatter_kernel(const pnce_req_desc* __restrict__ d, const int* __restrict__ row_req,
                       int kl_max, const float2* __restrict__ Hb) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int r = blockIdx.x;
    const int b = row_req[r];
    if (b < 0) return;
    const pnce_req_desc& q = d[b];
    const int kl = q.K * q.L;
    const float2* src = Hb + (long long)r * kl_max;
    float2* dst = static_cast<float2*>(q.H) + (long long)(r - q.row_offset) * kl;
    // 16-byte stores from the first 16-byte boundary of the destination on (its rows of
    // odd K*L start half-way into one every other row), loads of up to four pairs issued
    // before the stores
    const int head = ((uintptr_t)dst & 15u) ? 1 : 0;
    const int npairs = (kl - head) >> 1;
    float4* dpairs = reinterpret_cast<float4*>(dst + head);
    for (int i0 = threadIdx.x; i0 < npairs; i0 += 4 * THREADS) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * THREADS;
            if (i < npairs) {
                const float2 x0 = src[head + 2 * i], x1 = src[head + 2 * i + 1];
                v[u] = make_float4(x0.x, x0.y, x1.x, x1.y);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * THREADS;
            if (i < npairs) dpairs[i] = v[u];
        }
    }
    if (threadIdx.x == 0 && head) dst[0] = src[0];
    if (threadIdx.x == 1 && ((kl - head) & 1)) dst[kl - 1] = src[kl - 1];
}

template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kern)(KArgs...), unsigned grid, unsigned block,
                             cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(block, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

struct GroupedLayout {
    size_t d_off, m_off, y_off, h_off, q_off, total;
};

GroupedLayout grouped_layout(int rows, int N, int kl_max, int dtype) {
    GroupedLayout l{};
    l.d_off = 0;                                   // device copy of up to `rows` descriptors
    l.m_off = pnce::round_up((size_t)rows * sizeof(pnce_req_desc), 256);   // row -> request
    l.y_off = l.m_off + pnce::round_up((size_t)rows * sizeof(int), 256);
    // the batch copy of Y exists only for the FP32 path (the quantiser reads the rows
    // from the requests' buffers directly)
    const size_t y_bytes = dtype == PNCE_FP32_SIMT ? (size_t)rows * N * sizeof(float2) : 0;
    l.h_off = l.y_off + pnce::round_up(y_bytes, 256);
    l.q_off = l.h_off + pnce::round_up((size_t)rows * kl_max * sizeof(float2), 256);
    l.total = l.q_off;
    if (dtype != PNCE_FP32_SIMT) l.total += pnce::quant_layout(rows, N, dtype).total;
    return l;
}

bool grouped_shape_ok(int rows, int N, int kl_max, int dtype) {
    if (rows < 1 || N < 2 || kl_max < 1 || kl_max > N) return false;
    dtype = pnce::resolve_dtype(dtype, kl_max);
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
    return grouped_layout(rows, N, kl_max, pnce::resolve_dtype(dtype, kl_max)).total;
}

pnce_status pnce_estimate_grouped(pnce_handle* h, const pnce_pilot* pilot,
                                  const pnce_req_desc* descs, int nreq, int rows, int kl_max,
                                  int dtype, void* workspace_dev, size_t workspace_bytes,
                                  void* stream) {
    if (!h || !pilot || !workspace_dev || nreq < 0 || (nreq > 0 && !descs)) return PNCE_EINVAL;
    if (!grouped_shape_ok(rows, pilot->N, kl_max, dtype) || nreq > rows) return PNCE_EINVAL;
    if ((uintptr_t)workspace_dev & 255u) return PNCE_EINVAL;
    if ((uintptr_t)descs & 7u) return PNCE_EINVAL;
    dtype = pnce::resolve_dtype(dtype, kl_max);
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
    float2* Hb = reinterpret_cast<float2*>(ws + lay.h_off);
    pnce_req_desc* dd = reinterpret_cast<pnce_req_desc*>(ws + lay.d_off);
    int* row_req = reinterpret_cast<int*>(ws + lay.m_off);
    // prep (table copy + row map), then every kernel as a programmatic dependent of the one
    // before it: four graph nodes on the tensor-core path (prep, gather-quantise,
    // correlation, scatter), two or three on the FP32 path (prep, a row gather when the lags
    // span several tiles, the correlation writing into the requests' results)
    grouped_prep_kernel<<<1, PREP_THREADS, 0, s>>>(descs, nreq, rows, kl_max, dd, row_req,
                                                   h->status_dev);
    if (cudaGetLastError() != cudaSuccess) return PNCE_ECUDA;
    if (dtype == PNCE_FP32_SIMT) {
        float2* Yb = reinterpret_cast<float2*>(ws + lay.y_off);
        if (pnce::simt_grouped_ok(N, kl_max)) {
            // the SIMT kernel writes each row's lags into its request; it reads the rows
            // from the requests too when one lag tile covers kl_max, else from a row gather
            const bool direct = pnce::simt_grouped_reads_rows(kl_max);
            if (!direct && launch_dependent(grouped_gather_kernel, (unsigned)rows, THREADS, s,
                                            (const pnce_req_desc*)dd, (const int*)row_req, N,
                                            Yb) != cudaSuccess)
                return PNCE_ECUDA;
            pnce::TraceScope tr(h, s, pnce::TRACE_SIMT);
            return pnce::launch_simt_grouped(pilot, dd, row_req, rows, N, kl_max,
                                             direct ? nullptr : Yb, s, !h->trace_on) ==
                           cudaSuccess
                       ? PNCE_OK
                       : PNCE_ECUDA;
        }
        if (launch_dependent(grouped_gather_kernel, (unsigned)rows, THREADS, s,
                             (const pnce_req_desc*)dd, (const int*)row_req, N, Yb) != cudaSuccess)
            return PNCE_ECUDA;
        pnce::TraceScope tr(h, s, pnce::TRACE_SIMT);
        if (pnce::launch_simt_bits(pilot, Yb, rows, N, kl_max, Hb, s) != cudaSuccess)
            return PNCE_ECUDA;
    } else {
        const pnce::QuantLayout ql = pnce::quant_layout(rows, N, dtype);
        void* q = ws + lay.q_off;
        {
            pnce::TraceScope tr(h, s, pnce::TRACE_QUANTIZE);
            if (pnce::launch_quantize_grouped(dd, row_req, rows, N, dtype, pnce::ws_operand(q, ql),
                                              pnce::ws_factors(q, ql), s) != cudaSuccess)
                return PNCE_ECUDA;
        }
        pnce::TraceScope tr(h, s, pnce::TRACE_CORRELATE);
        const pnce_status st = pnce::launch_tc(h, pilot, rows, N, kl_max, dtype,
                                               pnce::ws_operand(q, ql), pnce::ws_factors(q, ql),
                                               Hb, s, /*pdl=*/!h->trace_on);
        if (st != PNCE_OK) return st;
    }
    return launch_dependent(grouped_scatter_kernel, (unsigned)rows, THREADS, s,
                            (const pnce_req_desc*)dd, (const int*)row_req, kl_max,
                            (const float2*)Hb) == cudaSuccess
               ? PNCE_OK
               : PNCE_ECUDA;
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
