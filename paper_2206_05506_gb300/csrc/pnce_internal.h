// Internal declarations shared by the translation units of libpnce (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "pnce.h"

// chunk slots of the host-buffer pipeline (pnce_estimate_host)
constexpr int kPnceHostSlots = 3;

struct pnce_handle {
    int device;
    int num_sms;
    int max_smem_optin;
    int cc_major, cc_minor;
    int* status_dev;                    // latched device-side status word
    // host-buffer pipeline (pnce_estimate_host): copy-in, compute and copy-out streams,
    // and per double-buffer slot events
    cudaStream_t s_h2d, s_comp, s_d2h;
    cudaEvent_t ev_in[kPnceHostSlots], ev_comp[kPnceHostSlots], ev_out[kPnceHostSlots];
    cudaEvent_t ev_start, ev_done[3];
    // pnce_estimate on large batches: quantisation of frame chunk i+1 (s_quant) overlaps
    // the tensor-core correlation of chunk i (s_corr)
    cudaStream_t s_quant, s_corr;
    cudaEvent_t ev_q[8], ev_est_start, ev_est_done[2];
    // tracing (pnce_trace_enable): start/end events around each kernel the estimate entry
    // points launch, recorded on the stream the kernel runs on
    int trace_on;
    int trace_n;
    cudaEvent_t* trace_ev;              // 2 * kTraceMax events, created on first enable
    int* trace_kind;
    // serialises the host-side enqueue of the sections that use the handle's own streams,
    // events or trace record, so calls from several threads cannot interleave them
    std::recursive_mutex lock;
};

namespace pnce {
// PNCE_AUTO: exact FP32 on the CUDA cores up to this many lags, FP16 tensor cores above
constexpr int kAutoSimtMaxLags = 16;
inline int resolve_dtype(int dtype, long long KL) {
    if (dtype != PNCE_AUTO) return dtype;
    return KL <= kAutoSimtMaxLags ? (int)PNCE_FP32_SIMT : (int)PNCE_FP16;
}
constexpr int kTraceMax = 8192;
enum TraceKind {
    TRACE_QUANTIZE = 0,
    TRACE_CORRELATE = 1,
    TRACE_SIMT = 2,
    TRACE_FMT = 3,
    TRACE_ADJOINT = 4,
};
// NVTX range names (profilers can filter launches by them)
inline const char* trace_name(int kind) {
    static const char* const names[] = {"pnce.quantize", "pnce.correlate", "pnce.simt",
                                        "pnce.fmt", "pnce.adjoint"};
    return kind >= 0 && kind <= TRACE_ADJOINT ? names[kind] : "pnce";
}
// Records a start event before / an end event after one kernel launch when tracing is on.
struct TraceScope {
    pnce_handle* h;
    cudaStream_t s;
    int slot;
    TraceScope(pnce_handle* h_, cudaStream_t s_, int kind) : h(h_), s(s_), slot(-1) {
        nvtxRangePushA(trace_name(kind));     // a no-op unless a profiler is attached
        if (h && h->trace_on) {
            std::lock_guard<std::recursive_mutex> g(h->lock);
            if (h->trace_n < kTraceMax) {
                slot = h->trace_n++;
                h->trace_kind[slot] = kind;
                cudaEventRecord(h->trace_ev[2 * slot], s);
            }
        }
    }
    ~TraceScope() {
        if (slot >= 0) cudaEventRecord(h->trace_ev[2 * slot + 1], s);
        nvtxRangePop();
    }
};
}  // namespace pnce

struct pnce_pilot {
    int device;
    int N;
    int ext_words;                      // words of the wrapped bit table
    uint32_t* ext_bits_dev;             // bit t = pilot bit (t mod N), t < 32 * ext_words
};

namespace pnce {

// Which correlation lags a launch computes and where they go in H.  Mode 0: the lags
// j = 0 .. ldH-1, stored at column j (transmitter k at cyclic shift k*L).  Mode 1:
// transmitter k at cyclic shift k*step; its lags k*step + l, l < L, stored at column
// k*L + l.  Kernels cut the lags into tiles of `tile` consecutive lags.
struct LagMap {
    int mode;
    int K, L;
    int step;
    int ldH;        // H row pitch in complex elements (= K*L)
};
inline LagMap lagmap_contiguous(int KL) { return LagMap{0, 1, KL, 0, KL}; }
__host__ __device__ inline long long lag_tiles(const LagMap& m, int tile) {
    return m.mode == 0 ? (m.ldH + tile - 1) / tile
                       : (long long)m.K * ((m.L + tile - 1) / tile);
}
// tile jt: first lag (origin), first output column and number of valid lags
__host__ __device__ inline void lag_tile(const LagMap& m, int tile, long long jt, long long& origin,
                                         int& col0, int& valid) {
    if (m.mode == 0) {
        origin = jt * tile;
        col0 = (int)origin;
        const int rest = m.ldH - col0;
        valid = rest < tile ? rest : tile;
    } else {
        const int tpk = (m.L + tile - 1) / tile;
        const int k = (int)(jt / tpk), lb = (int)(jt % tpk);
        origin = (long long)k * m.step + (long long)lb * tile;
        col0 = k * m.L + lb * tile;
        const int rest = m.L - lb * tile;
        valid = rest < tile ? rest : tile;
    }
}

// Elements of a quantised row are padded to a multiple of this (TMA row pitch).
constexpr int kRowPad = 64;

inline size_t round_up(size_t x, size_t m) { return (x + m - 1) / m * m; }
inline int row_pitch(int N) { return (int)round_up((size_t)N, kRowPad); }
int elem_bytes(int dtype);              // bytes per quantised element (0 for FP32_SIMT)

// Workspace carve-up for the tensor-core path.
// Operand row order: antennas in groups of 8, 16 rows per group -- the real parts of the
// group's 8 antennas, then their imaginary parts (so a 16-lane TMEM block of the product
// holds both parts of 8 antennas).  Rows of antennas >= A in the last group are zero.
__host__ __device__ inline long long operand_rows(long long A) { return 16 * ((A + 7) / 8); }
__host__ __device__ inline long long operand_row(long long a, int part) {
    return 16 * (a >> 3) + 8 * part + (a & 7);
}

struct QuantLayout {
    size_t a_offset, a_bytes;           // [operand_rows(A)][pitch] quantised operand
    size_t scale_offset;                // float[A]: 2^-s_a / N
    size_t total;
};
QuantLayout quant_layout(long long A, int N, int dtype);

// Launchers (return cudaSuccess or the launch error).
cudaError_t launch_simt_bits(const pnce_pilot* pilot, const float2* Y, long long A, int N,
                             int KL, float2* H, cudaStream_t s);
// general form: rows of Y y_stride elements apart (first sample at Y), lags per `lags`
// Serving batches on the FP32 path: batch row a is row a - row_offset of request
// dd[row_req[a]] (row_req < 0: no request); each row's first K*L lags are written into its
// request's H, and the rows are read from the requests' Y when Yb is null, else from Yb (a
// batch copy at pitch N).  simt_grouped_ok: where the warp kernel applies (kl_max > 32 and
// a pilot window within its shared-memory copy; cudaErrorNotSupported otherwise);
// simt_grouped_reads_rows: where reading from the requests pays (one lag tile covers
// kl_max).  pdl: launch as a programmatic dependent of the kernel before it.
bool simt_grouped_ok(int N, int kl_max);
bool simt_grouped_reads_rows(int kl_max);
cudaError_t launch_simt_grouped(const pnce_pilot* pilot, const pnce_req_desc* dd,
                                const int* row_req, long long rows, int N, int kl_max,
                                const float2* Yb, cudaStream_t s, bool pdl);
cudaError_t launch_simt_bits_ex(const pnce_pilot* pilot, const float2* Y, long long y_stride,
                                long long A, int N, const LagMap& lags, float2* H,
                                cudaStream_t s);
cudaError_t launch_simt_real(const float* p, bool tanh_map, const float2* Y, long long A, int N,
                             int KL, float2* H, cudaStream_t s);
// operand: [operand_rows(A)][row_pitch(N)] elements in operand_row order; factors:
// float[A] (2^-s_a / N).  max_blocks > 0
// caps the grid (blocks then loop over antennas), to leave room for a concurrent kernel.
cudaError_t launch_quantize(const float2* Y, long long A, int N, int dtype, void* operand,
                            float* factors, int32_t* exps, double* power, cudaStream_t s,
                            int max_blocks = 0, long long y_stride = 0 /* 0: N */);
// Serving batches: gather + quantise in one kernel (one block per batch row; a row's
// source comes from its request descriptor dd[row_req[row]]), launched as a programmatic
// dependent of the kernel before it.
cudaError_t launch_quantize_grouped(const pnce_req_desc* dd, const int* row_req, int rows, int N,
                                    int dtype, void* operand, float* factors, cudaStream_t s);
// status: PNCE_OK, or PNCE_ECUDA / PNCE_EUNSUPPORTED.  pdl: launch as a programmatic
// dependent of the kernel before it on the stream (the kernel's set-up -- barriers, TMEM,
// the resident pilot operand -- then overlaps that kernel's tail; it waits for it before
// touching the operand).
pnce_status launch_tc(const pnce_handle* h, const pnce_pilot* pilot, long long A, int N,
                      int KL, int dtype, const void* operand, const float* factors, float2* H,
                      cudaStream_t s, bool pdl = false);
pnce_status launch_tc_ex(const pnce_handle* h, const pnce_pilot* pilot, long long A, int N,
                         const LagMap& lags, int dtype, const void* operand,
                         const float* factors, float2* H, cudaStream_t s, bool pdl = false);
// the two pointers of a workspace laid out by quant_layout
inline void* ws_operand(void* ws, const QuantLayout& l) {
    return static_cast<unsigned char*>(ws) + l.a_offset;
}
inline float* ws_factors(void* ws, const QuantLayout& l) {
    return reinterpret_cast<float*>(static_cast<unsigned char*>(ws) + l.scale_offset);
}
cudaError_t launch_backward(const float* p, bool tanh_map, const float2* Y, const float2* G,
                            long long A, int N, int KL, float2* dY, float* dp, void* ws,
                            size_t ws_bytes, cudaStream_t s);
cudaError_t launch_adjoint_dy(const float* p, bool tanh_map, const float2* G, long long A, int N,
                              int KL, float2* dY, cudaStream_t s);
size_t backward_workspace(long long A, int N, int KL);
// copy `bytes` (a multiple of 8) from device memory into page-locked host memory with a
// kernel of at most num_sms blocks; dst must be the device-visible address of the
// page-locked buffer
cudaError_t launch_copy_to_host(const void* src_dev, void* dst_host_mapped, size_t bytes,
                                int num_sms, cudaStream_t s);

}  // namespace pnce
