// C ABI of libpnce: argument validation, handle / pilot objects and dispatch to the
// kernels.  Nothing here computes the estimate; every step of it runs in the kernels.
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "pnce_internal.h"

namespace {

constexpr long long kMaxN = (1LL << 24) - 1;

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool shape_ok(int F, int M, int N, int K, int L) {
    if (F < 1 || M < 1 || N < 2 || K < 1 || L < 1) return false;
    if ((long long)N > kMaxN) return false;
    if ((long long)K * L > N) return false;           // Eq. 7: shifts must not alias
    const long long A = (long long)F * M;
    if (A > (1LL << 31) - 1) return false;
    if (A * (long long)N > (1LL << 40)) return false; // 8 TB of Y: surely a caller error
    return true;
}

bool is_tc(int dtype) {
    return dtype == PNCE_TF32 || dtype == PNCE_FP16 || dtype == PNCE_BF16 ||
           dtype == PNCE_FP8E4M3;
}

pnce_status check_device(const pnce_handle* h) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return PNCE_ECUDA;
    return dev == h->device ? PNCE_OK : PNCE_ESTATE;
}

pnce_status from_cuda(cudaError_t e) { return e == cudaSuccess ? PNCE_OK : PNCE_ECUDA; }

// Frame chunks for pnce_estimate.  Off by default: the quantiser of a batch runs, then the
// tensor-core correlation.  PNCE_OVERLAP_CHUNKS=n (2..8) splits a large batch into n frame
// chunks and quantises chunk i+1 on one handle stream while chunk i is correlated on
// another.  Measured on GB300 (512 x 128 x 4095, fp16): 1.460 ms per estimate
// sequential, 1.493 / 1.440 / 1.431 / 1.567 ms with 2 / 3 / 4 / 6 chunks -- the quantiser
// and the correlation compete for the SMs' L1/shared-memory data path, so overlapping buys
// at most 2 %, and only when each chunk keeps >= 8 waves of 128 x 256 tiles.  Chunks must
// hold whole 8-antenna operand groups.
int estimate_chunks(const pnce_handle* h, int F, int M, int N, int KL) {
    (void)N;
    const char* e = getenv("PNCE_OVERLAP_CHUNKS");
    long long n = e ? atoll(e) : 1;
    if (n <= 1) return 1;
    if (n > 8) n = 8;
    if ((((long long)F + n - 1) / n * M) % 8 != 0) return 1;
    const long long row_blocks_per_frame = (2LL * M + 127) / 128;
    const long long jt = (KL + 255) / 256;
    const long long tiles = (long long)F * row_blocks_per_frame * jt;
    const long long most = tiles / (8LL * h->num_sms);       // chunks of >= 8 waves
    if (n > most) n = most;
    if (n > F) n = F;
    return n < 2 ? 1 : (int)n;
}

pnce_status estimate_overlapped(pnce_handle* h, const pnce_pilot* pilot, const float2* Y, int F,
                                int M, int N, int KL, int dtype, void* ws, float2* H,
                                cudaStream_t user, int nch) {
    std::lock_guard<std::recursive_mutex> guard(h->lock);   // uses the handle's streams
    const long long A = (long long)F * M;
    const pnce::QuantLayout lay = pnce::quant_layout(A, N, dtype);
    unsigned char* operand = static_cast<unsigned char*>(pnce::ws_operand(ws, lay));
    float* factors = pnce::ws_factors(ws, lay);
    const size_t row_bytes = (size_t)pnce::row_pitch(N) * pnce::elem_bytes(dtype);
    // both pipeline streams start after the work already queued on the caller's stream
    if (cudaEventRecord(h->ev_est_start, user) != cudaSuccess ||
        cudaStreamWaitEvent(h->s_quant, h->ev_est_start, 0) != cudaSuccess ||
        cudaStreamWaitEvent(h->s_corr, h->ev_est_start, 0) != cudaSuccess)
        return PNCE_ECUDA;
    const int per = (F + nch - 1) / nch;
    int i = 0;
    for (int f0 = 0; f0 < F; f0 += per, ++i) {
        const int fc = (F - f0 < per) ? (F - f0) : per;
        const long long a0 = (long long)f0 * M, ac = (long long)fc * M;
        // chunk i owns operand rows [2 a0, 2 a0 + operand_rows(ac)) and factors [a0, a0 + ac)
        // of the whole-batch layout (a0 is a multiple of 8), so chunks never share memory
        void* op = operand + (size_t)(2 * a0) * row_bytes;
        float* fa = factors + a0;
        cudaError_t e;
        {
            pnce::TraceScope tr(h, h->s_quant, pnce::TRACE_QUANTIZE);
            e = pnce::launch_quantize(Y + a0 * N, ac, N, dtype, op, fa, nullptr, nullptr,
                                      h->s_quant);
        }
        if (e != cudaSuccess || cudaEventRecord(h->ev_q[i], h->s_quant) != cudaSuccess ||
            cudaStreamWaitEvent(h->s_corr, h->ev_q[i], 0) != cudaSuccess)
            return PNCE_ECUDA;
        pnce::TraceScope tr(h, h->s_corr, pnce::TRACE_CORRELATE);
        pnce_status st = pnce::launch_tc(h, pilot, ac, N, KL, dtype, op, fa, H + a0 * KL, h->s_corr);
        if (st != PNCE_OK) return st;
    }
    // the caller's stream resumes when both pipeline streams are done
    if (cudaEventRecord(h->ev_est_done[0], h->s_quant) != cudaSuccess ||
        cudaEventRecord(h->ev_est_done[1], h->s_corr) != cudaSuccess ||
        cudaStreamWaitEvent(user, h->ev_est_done[0], 0) != cudaSuccess ||
        cudaStreamWaitEvent(user, h->ev_est_done[1], 0) != cudaSuccess)
        return PNCE_ECUDA;
    return PNCE_OK;
}

}  // namespace

extern "C" {

int pnce_version(void) { return 1 * 10000 + 0 * 100 + 0; }

const char* pnce_status_string(pnce_status s) {
    switch (s) {
        case PNCE_OK: return "PNCE_OK";
        case PNCE_EINVAL: return "PNCE_EINVAL: invalid argument";
        case PNCE_EUNSUPPORTED: return "PNCE_EUNSUPPORTED: not supported on this device/build";
        case PNCE_ENOMEM: return "PNCE_ENOMEM: allocation failed";
        case PNCE_ECUDA: return "PNCE_ECUDA: CUDA runtime error";
        case PNCE_ETIMEOUT: return "PNCE_ETIMEOUT: device-side wait ran out";
        case PNCE_ESTATE: return "PNCE_ESTATE: wrong device or object mismatch";
        default: return "PNCE_?: unknown status";
    }
}

pnce_status pnce_create(pnce_handle** out) {
    if (!out) return PNCE_EINVAL;
    *out = nullptr;
    pnce_handle* h = new (std::nothrow) pnce_handle();
    if (!h) return PNCE_ENOMEM;
    cudaDeviceProp prop;
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaGetDeviceProperties(&prop, h->device) != cudaSuccess) {
        delete h;
        return PNCE_ECUDA;
    }
    h->num_sms = prop.multiProcessorCount;
    h->max_smem_optin = (int)prop.sharedMemPerBlockOptin;
    h->cc_major = prop.major;
    h->cc_minor = prop.minor;
    if (cudaMalloc(&h->status_dev, sizeof(int)) != cudaSuccess) {
        delete h;
        return PNCE_ENOMEM;
    }
    bool ok = cudaMemset(h->status_dev, 0, sizeof(int)) == cudaSuccess;
    const unsigned sf = cudaStreamNonBlocking;
    ok = ok && cudaStreamCreateWithFlags(&h->s_h2d, sf) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&h->s_comp, sf) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&h->s_d2h, sf) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&h->s_quant, sf) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&h->s_corr, sf) == cudaSuccess;
    const unsigned ef = cudaEventDisableTiming;
    for (int i = 0; i < 8 && ok; ++i)
        ok = ok && cudaEventCreateWithFlags(&h->ev_q[i], ef) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&h->ev_est_start, ef) == cudaSuccess;
    for (int i = 0; i < 2 && ok; ++i)
        ok = ok && cudaEventCreateWithFlags(&h->ev_est_done[i], ef) == cudaSuccess;
    for (int i = 0; i < kPnceHostSlots && ok; ++i) {
        ok = ok && cudaEventCreateWithFlags(&h->ev_in[i], ef) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&h->ev_comp[i], ef) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&h->ev_out[i], ef) == cudaSuccess;
    }
    ok = ok && cudaEventCreateWithFlags(&h->ev_start, ef) == cudaSuccess;
    for (int i = 0; i < 3 && ok; ++i)
        ok = ok && cudaEventCreateWithFlags(&h->ev_done[i], ef) == cudaSuccess;
    if (!ok) {
        pnce_destroy(h);
        return PNCE_ECUDA;
    }
    *out = h;
    return PNCE_OK;
}

pnce_status pnce_destroy(pnce_handle* h) {
    if (!h) return PNCE_EINVAL;
    for (cudaStream_t s : {h->s_h2d, h->s_comp, h->s_d2h, h->s_quant, h->s_corr})
        if (s) cudaStreamDestroy(s);
    for (int i = 0; i < 8; ++i)
        if (h->ev_q[i]) cudaEventDestroy(h->ev_q[i]);
    if (h->ev_est_start) cudaEventDestroy(h->ev_est_start);
    for (int i = 0; i < 2; ++i)
        if (h->ev_est_done[i]) cudaEventDestroy(h->ev_est_done[i]);
    for (int i = 0; i < kPnceHostSlots; ++i)
        for (cudaEvent_t e : {h->ev_in[i], h->ev_comp[i], h->ev_out[i]})
            if (e) cudaEventDestroy(e);
    if (h->ev_start) cudaEventDestroy(h->ev_start);
    for (int i = 0; i < 3; ++i)
        if (h->ev_done[i]) cudaEventDestroy(h->ev_done[i]);
    if (h->trace_ev) {
        for (int i = 0; i < 2 * pnce::kTraceMax; ++i)
            if (h->trace_ev[i]) cudaEventDestroy(h->trace_ev[i]);
        delete[] h->trace_ev;
        delete[] h->trace_kind;
    }
    if (h->status_dev) cudaFree(h->status_dev);
    delete h;
    return PNCE_OK;
}

pnce_status pnce_trace_enable(pnce_handle* h, int on) {
    if (!h) return PNCE_EINVAL;
    std::lock_guard<std::recursive_mutex> guard(h->lock);
    if (on && !h->trace_ev) {
        pnce_status st = check_device(h);
        if (st != PNCE_OK) return st;
        h->trace_ev = new (std::nothrow) cudaEvent_t[2 * pnce::kTraceMax]();
        h->trace_kind = new (std::nothrow) int[pnce::kTraceMax]();
        if (!h->trace_ev || !h->trace_kind) return PNCE_ENOMEM;
        for (int i = 0; i < 2 * pnce::kTraceMax; ++i)
            if (cudaEventCreate(&h->trace_ev[i]) != cudaSuccess) return PNCE_ECUDA;
    }
    h->trace_on = on ? 1 : 0;
    h->trace_n = 0;
    return PNCE_OK;
}

pnce_status pnce_trace_read(pnce_handle* h, int* kinds, float* ms, int max_entries, int* count) {
    if (!h || !count || max_entries < 0 || (max_entries > 0 && (!kinds || !ms)))
        return PNCE_EINVAL;
    *count = 0;
    std::lock_guard<std::recursive_mutex> guard(h->lock);
    if (!h->trace_ev) return PNCE_OK;
    const int n = h->trace_n < max_entries ? h->trace_n : max_entries;
    for (int i = 0; i < n; ++i) {
        if (cudaEventSynchronize(h->trace_ev[2 * i + 1]) != cudaSuccess) return PNCE_ECUDA;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, h->trace_ev[2 * i], h->trace_ev[2 * i + 1]) != cudaSuccess)
            return PNCE_ECUDA;
        kinds[i] = h->trace_kind[i];
        ms[i] = t;
    }
    *count = n;
    h->trace_n = 0;
    return PNCE_OK;
}

pnce_status pnce_get_status(pnce_handle* h, void* stream) {
    if (!h) return PNCE_EINVAL;
    pnce_status st = check_device(h);
    if (st != PNCE_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return PNCE_ECUDA;
    int v = 0;
    if (cudaMemcpy(&v, h->status_dev, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return PNCE_ECUDA;
    if (v != 0 && cudaMemset(h->status_dev, 0, sizeof(int)) != cudaSuccess) return PNCE_ECUDA;
    return static_cast<pnce_status>(v);
}

pnce_status pnce_pilot_create(pnce_handle* h, const uint32_t* bits_host, int N, pnce_pilot** out) {
    if (!h || !bits_host || !out || N < 2 || (long long)N > kMaxN) return PNCE_EINVAL;
    *out = nullptr;
    pnce_status st = check_device(h);
    if (st != PNCE_OK) return st;
    // wrapped table: bit t = bit (t mod N) for t < 32 * words, words = ceil(N/32) + 2, so that
    // any 32-bit window starting below N is readable from two consecutive words
    const int words = (N + 31) / 32 + 2;
    std::vector<uint32_t> ext;
    try {
        ext.assign((size_t)words, 0u);
    } catch (...) {
        return PNCE_ENOMEM;
    }
    for (long long t = 0; t < 32LL * words; ++t) {
        const long long n = t % N;
        const uint32_t b = (bits_host[n >> 5] >> (n & 31)) & 1u;
        ext[(size_t)(t >> 5)] |= b << (t & 31);
    }
    pnce_pilot* p = new (std::nothrow) pnce_pilot();
    if (!p) return PNCE_ENOMEM;
    p->device = h->device;
    p->N = N;
    p->ext_words = words;
    if (cudaMalloc(&p->ext_bits_dev, sizeof(uint32_t) * words) != cudaSuccess) {
        delete p;
        return PNCE_ENOMEM;
    }
    if (cudaMemcpy(p->ext_bits_dev, ext.data(), sizeof(uint32_t) * words,
                   cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(p->ext_bits_dev);
        delete p;
        return PNCE_ECUDA;
    }
    *out = p;
    return PNCE_OK;
}

pnce_status pnce_pilot_destroy(pnce_pilot* p) {
    if (!p) return PNCE_EINVAL;
    cudaFree(p->ext_bits_dev);
    delete p;
    return PNCE_OK;
}

int pnce_auto_dtype(int N, int K, int L) {
    if (!shape_ok(1, 1, N, K, L)) return -1;
    return pnce::resolve_dtype(PNCE_AUTO, (long long)K * L);
}

size_t pnce_workspace_size(int F, int M, int N, int K, int L, int dtype) {
    if (!shape_ok(F, M, N, K, L)) return 0;
    dtype = pnce::resolve_dtype(dtype, (long long)K * L);
    if (dtype == PNCE_FP32_SIMT) return 0;
    if (!is_tc(dtype)) return 0;
    return pnce::quant_layout((long long)F * M, N, dtype).total;
}

pnce_status pnce_quantize(pnce_handle* h, const void* Y_dev, int F, int M, int N, int dtype,
                          void* workspace_dev, size_t workspace_bytes, int32_t* exps_dev,
                          double* power_dev, void* stream) {
    if (!h || !Y_dev || !workspace_dev || !is_tc(dtype)) return PNCE_EINVAL;
    if (!shape_ok(F, M, N, 1, 1)) return PNCE_EINVAL;
    if (!aligned16(Y_dev) || !aligned16(workspace_dev)) return PNCE_EINVAL;
    const long long A = (long long)F * M;
    if (workspace_bytes < pnce::quant_layout(A, N, dtype).total) return PNCE_EINVAL;
    pnce_status st = check_device(h);
    if (st != PNCE_OK) return st;
    const pnce::QuantLayout lay = pnce::quant_layout(A, N, dtype);
    pnce::TraceScope tr(h, static_cast<cudaStream_t>(stream), pnce::TRACE_QUANTIZE);
    return from_cuda(pnce::launch_quantize(static_cast<const float2*>(Y_dev), A, N, dtype,
                                           pnce::ws_operand(workspace_dev, lay),
                                           pnce::ws_factors(workspace_dev, lay), exps_dev,
                                           power_dev, static_cast<cudaStream_t>(stream)));
}

pnce_status pnce_correlate_quantized(pnce_handle* h, const pnce_pilot* pilot, int F, int M, int N,
                                     int K, int L, int dtype, const void* workspace_dev,
                                     size_t workspace_bytes, void* H_dev, void* stream) {
    if (!h || !pilot || !workspace_dev || !H_dev || !is_tc(dtype)) return PNCE_EINVAL;
    if (!shape_ok(F, M, N, K, L)) return PNCE_EINVAL;
    if (!aligned16(workspace_dev) || !aligned16(H_dev)) return PNCE_EINVAL;
    const long long A = (long long)F * M;
    if (workspace_bytes < pnce::quant_layout(A, N, dtype).total) return PNCE_EINVAL;
    pnce_status st = check_device(h);
    if (st != PNCE_OK) return st;
    if (pilot->device != h->device || pilot->N != N) return PNCE_ESTATE;
    const pnce::QuantLayout lay = pnce::quant_layout(A, N, dtype);
    void* ws = const_cast<void*>(workspace_dev);
    pnce::TraceScope tr(h, static_cast<cudaStream_t>(stream), pnce::TRACE_CORRELATE);
    return pnce::launch_tc(h, pilot, A, N, K * L, dtype, pnce::ws_operand(ws, lay),
                           pnce::ws_factors(ws, lay), static_cast<float2*>(H_dev),
                           static_cast<cudaStream_t>(stream));
}

pnce_status pnce_estimate(pnce_handle* h, const pnce_pilot* pilot, const void* Y_dev, int F,
                          int M, int N, int K, int L, int dtype, void* workspace_dev,
                          size_t workspace_bytes, void* H_dev, void* stream) {
    if (!h || !pilot || !Y_dev || !H_dev) return PNCE_EINVAL;
    if (!shape_ok(F, M, N, K, L)) return PNCE_EINVAL;
    if (!aligned16(Y_dev) || !aligned16(H_dev)) return PNCE_EINVAL;
    dtype = pnce::resolve_dtype(dtype, (long long)K * L);
    if (dtype != PNCE_FP32_SIMT && !is_tc(dtype)) return PNCE_EINVAL;
    pnce_status st = check_device(h);
    if (st != PNCE_OK) return st;
    if (pilot->device != h->device || pilot->N != N) return PNCE_ESTATE;
    const long long A = (long long)F * M;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == PNCE_FP32_SIMT) {
        pnce::TraceScope tr(h, s, pnce::TRACE_SIMT);
        return from_cuda(pnce::launch_simt_bits(pilot, static_cast<const float2*>(Y_dev), A, N,
                                                K * L, static_cast<float2*>(H_dev), s));
    }
    if (!workspace_dev || !aligned16(workspace_dev)) return PNCE_EINVAL;
    if (workspace_bytes < pnce::quant_layout(A, N, dtype).total) return PNCE_EINVAL;
    if (!(h->cc_major == 10 && h->cc_minor == 3)) return PNCE_EUNSUPPORTED;
    const int nch = estimate_chunks(h, F, M, N, K * L);
    if (nch <= 1) {
        const pnce::QuantLayout lay = pnce::quant_layout(A, N, dtype);
        {
            pnce::TraceScope tr(h, s, pnce::TRACE_QUANTIZE);
            st = from_cuda(pnce::launch_quantize(static_cast<const float2*>(Y_dev), A, N, dtype,
                                                 pnce::ws_operand(workspace_dev, lay),
                                                 pnce::ws_factors(workspace_dev, lay), nullptr,
                                                 nullptr, s));
        }
        if (st != PNCE_OK) return st;
        pnce::TraceScope tr(h, s, pnce::TRACE_CORRELATE);
        return pnce::launch_tc(h, pilot, A, N, K * L, dtype, pnce::ws_operand(workspace_dev, lay),
                               pnce::ws_factors(workspace_dev, lay),
                               static_cast<float2*>(H_dev), s);
    }
    return estimate_overlapped(h, pilot, static_cast<const float2*>(Y_dev), F, M, N, K * L, dtype,
                               workspace_dev, static_cast<float2*>(H_dev), s, nch);
}

pnce_status pnce_estimate_ex(pnce_handle* h, const pnce_pilot* pilot, const void* Y_dev, int F,
                             int M, int N, int K, int L, int dtype, const pnce_frame_opts* opts,
                             void* workspace_dev, size_t workspace_bytes, void* H_dev,
                             void* stream) {
    if (!opts)
        return pnce_estimate(h, pilot, Y_dev, F, M, N, K, L, dtype, workspace_dev,
                             workspace_bytes, H_dev, stream);
    if (!h || !pilot || !Y_dev || !H_dev) return PNCE_EINVAL;
    if (opts->cp_len < 0 || (opts->shift_rule != PNCE_SHIFT_KL &&
                             opts->shift_rule != PNCE_SHIFT_SPREAD))
        return PNCE_EINVAL;
    if (!shape_ok(F, M, N, K, L)) return PNCE_EINVAL;
    if (opts->shift_rule == PNCE_SHIFT_SPREAD && L > N / K) return PNCE_EINVAL;
    if (!aligned16(Y_dev) || !aligned16(H_dev)) return PNCE_EINVAL;
    dtype = pnce::resolve_dtype(dtype, (long long)K * L);
    if (dtype != PNCE_FP32_SIMT && !is_tc(dtype)) return PNCE_EINVAL;
    pnce_status st = check_device(h);
    if (st != PNCE_OK) return st;
    if (pilot->device != h->device || pilot->N != N) return PNCE_ESTATE;
    const long long A = (long long)F * M;
    const long long stride = (long long)N + opts->cp_len;
    const float2* Y = static_cast<const float2*>(Y_dev) + opts->cp_len;
    const pnce::LagMap lm = opts->shift_rule == PNCE_SHIFT_KL
                                ? pnce::lagmap_contiguous(K * L)
                                : pnce::LagMap{1, K, L, N / K, K * L};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float2* H = static_cast<float2*>(H_dev);
    if (dtype == PNCE_FP32_SIMT) {
        pnce::TraceScope tr(h, s, pnce::TRACE_SIMT);
        return from_cuda(pnce::launch_simt_bits_ex(pilot, Y, stride, A, N, lm, H, s));
    }
    if (!workspace_dev || !aligned16(workspace_dev)) return PNCE_EINVAL;
    const pnce::QuantLayout lay = pnce::quant_layout(A, N, dtype);
    if (workspace_bytes < lay.total) return PNCE_EINVAL;
    if (!(h->cc_major == 10 && h->cc_minor == 3)) return PNCE_EUNSUPPORTED;
    {
        pnce::TraceScope tr(h, s, pnce::TRACE_QUANTIZE);
        st = from_cuda(pnce::launch_quantize(Y, A, N, dtype, pnce::ws_operand(workspace_dev, lay),
                                             pnce::ws_factors(workspace_dev, lay), nullptr,
                                             nullptr, s, 0, stride));
    }
    if (st != PNCE_OK) return st;
    pnce::TraceScope tr(h, s, pnce::TRACE_CORRELATE);
    return pnce::launch_tc_ex(h, pilot, A, N, lm, dtype, pnce::ws_operand(workspace_dev, lay),
                              pnce::ws_factors(workspace_dev, lay), H, s);
}

pnce_status pnce_estimate_real_pilot(pnce_handle* h, const float* p_dev, int pilot_map,
                                     const void* Y_dev, int F, int M, int N, int K, int L,
                                     void* H_dev, void* stream) {
    if (!h || !p_dev || !Y_dev || !H_dev) return PNCE_EINVAL;
    if (pilot_map != PNCE_PILOT_REAL && pilot_map != PNCE_PILOT_TANH) return PNCE_EINVAL;
    if (!shape_ok(F, M, N, K, L)) return PNCE_EINVAL;
    if (!aligned16(Y_dev) || !aligned16(H_dev) || !aligned16(p_dev)) return PNCE_EINVAL;
    pnce_status st = check_device(h);
    if (st != PNCE_OK) return st;
    pnce::TraceScope tr(h, static_cast<cudaStream_t>(stream), pnce::TRACE_SIMT);
    return from_cuda(pnce::launch_simt_real(p_dev, pilot_map == PNCE_PILOT_TANH,
                                            static_cast<const float2*>(Y_dev),
                                            (long long)F * M, N, K * L,
                                            static_cast<float2*>(H_dev),
                                            static_cast<cudaStream_t>(stream)));
}

size_t pnce_backward_workspace_size(int F, int M, int N, int K, int L) {
    if (!shape_ok(F, M, N, K, L)) return 0;
    return pnce::backward_workspace((long long)F * M, N, K * L);
}

pnce_status pnce_backward(pnce_handle* h, const float* p_dev, int pilot_map, const void* Y_dev,
                          const void* G_dev, int F, int M, int N, int K, int L, void* dY_dev,
                          float* dp_dev, void* workspace_dev, size_t workspace_bytes,
                          void* stream) {
    if (!h || !p_dev || !G_dev) return PNCE_EINVAL;
    if (pilot_map != PNCE_PILOT_REAL && pilot_map != PNCE_PILOT_TANH) return PNCE_EINVAL;
    if (!shape_ok(F, M, N, K, L)) return PNCE_EINVAL;
    if (!aligned16(p_dev) || !aligned16(G_dev)) return PNCE_EINVAL;
    if (dY_dev && !aligned16(dY_dev)) return PNCE_EINVAL;
    if (dp_dev) {
        if (!Y_dev || !aligned16(Y_dev) || !aligned16(dp_dev)) return PNCE_EINVAL;
        const size_t need = pnce::backward_workspace((long long)F * M, N, K * L);
        if (need > 0 && (!workspace_dev || !aligned16(workspace_dev) || workspace_bytes < need))
            return PNCE_EINVAL;
    }
    pnce_status st = check_device(h);
    if (st != PNCE_OK) return st;
    pnce::TraceScope tr(h, static_cast<cudaStream_t>(stream), pnce::TRACE_ADJOINT);
    return from_cuda(pnce::launch_backward(
        p_dev, pilot_map == PNCE_PILOT_TANH, static_cast<const float2*>(Y_dev),
        static_cast<const float2*>(G_dev),
        (long long)F * M, N, K * L, static_cast<float2*>(dY_dev), dp_dev, workspace_dev,
        workspace_bytes, static_cast<cudaStream_t>(stream)));
}

namespace {

// Host pipeline layout: frames go through in chunks of fc frames, kPnceHostSlots slots of
// (Y chunk, H chunk) so that copy-in of the next chunks and copy-out of the previous ones
// overlap the kernels of chunk i without waiting on each other slot by slot, plus the
// quantisation workspace of one chunk.
struct HostLayout {
    int fc;                        // frames per chunk
    size_t y_bytes, h_bytes;       // per slot
    size_t y_off[kPnceHostSlots], h_off[kPnceHostSlots], q_off, total;
};

HostLayout host_layout(int F, int M, int N, int K, int L, int dtype) {
    HostLayout l{};
    const size_t frame_y = (size_t)M * N * 8;
    const size_t target = (size_t)64 << 20;        // ~64 MB of Y per chunk
    long long fc = (long long)((target + frame_y - 1) / frame_y);
    const long long min_chunks = 4;                // enough chunks to overlap copy and compute
    if ((F + fc - 1) / fc < min_chunks) fc = (F + min_chunks - 1) / min_chunks;
    if (fc < 1) fc = 1;
    if (fc > F) fc = F;
    l.fc = (int)fc;
    l.y_bytes = pnce::round_up((size_t)fc * frame_y, 256);
    l.h_bytes = pnce::round_up((size_t)fc * M * (size_t)K * L * 8, 256);
    size_t off = 0;
    for (int b = 0; b < kPnceHostSlots; ++b) {
        l.y_off[b] = off;
        off += l.y_bytes;
        l.h_off[b] = off;
        off += l.h_bytes;
    }
    l.q_off = off;
    if (dtype != PNCE_FP32_SIMT) off += pnce::quant_layout((long long)fc * M, N, dtype).total;
    l.total = off;
    return l;
}

}  // namespace

size_t pnce_host_workspace_size(int F, int M, int N, int K, int L, int dtype) {
    if (!shape_ok(F, M, N, K, L)) return 0;
    dtype = pnce::resolve_dtype(dtype, (long long)K * L);
    if (dtype != PNCE_FP32_SIMT && !is_tc(dtype)) return 0;
    return host_layout(F, M, N, K, L, dtype).total;
}

pnce_status pnce_estimate_host(pnce_handle* h, const pnce_pilot* pilot, const void* Y_host, int F,
                               int M, int N, int K, int L, int dtype, void* workspace_dev,
                               size_t workspace_bytes, void* H_host, void* stream) {
    if (!h || !pilot || !Y_host || !H_host || !workspace_dev) return PNCE_EINVAL;
    if (!shape_ok(F, M, N, K, L)) return PNCE_EINVAL;
    dtype = pnce::resolve_dtype(dtype, (long long)K * L);
    if (dtype != PNCE_FP32_SIMT && !is_tc(dtype)) return PNCE_EINVAL;
    if (!aligned16(workspace_dev)) return PNCE_EINVAL;
    const HostLayout lay = host_layout(F, M, N, K, L, dtype);
    if (workspace_bytes < lay.total) return PNCE_EINVAL;
    pnce_status st = check_device(h);
    if (st != PNCE_OK) return st;
    if (pilot->device != h->device || pilot->N != N) return PNCE_ESTATE;
    if (dtype != PNCE_FP32_SIMT && !(h->cc_major == 10 && h->cc_minor == 3))
        return PNCE_EUNSUPPORTED;

    // copy-out: into page-locked H_host by a kernel (it shares the host link with the
    // copy-in DMA better than a second DMA does); into pageable memory by cudaMemcpyAsync
    unsigned char* h_mapped = nullptr;
    {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, H_host) == cudaSuccess) {
            if (at.type == cudaMemoryTypeHost && at.devicePointer != nullptr &&
                ((uintptr_t)at.devicePointer & 7u) == 0)
                h_mapped = static_cast<unsigned char*>(at.devicePointer);
        } else {
            cudaGetLastError();                  // unknown pointer: take the copy path
        }
    }

    std::lock_guard<std::recursive_mutex> guard(h->lock);   // uses the handle's streams
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    unsigned char* ws = static_cast<unsigned char*>(workspace_dev);
    const unsigned char* yh = static_cast<const unsigned char*>(Y_host);
    unsigned char* hh = static_cast<unsigned char*>(H_host);
    const size_t frame_y = (size_t)M * N * 8, frame_h = (size_t)M * K * L * 8;

    // the pipeline starts after the work already queued on the caller's stream
    if (cudaEventRecord(h->ev_start, user) != cudaSuccess) return PNCE_ECUDA;
    // Host-side fault injection for the test of the join below: PNCE_TEST_HOST_FAIL_CHUNK=i
    // makes the call give up with PNCE_ECUDA when it reaches chunk i, as a failed launch
    // or copy there would.
    const char* fail_env = getenv("PNCE_TEST_HOST_FAIL_CHUNK");
    const long long fail_at = fail_env ? atoll(fail_env) : -1;
    auto run = [&]() -> pnce_status {
        for (cudaStream_t s : {h->s_h2d, h->s_comp, h->s_d2h})
            if (cudaStreamWaitEvent(s, h->ev_start, 0) != cudaSuccess) return PNCE_ECUDA;
        for (int f0 = 0, i = 0; f0 < F; f0 += lay.fc, ++i) {
            if (i == fail_at) return PNCE_ECUDA;
            const int b = i % kPnceHostSlots;
            const int fc = (F - f0 < lay.fc) ? (F - f0) : lay.fc;
            void* yd = ws + lay.y_off[b];
            void* hd = ws + lay.h_off[b];
            // copy-in: slot b is free once the kernels of its previous chunk have read it
            if (i >= kPnceHostSlots &&
                cudaStreamWaitEvent(h->s_h2d, h->ev_comp[b], 0) != cudaSuccess)
                return PNCE_ECUDA;
            if (cudaMemcpyAsync(yd, yh + (size_t)f0 * frame_y, (size_t)fc * frame_y,
                                cudaMemcpyHostToDevice, h->s_h2d) != cudaSuccess ||
                cudaEventRecord(h->ev_in[b], h->s_h2d) != cudaSuccess)
                return PNCE_ECUDA;
            // kernels: need the input, and H slot b drained by the copy-out of its previous
            // chunk
            if (cudaStreamWaitEvent(h->s_comp, h->ev_in[b], 0) != cudaSuccess) return PNCE_ECUDA;
            if (i >= kPnceHostSlots &&
                cudaStreamWaitEvent(h->s_comp, h->ev_out[b], 0) != cudaSuccess)
                return PNCE_ECUDA;
            const long long A = (long long)fc * M;
            pnce_status cst;
            if (dtype == PNCE_FP32_SIMT) {
                cst = from_cuda(pnce::launch_simt_bits(pilot, static_cast<const float2*>(yd), A,
                                                       N, K * L, static_cast<float2*>(hd),
                                                       h->s_comp));
            } else {
                const pnce::QuantLayout ql = pnce::quant_layout(A, N, dtype);
                void* q = ws + lay.q_off;
                cst = from_cuda(pnce::launch_quantize(static_cast<const float2*>(yd), A, N,
                                                      dtype, pnce::ws_operand(q, ql),
                                                      pnce::ws_factors(q, ql), nullptr, nullptr,
                                                      h->s_comp));
                if (cst == PNCE_OK)
                    cst = pnce::launch_tc(h, pilot, A, N, K * L, dtype, pnce::ws_operand(q, ql),
                                          pnce::ws_factors(q, ql), static_cast<float2*>(hd),
                                          h->s_comp);
            }
            if (cst != PNCE_OK) return cst;
            if (cudaEventRecord(h->ev_comp[b], h->s_comp) != cudaSuccess) return PNCE_ECUDA;
            // copy-out
            if (cudaStreamWaitEvent(h->s_d2h, h->ev_comp[b], 0) != cudaSuccess)
                return PNCE_ECUDA;
            const cudaError_t ce =
                h_mapped ? pnce::launch_copy_to_host(hd, h_mapped + (size_t)f0 * frame_h,
                                                     (size_t)fc * frame_h, h->num_sms, h->s_d2h)
                         : cudaMemcpyAsync(hh + (size_t)f0 * frame_h, hd, (size_t)fc * frame_h,
                                           cudaMemcpyDeviceToHost, h->s_d2h);
            if (ce != cudaSuccess || cudaEventRecord(h->ev_out[b], h->s_d2h) != cudaSuccess)
                return PNCE_ECUDA;
        }
        return PNCE_OK;
    };
    st = run();
    // The caller's stream resumes when all three pipeline streams are done -- after an
    // error part way too, so that a caller who synchronises its stream and then frees or
    // reuses the buffers never races with copies or kernels of earlier chunks still in
    // flight on the handle's streams.
    cudaStream_t ss[3] = {h->s_h2d, h->s_comp, h->s_d2h};
    for (int k = 0; k < 3; ++k) {
        if (cudaEventRecord(h->ev_done[k], ss[k]) != cudaSuccess ||
            cudaStreamWaitEvent(user, h->ev_done[k], 0) != cudaSuccess)
            if (st == PNCE_OK) st = PNCE_ECUDA;
    }
    return st;
}

}  // extern "C"
