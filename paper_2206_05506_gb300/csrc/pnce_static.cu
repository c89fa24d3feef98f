// Allocation-free estimate: the tensor-core estimate with its scratch (the quantised
// operand and the per-antenna output factors) in a fixed device array that is part of the
// library image, so the call itself never allocates.  Meant for callers that cannot call
// cudaMalloc on their path: real-time receive pipelines that must not hit the allocator
// (its latency is unbounded and it may synchronise the device), and hosts that hand the
// library a fixed memory budget with no allocator at all.
#include <mutex>

#include "pnce_internal.h"

namespace {

// The scratch array.  Every device on which the library's module is loaded reserves
// PNCE_STATIC_SCRATCH_BYTES for it until the process exits.  In host code the name
// g_static_scratch is only a host-side stand-in: its device address comes from
// cudaGetSymbolAddress, taken once per device below.
__device__ __align__(256) unsigned char g_static_scratch[PNCE_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `dev` (which must be the current device).  The
// first call on a device looks it up; later calls reuse it.
pnce_status scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return PNCE_EUNSUPPORTED;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return PNCE_ECUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return PNCE_OK;
}

}  // namespace

extern "C" pnce_status pnce_estimate_static(pnce_handle* h, const pnce_pilot* pilot,
                                            const void* Y_dev, int F, int M, int N, int K,
                                            int L, int dtype, void* H_dev, void* stream) {
    if (!h || !pilot || !Y_dev || !H_dev) return PNCE_EINVAL;
    if (dtype != PNCE_TF32 && dtype != PNCE_FP16 && dtype != PNCE_BF16 && dtype != PNCE_FP8E4M3)
        return PNCE_EINVAL;
    if (F < 1 || M < 1 || N < 2 || K < 1 || L < 1 || (long long)K * L > N) return PNCE_EINVAL;
    if (((uintptr_t)Y_dev & 15u) || ((uintptr_t)H_dev & 15u)) return PNCE_EINVAL;
    const long long A = (long long)F * M;
    if (A > (1LL << 31) - 1) return PNCE_EINVAL;
    // the quantised operand of this shape must fit the fixed scratch array
    if (pnce::quant_layout(A, N, dtype).total > (size_t)PNCE_STATIC_SCRATCH_BYTES)
        return PNCE_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return PNCE_ECUDA;
    if (dev != h->device || pilot->device != h->device) return PNCE_ESTATE;
    if (pilot->N != N) return PNCE_ESTATE;
    if (!(h->cc_major == 10 && h->cc_minor == 3)) return PNCE_EUNSUPPORTED;
    void* ws = nullptr;
    pnce_status st = scratch_address(dev, &ws);
    if (st != PNCE_OK) return st;
    // nothing in the scratch needs clearing: every row and factor the correlation reads is
    // rewritten by the quantiser first, and the pad columns past N are never read
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const pnce::QuantLayout lay = pnce::quant_layout(A, N, dtype);
    {
        pnce::TraceScope tr(h, s, pnce::TRACE_QUANTIZE);
        if (pnce::launch_quantize(static_cast<const float2*>(Y_dev), A, N, dtype,
                                  pnce::ws_operand(ws, lay), pnce::ws_factors(ws, lay), nullptr,
                                  nullptr, s) != cudaSuccess)
            return PNCE_ECUDA;
    }
    pnce::TraceScope tr(h, s, pnce::TRACE_CORRELATE);
    return pnce::launch_tc(h, pilot, A, N, K * L, dtype, pnce::ws_operand(ws, lay),
                           pnce::ws_factors(ws, lay), static_cast<float2*>(H_dev), s);
}
