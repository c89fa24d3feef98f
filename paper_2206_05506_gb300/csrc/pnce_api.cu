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
    if (cudaMemset(h->status_dev, 0, sizeof(int)) != cudaSuccess) {
        cudaFree(h->status_dev);
        delete h;
        return PNCE_ECUDA;
    }
    *out = h;
    return PNCE_OK;
}

pnce_status pnce_destroy(pnce_handle* h) {
    if (!h) return PNCE_EINVAL;
    cudaFree(h->status_dev);
    delete h;
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
    std::vector<uint32_t> ext((size_t)words, 0u);
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

size_t pnce_workspace_size(int F, int M, int N, int K, int L, int dtype) {
    if (!shape_ok(F, M, N, K, L)) return 0;
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
    return from_cuda(pnce::launch_quantize(static_cast<const float2*>(Y_dev), A, N, dtype,
                                           workspace_dev, exps_dev, power_dev,
                                           static_cast<cudaStream_t>(stream)));
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
    return pnce::launch_tc(h, pilot, A, N, K * L, dtype, workspace_dev,
                           static_cast<float2*>(H_dev), static_cast<cudaStream_t>(stream));
}

pnce_status pnce_estimate(pnce_handle* h, const pnce_pilot* pilot, const void* Y_dev, int F,
                          int M, int N, int K, int L, int dtype, void* workspace_dev,
                          size_t workspace_bytes, void* H_dev, void* stream) {
    if (!h || !pilot || !Y_dev || !H_dev) return PNCE_EINVAL;
    if (!shape_ok(F, M, N, K, L)) return PNCE_EINVAL;
    if (!aligned16(Y_dev) || !aligned16(H_dev)) return PNCE_EINVAL;
    if (dtype != PNCE_FP32_SIMT && !is_tc(dtype)) return PNCE_EINVAL;
    pnce_status st = check_device(h);
    if (st != PNCE_OK) return st;
    if (pilot->device != h->device || pilot->N != N) return PNCE_ESTATE;
    const long long A = (long long)F * M;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == PNCE_FP32_SIMT) {
        return from_cuda(pnce::launch_simt_bits(pilot, static_cast<const float2*>(Y_dev), A, N,
                                                K * L, static_cast<float2*>(H_dev), s));
    }
    if (!workspace_dev || !aligned16(workspace_dev)) return PNCE_EINVAL;
    if (workspace_bytes < pnce::quant_layout(A, N, dtype).total) return PNCE_EINVAL;
    if (!(h->cc_major == 10 && h->cc_minor == 3)) return PNCE_EUNSUPPORTED;
    st = from_cuda(pnce::launch_quantize(static_cast<const float2*>(Y_dev), A, N, dtype,
                                         workspace_dev, nullptr, nullptr, s));
    if (st != PNCE_OK) return st;
    return pnce::launch_tc(h, pilot, A, N, K * L, dtype, workspace_dev,
                           static_cast<float2*>(H_dev), s);
}

pnce_status pnce_estimate_real_pilot(pnce_handle* h, const float* p_dev, const void* Y_dev, int F,
                                     int M, int N, int K, int L, void* H_dev, void* stream) {
    if (!h || !p_dev || !Y_dev || !H_dev) return PNCE_EINVAL;
    if (!shape_ok(F, M, N, K, L)) return PNCE_EINVAL;
    if (!aligned16(Y_dev) || !aligned16(H_dev) || !aligned16(p_dev)) return PNCE_EINVAL;
    pnce_status st = check_device(h);
    if (st != PNCE_OK) return st;
    return from_cuda(pnce::launch_simt_real(p_dev, static_cast<const float2*>(Y_dev),
                                            (long long)F * M, N, K * L,
                                            static_cast<float2*>(H_dev),
                                            static_cast<cudaStream_t>(stream)));
}

size_t pnce_backward_workspace_size(int F, int M, int N, int K, int L) {
    if (!shape_ok(F, M, N, K, L)) return 0;
    return pnce::backward_workspace((long long)F * M, N, K * L);
}

pnce_status pnce_backward(pnce_handle* h, const float* p_dev, const void* Y_dev, const void* G_dev,
                          int F, int M, int N, int K, int L, void* dY_dev, float* dp_dev,
                          void* workspace_dev, size_t workspace_bytes, void* stream) {
    if (!h || !p_dev || !G_dev) return PNCE_EINVAL;
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
    return from_cuda(pnce::launch_backward(
        p_dev, static_cast<const float2*>(Y_dev), static_cast<const float2*>(G_dev),
        (long long)F * M, N, K * L, static_cast<float2*>(dY_dev), dp_dev, workspace_dev,
        workspace_bytes, static_cast<cudaStream_t>(stream)));
}

size_t pnce_host_workspace_size(int F, int M, int N, int K, int L, int dtype) {
    (void)F; (void)M; (void)N; (void)K; (void)L; (void)dtype;
    return 0;
}

pnce_status pnce_estimate_host(pnce_handle* h, const pnce_pilot* pilot, const void* Y_host, int F,
                               int M, int N, int K, int L, int dtype, void* workspace_dev,
                               size_t workspace_bytes, void* H_host, void* stream) {
    (void)h; (void)pilot; (void)Y_host; (void)F; (void)M; (void)N; (void)K; (void)L;
    (void)dtype; (void)workspace_dev; (void)workspace_bytes; (void)H_host; (void)stream;
    return PNCE_EUNSUPPORTED;
}

}  // extern "C"
