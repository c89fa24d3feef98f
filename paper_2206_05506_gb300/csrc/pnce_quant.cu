// Reduced-precision operand for the tensor-core correlation (Sec. III-B: the received
// block is converted to the tensor cores' input format before the product).
//
// One block per antenna a: pass 1 reduces A_a = max |component| (FP32, exact) and, only
// when the caller asks for it, E_a = sum |y|^2 in FP64 (squares of FP32 values are exact
// in FP64; GB300's FP64 rate is low, so the estimate path does not request it); the
// power-of-two scale 2^s_a is taken from A_a; pass 2 re-reads the row (an L2 hit) and
// writes rows operand_row(a, 0) (real) and operand_row(a, 1) (imaginary) of
// round(y 2^s_a), four samples per thread per step.  Blocks past the last antenna zero
// the padding rows of the last 8-antenna group.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "pnce_internal.h"

namespace {

constexpr int THREADS = 256;

template <int DT> struct Fmt;
template <> struct Fmt<PNCE_FP16> { static constexpr int target = 15; using T = uint16_t; };
template <> struct Fmt<PNCE_BF16> { static constexpr int target = 0; using T = uint16_t; };
template <> struct Fmt<PNCE_TF32> { static constexpr int target = 0; using T = uint32_t; };
template <> struct Fmt<PNCE_FP8E4M3> { static constexpr int target = 8; using T = uint8_t; };

__device__ __forceinline__ uint16_t to_f16(float x) {
    return __half_as_ushort(__float2half_rn(x));
}
__device__ __forceinline__ uint16_t to_bf16(float x) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
// two e4m3 codes (lo from a, hi from b), round to nearest even, saturate to +-448
__device__ __forceinline__ uint16_t to_e4m3x2(float a, float b) {
    uint16_t r;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %2, %1;" : "=h"(r) : "f"(a), "f"(b));
    return r;
}

// write four consecutive converted values v[0..3] at element n of row `row`
template <int DT>
__device__ __forceinline__ void store4(void* base, long long row, int pitch, int n,
                                       const float v[4], int valid) {
    using T = typename Fmt<DT>::T;
    T* p = reinterpret_cast<T*>(base) + row * (long long)pitch + n;
    if constexpr (DT == PNCE_FP16 || DT == PNCE_BF16) {
        uint16_t c[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) c[i] = (DT == PNCE_FP16) ? to_f16(v[i]) : to_bf16(v[i]);
        if (valid == 4) {
            uint2 w;
            w.x = c[0] | ((uint32_t)c[1] << 16);
            w.y = c[2] | ((uint32_t)c[3] << 16);
            *reinterpret_cast<uint2*>(p) = w;
        } else {
            for (int i = 0; i < valid; ++i) p[i] = c[i];
        }
    } else if constexpr (DT == PNCE_TF32) {
        uint32_t c[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) c[i] = to_tf32(v[i]);
        if (valid == 4) {
            *reinterpret_cast<uint4*>(p) = make_uint4(c[0], c[1], c[2], c[3]);
        } else {
            for (int i = 0; i < valid; ++i) p[i] = c[i];
        }
    } else {
        const uint16_t lo = to_e4m3x2(v[0], v[1]);
        const uint16_t hi = to_e4m3x2(v[2], v[3]);
        if (valid == 4) {
            *reinterpret_cast<uint32_t*>(p) = lo | ((uint32_t)hi << 16);
        } else {
            const uint8_t c[4] = {(uint8_t)(lo & 0xff), (uint8_t)(lo >> 8), (uint8_t)(hi & 0xff),
                                  (uint8_t)(hi >> 8)};
            for (int i = 0; i < valid; ++i) p[i] = c[i];
        }
    }
}

template <int DT, bool POW>
__global__ void __launch_bounds__(THREADS)
quantize_kernel(const float2* __restrict__ Y, long long A, int N, long long y_stride, int pitch,
                void* __restrict__ Q,
                float* __restrict__ out_scale, int32_t* __restrict__ exps,
                double* __restrict__ power, float invN) {
    __shared__ float s_max[THREADS / 32];
    __shared__ double s_pow[THREADS / 32];
    __shared__ float s_scale;
    const int tid = threadIdx.x;

  const long long A_pad = (A + 7) / 8 * 8;
  for (long long a = blockIdx.x; a < A_pad; a += gridDim.x) {
    if (a >= A) {                  // padding antenna of the last group: zero rows
        const float z[4] = {0.f, 0.f, 0.f, 0.f};
        for (int n = 4 * tid; n < N; n += 4 * THREADS) {
            const int valid = min(4, N - n);
            store4<DT>(Q, pnce::operand_row(a, 0), pitch, n, z, valid);
            store4<DT>(Q, pnce::operand_row(a, 1), pitch, n, z, valid);
        }
        continue;
    }
    const float2* row = Y + a * y_stride;

    float amax = 0.f;
    double e = 0.0;
    for (int n = tid; n < N; n += THREADS) {
        const float2 y = row[n];
        amax = fmaxf(amax, fmaxf(fabsf(y.x), fabsf(y.y)));
        if constexpr (POW) e += (double)y.x * (double)y.x + (double)y.y * (double)y.y;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        if constexpr (POW) e += __shfl_xor_sync(0xffffffffu, e, o);
    }
    if ((tid & 31) == 0) {
        s_max[tid >> 5] = amax;
        s_pow[tid >> 5] = e;
    }
    __syncthreads();
    if (tid == 0) {
        float m = 0.f;
        double et = 0.0;
        for (int w = 0; w < THREADS / 32; ++w) {   // fixed order: deterministic
            m = fmaxf(m, s_max[w]);
            et += s_pow[w];
        }
        int se = 0;
        if (Fmt<DT>::target != 0 && m > 0.f && isfinite(m)) {
            int ex;
            frexpf(m, &ex);                          // m = mant * 2^ex, mant in [0.5, 1)
            se = Fmt<DT>::target - ex;
            se = se < -100 ? -100 : (se > 100 ? 100 : se);
        }
        s_scale = ldexpf(1.0f, se);
        out_scale[a] = ldexpf(invN, -se);
        if (exps) exps[a] = se;
        if constexpr (POW) power[a] = et / (double)N;
    }
    __syncthreads();
    const float sc = s_scale;

    // pass 2: four consecutive samples per thread per step
    for (int n = 4 * tid; n < N; n += 4 * THREADS) {
        const int valid = min(4, N - n);
        float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (i < valid) {
                const float2 y = __ldcs(row + n + i);   // last use: evict first
                re[i] = y.x * sc;          // exact: power-of-two scale
                im[i] = y.y * sc;
            }
        }
        store4<DT>(Q, pnce::operand_row(a, 0), pitch, n, re, valid);
        store4<DT>(Q, pnce::operand_row(a, 1), pitch, n, im, valid);
    }
    __syncthreads();   // s_max / s_scale are reused by the next antenna
  }
}

template <int DT>
cudaError_t launch_dt(const float2* Y, long long A, int N, void* operand, float* factors,
                      int32_t* exps, double* power, cudaStream_t s, int max_blocks,
                      long long y_stride) {
    const float invN = (float)(1.0 / (double)N);
    long long grid = (A + 7) / 8 * 8;               // padding antennas included
    if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
    if (grid > 0x7fffffffLL) grid = 0x7fffffffLL;
    auto kern = power ? quantize_kernel<DT, true> : quantize_kernel<DT, false>;
    kern<<<(unsigned)grid, THREADS, 0, s>>>(Y, A, N, y_stride > 0 ? y_stride : N,
                                            pnce::row_pitch(N), operand, factors, exps, power,
                                            invN);
    return cudaGetLastError();
}

// Serving batches (pnce_estimate_grouped): the row gather and the quantiser in one pass.
// Block a handles batch row a: the request that owns it (row_req, built by the grouped
// prep kernel) names where the received row lives -- page-locked host memory or device
// memory -- and the block reads it from there once (kept in shared memory when STAGE),
// so the samples cross the host link once and no batch copy of Y exists.  Rows no request
// covers, and the padding rows of the last 8-antenna group, get zero codes and factor 0.
// Launched as a programmatic dependent of the prep kernel: it lets the correlation that
// follows start its set-up at once, then waits for the row map.
template <int DT, bool STAGE>
__global__ void __launch_bounds__(THREADS)
grouped_quantize_kernel(const pnce_req_desc* __restrict__ dd, const int* __restrict__ row_req,
                        int rows, int N, int pitch, void* __restrict__ Q,
                        float* __restrict__ out_scale, float invN) {
    extern __shared__ float2 s_row[];
    __shared__ float s_max[THREADS / 32];
    __shared__ float s_scale;
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int tid = threadIdx.x;
    const long long a = blockIdx.x;
    const int b = a < rows ? row_req[a] : -1;
    if (b < 0) {
        const float z[4] = {0.f, 0.f, 0.f, 0.f};
        for (int n = 4 * tid; n < N; n += 4 * THREADS) {
            const int valid = min(4, N - n);
            store4<DT>(Q, pnce::operand_row(a, 0), pitch, n, z, valid);
            store4<DT>(Q, pnce::operand_row(a, 1), pitch, n, z, valid);
        }
        if (a < rows && tid == 0) out_scale[a] = 0.f;
        return;
    }
    const pnce_req_desc q = dd[b];
    const float2* row = static_cast<const float2*>(q.Y) + (long long)(a - q.row_offset) * N;

    // The row crosses the host link (or comes from device memory) once.  Sample pairs are
    // read as 16-byte loads from the first 16-byte boundary on (a row of odd N starts
    // half-way into one every other row), four pairs per thread issued before any is used
    // so that enough requests are in flight to cover the link's latency.
    float amax = 0.f;
    const int head = ((uintptr_t)row & 15u) ? 1 : 0;
    const int npairs = (N - head) >> 1;
    const float4* pairs = reinterpret_cast<const float4*>(row + head);
    for (int i0 = tid; i0 < npairs; i0 += 4 * THREADS) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * THREADS;
            v[u] = i < npairs ? pairs[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * THREADS;
            if (i < npairs) {
                if constexpr (STAGE) {
                    s_row[head + 2 * i] = make_float2(v[u].x, v[u].y);
                    s_row[head + 2 * i + 1] = make_float2(v[u].z, v[u].w);
                }
                amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v[u].x), fabsf(v[u].y)),
                                         fmaxf(fabsf(v[u].z), fabsf(v[u].w))));
            }
        }
    }
    if (tid < 2) {                     // the unpaired sample at the head and / or the tail
        const int n = tid == 0 ? (head ? 0 : -1) : ((N - head) & 1 ? N - 1 : -1);
        if (n >= 0) {
            const float2 y = row[n];
            if constexpr (STAGE) s_row[n] = y;
            amax = fmaxf(amax, fmaxf(fabsf(y.x), fabsf(y.y)));
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((tid & 31) == 0) s_max[tid >> 5] = amax;
    __syncthreads();
    if (tid == 0) {
        float m = 0.f;
        for (int w = 0; w < THREADS / 32; ++w) m = fmaxf(m, s_max[w]);
        int se = 0;
        if (Fmt<DT>::target != 0 && m > 0.f && isfinite(m)) {
            int ex;
            frexpf(m, &ex);
            se = Fmt<DT>::target - ex;
            se = se < -100 ? -100 : (se > 100 ? 100 : se);
        }
        s_scale = ldexpf(1.0f, se);
        out_scale[a] = ldexpf(invN, -se);
    }
    __syncthreads();
    const float sc = s_scale;
    for (int n = 4 * tid; n < N; n += 4 * THREADS) {
        const int valid = min(4, N - n);
        float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (i < valid) {
                const float2 y = STAGE ? s_row[n + i] : row[n + i];
                re[i] = y.x * sc;
                im[i] = y.y * sc;
            }
        }
        store4<DT>(Q, pnce::operand_row(a, 0), pitch, n, re, valid);
        store4<DT>(Q, pnce::operand_row(a, 1), pitch, n, im, valid);
    }
}

template <int DT>
cudaError_t launch_grouped_dt(const pnce_req_desc* dd, const int* row_req, int rows, int N,
                              void* operand, float* factors, cudaStream_t s) {
    const float invN = (float)(1.0 / (double)N);
    const size_t row_bytes = (size_t)N * sizeof(float2);
    const bool stage = row_bytes <= (size_t)48 * 1024;      // no opt-in shared memory needed
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((rows + 7) / 8 * 8), 1, 1);   // padding rows included
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = stage ? row_bytes : 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const int pitch = pnce::row_pitch(N);
    return stage ? cudaLaunchKernelEx(&cfg, grouped_quantize_kernel<DT, true>, dd, row_req, rows,
                                      N, pitch, operand, factors, invN)
                 : cudaLaunchKernelEx(&cfg, grouped_quantize_kernel<DT, false>, dd, row_req,
                                      rows, N, pitch, operand, factors, invN);
}

}  // namespace

namespace pnce {

cudaError_t launch_quantize_grouped(const pnce_req_desc* dd, const int* row_req, int rows, int N,
                                    int dtype, void* operand, float* factors, cudaStream_t s) {
    switch (dtype) {
        case PNCE_FP16:
            return launch_grouped_dt<PNCE_FP16>(dd, row_req, rows, N, operand, factors, s);
        case PNCE_BF16:
            return launch_grouped_dt<PNCE_BF16>(dd, row_req, rows, N, operand, factors, s);
        case PNCE_TF32:
            return launch_grouped_dt<PNCE_TF32>(dd, row_req, rows, N, operand, factors, s);
        case PNCE_FP8E4M3:
            return launch_grouped_dt<PNCE_FP8E4M3>(dd, row_req, rows, N, operand, factors, s);
        default: return cudaErrorInvalidValue;
    }
}

int elem_bytes(int dtype) {
    switch (dtype) {
        case PNCE_FP16: case PNCE_BF16: return 2;
        case PNCE_TF32: return 4;
        case PNCE_FP8E4M3: return 1;
        default: return 0;
    }
}

QuantLayout quant_layout(long long A, int N, int dtype) {
    QuantLayout l{};
    l.a_offset = 0;
    l.a_bytes = (size_t)operand_rows(A) * (size_t)row_pitch(N) * (size_t)elem_bytes(dtype);
    l.scale_offset = round_up(l.a_bytes, 256);
    l.total = round_up(l.scale_offset + (size_t)A * sizeof(float), 256);
    return l;
}

cudaError_t launch_quantize(const float2* Y, long long A, int N, int dtype, void* operand,
                            float* factors, int32_t* exps, double* power, cudaStream_t s,
                            int mb, long long ys) {
    switch (dtype) {
        case PNCE_FP16:
            return launch_dt<PNCE_FP16>(Y, A, N, operand, factors, exps, power, s, mb, ys);
        case PNCE_BF16:
            return launch_dt<PNCE_BF16>(Y, A, N, operand, factors, exps, power, s, mb, ys);
        case PNCE_TF32:
            return launch_dt<PNCE_TF32>(Y, A, N, operand, factors, exps, power, s, mb, ys);
        case PNCE_FP8E4M3:
            return launch_dt<PNCE_FP8E4M3>(Y, A, N, operand, factors, exps, power, s, mb, ys);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pnce
