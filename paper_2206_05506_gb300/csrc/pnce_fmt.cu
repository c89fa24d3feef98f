// Fast m-sequence transform: a yardstick beside the paper's method (the paper correlates
// with the dense circulant, Sec. III-B; this computes the same estimate in O(N log N)).
//
// For an m-sequence of degree r (N = 2^r - 1) the r-bit windows s_n = sum_{i<r} b[n+i] 2^i
// run through every nonzero r-bit vector exactly once, and since the sequence obeys a
// linear recurrence of order r, every bit of it is a GF(2)-linear function of any window:
// b[(n - j) mod N] = <u_j, s_n> (mod 2) with a vector u_j that depends on the lag j only.
// The pilot of Eq. 1 is then p[(n - j) mod N] = (-1)^<u_j, s_n>, and the estimate of Eq. 3
//     N H[j] = sum_n y[n] (-1)^<u_j, s_n> = W[u_j],
// where W is the Walsh-Hadamard transform of the length-2^r vector X with X[s_n] = y[n]
// and X[0] = 0.  u_j follows from the windows that are unit vectors: if s_{n_i} = 2^i then
// bit i of u_j is b[(n_i - j) mod N].
//
// Kernels: one CTA per received row; the row is scattered into X in shared memory
// (2^r complex values), the transform runs in a few passes over X with the butterfly
// levels of a pass held in registers (and lane exchanges), and the K*L wanted lags are
// gathered, scaled by 1/N and written out.  FP32 throughout: every output is a sum of +-y, so the only error is
// the FP32 rounding of r levels of additions.
#include <new>
#include <vector>

#include "pnce_internal.h"

struct pnce_fmt {
    int device;
    int N;
    int r;
    uint16_t* pos_dev;      // s_n, n < N
    uint16_t* lag_dev;      // u_j, j < N
};

namespace {

constexpr int THREADS = 256;
constexpr int MAX_R = 14;   // 2^14 complex values = 128 KB of shared memory

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
pnce_status on_device(const pnce_handle* h) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return PNCE_ECUDA;
    return dev == h->device ? PNCE_OK : PNCE_ESTATE;
}

// One pass of the transform: butterfly levels at distances h, 2h, .., 2^(K-1) h, each
// thread holding 2^K elements of one group in registers.
template <int K>
__device__ __forceinline__ void fwht_pass(float2* X, int r, int lh, int tid) {
    constexpr int R = 1 << K;
    const int h = 1 << lh;
    const int groups = (1 << r) >> K;
    for (int g = tid; g < groups; g += THREADS) {
        const int base = ((g >> lh) << (lh + K)) | (g & (h - 1));
        float2 v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = X[base + k * h];
#pragma unroll
        for (int lvl = 0; lvl < K; ++lvl) {
            const int d = 1 << lvl;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                if (k & d) continue;
                const float2 a = v[k], b = v[k + d];
                v[k] = make_float2(a.x + b.x, a.y + b.y);
                v[k + d] = make_float2(a.x - b.x, a.y - b.y);
            }
        }
#pragma unroll
        for (int k = 0; k < R; ++k) X[base + k * h] = v[k];
    }
}

__global__ void __launch_bounds__(THREADS)
fmt_kernel(const float2* __restrict__ Y, long long A, int N, int r,
           const uint16_t* __restrict__ pos, const uint16_t* __restrict__ lagvec, int KL,
           float invN, float2* __restrict__ H) {
    extern __shared__ float2 X[];
    const int tid = threadIdx.x;
    for (long long a = blockIdx.x; a < A; a += gridDim.x) {
        const float2* y = Y + a * N;
        if (tid == 0) X[0] = make_float2(0.f, 0.f);
        for (int n = tid; n < N; n += THREADS) X[__ldg(pos + n)] = __ldcs(y + n);
        __syncthreads();
        int lh = 0;
        while (lh < r) {
            const int k = (r - lh) >= 3 ? 3 : (r - lh);
            if (k == 3) fwht_pass<3>(X, r, lh, tid);
            else if (k == 2) fwht_pass<2>(X, r, lh, tid);
            else fwht_pass<1>(X, r, lh, tid);
            lh += k;
            __syncthreads();
        }
        float2* out = H + a * KL;
        for (int j = tid; j < KL; j += THREADS) {
            const float2 w = X[__ldg(lagvec + j)];
            out[j] = make_float2(w.x * invN, w.y * invN);
        }
        __syncthreads();   // X is refilled for the next row
    }
}

// The same for 2^r >= 512 (r <= 14), laid out to keep shared memory conflict-free: warp w
// takes segments of 512 consecutive entries, lane l holding entries l + 32 m (m < 16), so
// the butterfly levels at distances 1..16 are lane exchanges (shuffles) and those at
// 32..256 stay in the thread's registers; the r - 9 levels at distances 512.. S/2 follow
// in one more pass over groups of entries 512 apart.  Every shared-memory access of the
// passes is 32 consecutive entries per warp instruction.
template <int R>
__global__ void __launch_bounds__(THREADS, R >= 14 ? 3 : 4)   // 4 rows in flight per SM
fmt_kernel_seg(const float2* __restrict__ Y, long long A, int N,
               const uint16_t* __restrict__ pos, const uint16_t* __restrict__ lagvec, int KL,
               float invN, float2* __restrict__ H) {
    constexpr int S = 1 << R;
    constexpr int SEG = 512, NSEG = S / SEG;
    constexpr int CR = R - 9;                  // levels across segments
    constexpr int CG = 1 << CR;                // entries per group of the last pass
    extern __shared__ float2 X[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (long long a = blockIdx.x; a < A; a += gridDim.x) {
        const float2* y = Y + a * N;
        if (tid == 0) X[0] = make_float2(0.f, 0.f);
        for (int n = tid; n < N; n += THREADS) X[__ldg(pos + n)] = __ldcs(y + n);
        __syncthreads();
        for (int seg = warp; seg < NSEG; seg += THREADS / 32) {
            float2* xs = X + seg * SEG + lane;
            float2 v[16];
#pragma unroll
            for (int m = 0; m < 16; ++m) v[m] = xs[32 * m];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const bool upper = (lane & d) != 0;
#pragma unroll
                for (int m = 0; m < 16; ++m) {
                    const float px = __shfl_xor_sync(0xffffffffu, v[m].x, d);
                    const float py = __shfl_xor_sync(0xffffffffu, v[m].y, d);
                    v[m] = upper ? make_float2(px - v[m].x, py - v[m].y)
                                 : make_float2(v[m].x + px, v[m].y + py);
                }
            }
#pragma unroll
            for (int dm = 1; dm < 16; dm <<= 1) {
#pragma unroll
                for (int m = 0; m < 16; ++m) {
                    if (m & dm) continue;
                    const float2 p = v[m], q = v[m + dm];
                    v[m] = make_float2(p.x + q.x, p.y + q.y);
                    v[m + dm] = make_float2(p.x - q.x, p.y - q.y);
                }
            }
#pragma unroll
            for (int m = 0; m < 16; ++m) xs[32 * m] = v[m];
        }
        __syncthreads();
        if constexpr (CR > 0) {
            for (int g = tid; g < SEG; g += THREADS) {
                float2 w[CG];
#pragma unroll
                for (int k = 0; k < CG; ++k) w[k] = X[g + SEG * k];
#pragma unroll
                for (int dk = 1; dk < CG; dk <<= 1) {
#pragma unroll
                    for (int k = 0; k < CG; ++k) {
                        if (k & dk) continue;
                        const float2 p = w[k], q = w[k + dk];
                        w[k] = make_float2(p.x + q.x, p.y + q.y);
                        w[k + dk] = make_float2(p.x - q.x, p.y - q.y);
                    }
                }
#pragma unroll
                for (int k = 0; k < CG; ++k) X[g + SEG * k] = w[k];
            }
            __syncthreads();
        }
        float2* out = H + a * KL;
        for (int j = tid; j < KL; j += THREADS) {
            const float2 w = X[__ldg(lagvec + j)];
            out[j] = make_float2(w.x * invN, w.y * invN);
        }
        __syncthreads();   // X is refilled for the next row
    }
}

}  // namespace

extern "C" {

pnce_status pnce_fmt_tables(const uint32_t* bits_host, int N, uint16_t* pos, uint16_t* lagvec) {
    if (!bits_host || !pos || !lagvec || N < 3) return PNCE_EINVAL;
    int r = 0;
    while ((1LL << r) < (long long)N + 1) ++r;
    if ((1LL << r) != (long long)N + 1 || r < 2 || r > MAX_R) return PNCE_EINVAL;
    std::vector<uint8_t> b((size_t)N);
    for (int n = 0; n < N; ++n) b[(size_t)n] = (uint8_t)((bits_host[n >> 5] >> (n & 31)) & 1u);
    // windows: distinct and nonzero
    std::vector<int> inv((size_t)1 << r, -1);
    for (int n = 0; n < N; ++n) {
        uint32_t s = 0;
        for (int i = 0; i < r; ++i) s |= (uint32_t)b[(size_t)((n + i) % N)] << i;
        if (s == 0 || inv[s] >= 0) return PNCE_EINVAL;
        inv[s] = n;
        pos[n] = (uint16_t)s;
    }
    // u_j from the unit windows
    for (int j = 0; j < N; ++j) {
        uint32_t u = 0;
        for (int i = 0; i < r; ++i) {
            const long long ni = inv[(size_t)1 << i];
            u |= (uint32_t)b[(size_t)(((ni - j) % N + N) % N)] << i;
        }
        lagvec[j] = (uint16_t)u;
    }
    // the recurrence the windows imply must hold over the whole period: with j = N - r,
    // b[n + r] = <u_j, s_n> for every n (then every u_j is right, by linearity)
    const uint32_t c = lagvec[N - r];
    for (int n = 0; n < N; ++n) {
        const uint32_t x = c & pos[n];
        if ((uint32_t)(__builtin_popcount(x) & 1) != b[(size_t)((n + r) % N)]) return PNCE_EINVAL;
    }
    return PNCE_OK;
}

pnce_status pnce_fmt_create(pnce_handle* h, const uint32_t* bits_host, int N, pnce_fmt** out) {
    if (!h || !bits_host || !out) return PNCE_EINVAL;
    *out = nullptr;
    if (N < 3 || (long long)N + 1 > (1LL << MAX_R)) return PNCE_EINVAL;   // before allocating
    std::vector<uint16_t> pos, lag;
    try {
        pos.resize((size_t)N);
        lag.resize((size_t)N);
    } catch (...) {
        return PNCE_ENOMEM;
    }
    pnce_status st = pnce_fmt_tables(bits_host, N, pos.data(), lag.data());
    if (st != PNCE_OK) return st;
    st = on_device(h);
    if (st != PNCE_OK) return st;
    pnce_fmt* f = new (std::nothrow) pnce_fmt();
    if (!f) return PNCE_ENOMEM;
    f->device = h->device;
    f->N = N;
    f->r = 0;
    while ((1 << f->r) < N + 1) ++f->r;
    f->pos_dev = nullptr;
    f->lag_dev = nullptr;
    const size_t bytes = sizeof(uint16_t) * (size_t)N;
    if (cudaMalloc(&f->pos_dev, bytes) != cudaSuccess || cudaMalloc(&f->lag_dev, bytes) != cudaSuccess) {
        cudaFree(f->pos_dev);
        delete f;
        return PNCE_ENOMEM;
    }
    if (cudaMemcpy(f->pos_dev, pos.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(f->lag_dev, lag.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(f->pos_dev);
        cudaFree(f->lag_dev);
        delete f;
        return PNCE_ECUDA;
    }
    *out = f;
    return PNCE_OK;
}

pnce_status pnce_fmt_destroy(pnce_fmt* f) {
    if (!f) return PNCE_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(f->device);
    cudaFree(f->pos_dev);
    cudaFree(f->lag_dev);
    if (prev >= 0) cudaSetDevice(prev);
    delete f;
    return PNCE_OK;
}

pnce_status pnce_estimate_fmt(pnce_handle* h, const pnce_fmt* f, const void* Y_dev, int F, int M,
                              int N, int K, int L, void* H_dev, void* stream) {
    if (!h || !f || !Y_dev || !H_dev) return PNCE_EINVAL;
    if (F < 1 || M < 1 || K < 1 || L < 1 || N != f->N || (long long)K * L > N) return PNCE_EINVAL;
    if (!aligned16(Y_dev) || !aligned16(H_dev)) return PNCE_EINVAL;
    pnce_status st = on_device(h);
    if (st != PNCE_OK) return st;
    if (f->device != h->device) return PNCE_ESTATE;
    const long long A = (long long)F * M;
    const size_t smem = sizeof(float2) << f->r;
    if (f->r < 9 && cudaFuncSetAttribute(fmt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem) != cudaSuccess)
        return PNCE_ECUDA;
    const long long grid = A < 0x7fffffffLL ? A : 0x7fffffffLL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float2* Y = static_cast<const float2*>(Y_dev);
    float2* H = static_cast<float2*>(H_dev);
    const float invN = (float)(1.0 / (double)N);
    pnce::TraceScope tr(h, s, pnce::TRACE_FMT);
    if (f->r >= 9) {
        void (*kern)(const float2*, long long, int, const uint16_t*, const uint16_t*, int,
                     float, float2*) = nullptr;
        switch (f->r) {
            case 9: kern = fmt_kernel_seg<9>; break;
            case 10: kern = fmt_kernel_seg<10>; break;
            case 11: kern = fmt_kernel_seg<11>; break;
            case 12: kern = fmt_kernel_seg<12>; break;
            case 13: kern = fmt_kernel_seg<13>; break;
            default: kern = fmt_kernel_seg<14>; break;
        }
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return PNCE_ECUDA;
        kern<<<(unsigned)grid, THREADS, smem, s>>>(Y, A, N, f->pos_dev, f->lag_dev, K * L, invN,
                                                   H);
    } else {
        fmt_kernel<<<(unsigned)grid, THREADS, smem, s>>>(Y, A, N, f->r, f->pos_dev, f->lag_dev,
                                                         K * L, invN, H);
    }
    return cudaGetLastError() == cudaSuccess ? PNCE_OK : PNCE_ECUDA;
}

}  // extern "C"
