// Adjoint of the real-pilot correlation (pilot optimisation through the estimator).
//
// Forward: H[a][j] = (1/N) sum_n Y[a][n] p[(n - j) mod N], p real.  For a real loss with
// G = dLoss/dRe(H) + i dLoss/dIm(H):
//   dY[a][n] = (1/N) sum_j G[a][j] p[(n - j) mod N]       (pnce_simt.cu, pilot reversed)
//   dp[q]    = (1/N) sum_a sum_j Re(conj(G[a][j]) Y[a][(q + j) mod N])   (this file)
// and, when the pilot is p = tanh(theta), dtheta[q] = dp[q] (1 - tanh(theta[q])^2).
//
// dp: the grid is a fixed number of warps (DP_WARPS, one wave of 2 blocks x 8 warps on
// each of 152 SMs), independent of the device so that results are the same everywhere.
// A warp owns one q-tile of 32 R consecutive outputs (R per lane; R = 16, or 8 when
// N <= 256 so that short pilots do not compute mostly wasted tiles) and a round-robin
// share of the (antenna, 128-lag chunk) items: warp w takes the tile w % Q and the items
// w / Q, w / Q + P, ... (P = warps per tile), so all warps carry the same share of the
// sum.  Per item the warp stages the cyclic window Y[a][(q0 + j0 + t) mod N]
// (t < 32 R + 136) and G[a][j0 .. j0+127] in its own shared buffers with cp.async,
// double buffered so that the next item's copies fly while this one is summed.  A lane's
// R outputs read Y at consecutive offsets: an (R + 7)-entry register window slides along
// the staged row (fully unrolled, so the slide is only register renaming), and the real
// and imaginary products go into the two halves of packed FP32 FMAs.  Each warp writes
// one partial row; a second kernel adds the partial rows of each q-tile in a fixed
// order.  The result is bitwise reproducible.
#include <algorithm>

#include "pnce_internal.h"

namespace {

constexpr int JC = 128;             // lags per chunk
constexpr int DP_WARPS = 2432;      // warps in the grid: 152 SMs x 2 blocks x 8 warps
constexpr int DP_WPB = 8;           // warps per block

template <int R>
struct DpShape {
    static constexpr int QT = 32 * R;             // outputs per warp tile
    static constexpr int WN = R + 7;              // register window entries
    static constexpr int WLEN = JC + QT + 8;      // staged window entries (a lane reads up to
                                                  // R*31 + WN + 8*14 + 7 < WLEN)
    static constexpr int WPAD = ((WLEN + WLEN / R + 1) + 1) & ~1;   // even: g 16-byte aligned
};

// float2 entries padded by one per R, so that lanes R entries apart are R + 1 (odd) float2
// apart and a half-warp's 8-byte loads hit 16 distinct bank pairs
template <int R>
__device__ __forceinline__ int wpos(int t) { return t + t / R; }

template <int R>
struct __align__(16) DpStage {
    float2 w[DpShape<R>::WPAD];
    float2 g[JC];
};
template <int R>
constexpr size_t dp_smem() { return sizeof(DpStage<R>) * 2 * DP_WPB; }

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int bytes = valid ? 8 : 0;      // 0: the destination is zero filled
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes)
                 : "memory");
}

// copies of one (antenna, chunk) into a stage; one commit group per call
template <int R>
__device__ __forceinline__ void dp_stage(DpStage<R>& st, const float2* yrow, const float2* grow,
                                         int N, int KL, int q0, int j0, int lane) {
    constexpr int WLEN = DpShape<R>::WLEN;
    const int p0 = (q0 + j0) % N;
    if (N >= WLEN) {                          // the window wraps at most once
#pragma unroll
        for (int i = 0; i < (WLEN + 31) / 32; ++i) {
            const int t = lane + 32 * i;
            const int pos = p0 + t >= N ? p0 + t - N : p0 + t;
            if (t < WLEN) cp_async8(&st.w[wpos<R>(t)], yrow + pos, true);
        }
    } else {
        int pos = (p0 + lane) % N;
        for (int i = 0; i < (WLEN + 31) / 32; ++i) {
            const int t = lane + 32 * i;
            if (t < WLEN) cp_async8(&st.w[wpos<R>(t)], yrow + pos, true);
            pos = (pos + 32) % N;
        }
    }
#pragma unroll
    for (int i = 0; i < JC / 32; ++i) {
        const int u = lane + 32 * i;
        const bool ok = j0 + u < KL;
        cp_async8(&st.g[u], ok ? grow + j0 + u : grow, ok);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int R>
__global__ void __launch_bounds__(DP_WPB * 32, 2)
dp_partial_kernel(const float2* __restrict__ G, const float2* __restrict__ Y, long long A, int N,
                  int KL, int Q, long long P, int chunks, float* __restrict__ partial) {
    constexpr int QT = DpShape<R>::QT, WN = DpShape<R>::WN;
    extern __shared__ __align__(16) unsigned char dp_smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long gw = (long long)blockIdx.x * DP_WPB + warp;
    if (gw >= P * Q) return;                  // no block-wide barrier below
    DpStage<R>* buf = reinterpret_cast<DpStage<R>*>(dp_smem_raw) + 2 * warp;
    const int q0 = (int)(gw % Q) * QT;
    const long long slot = gw / Q;
    // items i = a * chunks + c for i = slot, slot + P, ... < A * chunks (slot < P <= A)
    const long long items = (A * chunks - slot + P - 1) / P;
    long long next_a = slot / chunks;
    int next_c = (int)(slot % chunks);
    const long long step_a = P / chunks;
    const int step_c = (int)(P % chunks);
    auto issue = [&](DpStage<R>& st) {
        dp_stage<R>(st, Y + next_a * N, G + next_a * KL, N, KL, q0, next_c * JC, lane);
        next_c += step_c;
        next_a += step_a;
        if (next_c >= chunks) {
            next_c -= chunks;
            next_a += 1;
        }
    };

    float2 acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = make_float2(0.f, 0.f);

    issue(buf[0]);
    for (long long k = 0; k < items; ++k) {
        if (k + 1 < items) {
            issue(buf[(k + 1) & 1]);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncwarp();
        const DpStage<R>& st = buf[k & 1];
        // output q0 + R*lane + r at lag j0 + u reads window entry R*lane + r + u
        const int base = R * lane;
        float2 w[WN];
#pragma unroll
        for (int i = 0; i < WN; ++i) w[i] = st.w[wpos<R>(base + i)];
#pragma unroll
        for (int s = 0; s < JC / 8; ++s) {
            float2 nw[8];
            if (s + 1 < JC / 8) {
#pragma unroll
                for (int i = 0; i < 8; ++i) nw[i] = st.w[wpos<R>(base + 8 * s + WN + i)];
            }
            const float4* g4 = reinterpret_cast<const float4*>(st.g + 8 * s);
#pragma unroll
            for (int u2 = 0; u2 < 4; ++u2) {
                const float4 gg = g4[u2];
                const float2 ga = make_float2(gg.x, gg.y), gb = make_float2(gg.z, gg.w);
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] = __ffma2_rn(ga, w[2 * u2 + r], acc[r]);
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] = __ffma2_rn(gb, w[2 * u2 + 1 + r], acc[r]);
            }
            if (s + 1 < JC / 8) {
#pragma unroll
                for (int i = 0; i < WN - 8; ++i) w[i] = w[i + 8];
#pragma unroll
                for (int i = 0; i < 8; ++i) w[WN - 8 + i] = nw[i];
            }
        }
        __syncwarp();                         // every lane is done with this stage
    }
    float4* out = reinterpret_cast<float4*>(partial + gw * QT + R * lane);
#pragma unroll
    for (int r = 0; r < R; r += 4)
        out[r / 4] = make_float4(acc[r].x + acc[r].y, acc[r + 1].x + acc[r + 1].y,
                                 acc[r + 2].x + acc[r + 2].y, acc[r + 3].x + acc[r + 3].y);
}

// dp[q] = invN * sum over the P partial rows of q's tile (fixed order), or, for the tanh
// map, that times 1 - tanh(theta)^2.  Block = 32 consecutive q; warp w adds the rows
// w, w + 8, ...; warp 0 adds the 8 warp sums in order.
__global__ void __launch_bounds__(256)
dp_final_kernel(const float* __restrict__ partial, int QT, int Q, long long P, int N,
                float invN, const float* __restrict__ theta, float* __restrict__ dp) {
    __shared__ float red[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = blockIdx.x * 32 + lane;
    float s = 0.f;
    if (q < N) {
        const int qt = q / QT, off = q % QT;
        for (long long slot = warp; slot < P; slot += 8) s += partial[(slot * Q + qt) * QT + off];
    }
    red[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && q < N) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += red[w][lane];
        t *= invN;
        if (theta) {
            const float th = tanhf(theta[q]);
            t *= (1.0f - th * th);
        }
        dp[q] = t;
    }
}

struct DpGrid {
    int R, QT, Q;
    long long P;
};

DpGrid dp_grid(long long A, int N) {
    DpGrid g;
    g.R = N <= 256 ? 8 : 16;
    g.QT = 32 * g.R;
    g.Q = (N + g.QT - 1) / g.QT;
    g.P = std::max(1LL, std::min(A, (long long)(DP_WARPS / g.Q)));
    return g;
}

template <int R>
cudaError_t launch_dp(const DpGrid& g, const float2* G, const float2* Y, long long A, int N,
                      int KL, float* partial, cudaStream_t s) {
    const long long blocks = (g.P * g.Q + DP_WPB - 1) / DP_WPB;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(dp_partial_kernel<R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dp_smem<R>());
    if (e != cudaSuccess) return e;
    const int chunks = (KL + JC - 1) / JC;
    dp_partial_kernel<R><<<(unsigned)blocks, DP_WPB * 32, dp_smem<R>(), s>>>(G, Y, A, N, KL, g.Q,
                                                                           g.P, chunks, partial);
    return cudaGetLastError();
}

}  // namespace

namespace pnce {

size_t backward_workspace(long long A, int N, int KL) {
    (void)KL;
    const DpGrid g = dp_grid(A, N);
    return round_up((size_t)(g.P * g.Q) * (size_t)g.QT * sizeof(float), 256);
}

cudaError_t launch_backward(const float* p, bool tanh_map, const float2* Y, const float2* G,
                            long long A, int N, int KL, float2* dY, float* dp, void* ws,
                            size_t ws_bytes, cudaStream_t s) {
    if (dY) {
        cudaError_t e = launch_adjoint_dy(p, tanh_map, G, A, N, KL, dY, s);
        if (e != cudaSuccess) return e;
    }
    if (dp) {
        if (ws_bytes < backward_workspace(A, N, KL)) return cudaErrorInvalidValue;
        const DpGrid g = dp_grid(A, N);
        float* partial = static_cast<float*>(ws);
        cudaError_t e = g.R == 8 ? launch_dp<8>(g, G, Y, A, N, KL, partial, s)
                                 : launch_dp<16>(g, G, Y, A, N, KL, partial, s);
        if (e != cudaSuccess) return e;
        dp_final_kernel<<<(N + 31) / 32, 256, 0, s>>>(partial, g.QT, g.Q, g.P, N,
                                                      (float)(1.0 / (double)N),
                                                      tanh_map ? p : nullptr, dp);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

}  // namespace pnce
