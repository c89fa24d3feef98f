// Adjoint of the real-pilot correlation (pilot optimisation through the estimator).
//
// Forward: H[a][j] = (1/N) sum_n Y[a][n] p[(n - j) mod N], p real.  For a real loss with
// G = dLoss/dRe(H) + i dLoss/dIm(H):
//   dY[a][n] = (1/N) sum_j G[a][j] p[(n - j) mod N]       (pnce_simt.cu, pilot reversed)
//   dp[q]    = (1/N) sum_a sum_j Re(conj(G[a][j]) Y[a][(q + j) mod N])   (this file)
// and, when the pilot is p = tanh(theta), dtheta[q] = dp[q] (1 - tanh(theta[q])^2).
//
// dp: block = 8 warps over one tile of 256 consecutive q (8 per lane); each warp takes
// antennas warp, warp+8, ... of the block's antenna group and, per 128-lag chunk, stages
// the cyclic window Y[a][(q0 + j0 + t) mod N] (t < 392) and G[a][j0 .. j0+127] in its own
// shared buffers.  A lane's 8 outputs read Y at consecutive offsets, so a 15-entry
// register window slides along the staged row.  The 8 warps' sums are added in a fixed
// order and written as one partial row per antenna group; a second kernel adds the
// partial rows in a fixed order.  The result is bitwise reproducible.
#include "pnce_internal.h"

namespace {

constexpr int QT = 256;             // outputs per block (8 per lane)
constexpr int JC = 128;             // lags per chunk
constexpr int WLEN = JC + QT + 8;   // staged window entries
constexpr int AGROUP = 64;          // antennas per block (partial row)

// float2 entries padded by one per 8 so that lanes 8 entries apart hit distinct banks
__device__ __forceinline__ int wpos(int t) { return t + (t >> 3); }
constexpr int WPAD = WLEN + WLEN / 8 + 2;

struct WarpBuf {
    float2 w[WPAD];
    float2 g[JC];
};

__global__ void __launch_bounds__(256)
dp_partial_kernel(const float2* __restrict__ G, const float2* __restrict__ Y, long long A, int N,
                  int KL, int num_qt, float* __restrict__ partial, int pitch) {
    __shared__ WarpBuf wb[8];
    __shared__ float red[8][QT];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q0 = (int)(blockIdx.x % num_qt) * QT;
    const long long grp = blockIdx.x / num_qt;
    const long long a_begin = grp * AGROUP;
    const long long a_end = min(A, a_begin + AGROUP);
    WarpBuf& B = wb[warp];

    float acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = 0.f;

    for (long long a = a_begin + warp; a < a_end; a += 8) {
        const float2* yrow = Y + a * N;
        const float2* grow = G + a * KL;
        for (int j0 = 0; j0 < KL; j0 += JC) {
            __syncwarp();
            // window entry t = Y[(q0 + j0 + t) mod N]
            int pos = (int)(((long long)q0 + j0 + lane) % N);
            for (int t = lane; t < WLEN; t += 32) {
                B.w[wpos(t)] = yrow[pos];
                pos += 32;
                while (pos >= N) pos -= N;
            }
            for (int u = lane; u < JC; u += 32)
                B.g[u] = (j0 + u < KL) ? grow[j0 + u] : make_float2(0.f, 0.f);
            __syncwarp();
            // output q0 + 8*lane + r at lag j0 + u reads entry 8*lane + r + u
            const int base = 8 * lane;
            float2 w[15];
#pragma unroll
            for (int i = 0; i < 15; ++i) w[i] = B.w[wpos(base + i)];
            const int nblk = min(JC, KL - j0 + 7) / 8;
#pragma unroll 1
            for (int s = 0; s < nblk; ++s) {
                float2 nw[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) nw[i] = B.w[wpos(base + 8 * s + 15 + i)];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float2 g = B.g[8 * s + u];
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        acc[r] = fmaf(g.x, w[u + r].x, acc[r]);
                        acc[r] = fmaf(g.y, w[u + r].y, acc[r]);
                    }
                }
#pragma unroll
                for (int i = 0; i < 7; ++i) w[i] = w[i + 8];
#pragma unroll
                for (int i = 0; i < 8; ++i) w[7 + i] = nw[i];
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) red[warp][8 * lane + r] = acc[r];
    __syncthreads();
    for (int q = tid; q < QT; q += 256) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) s += red[w][q];
        if (q0 + q < N) partial[grp * (long long)pitch + q0 + q] = s;
    }
}

// dp[q] = invN * sum_g partial[g][q], or, for the tanh map, that times 1 - tanh(theta)^2
__global__ void dp_final_kernel(const float* __restrict__ partial, long long groups, int N,
                                int pitch, float invN, const float* __restrict__ theta,
                                float* __restrict__ dp) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N) return;
    float s = 0.f;
    for (long long g = 0; g < groups; ++g) s += partial[g * (long long)pitch + q];
    s *= invN;
    if (theta) {
        const float t = tanhf(theta[q]);
        s *= (1.0f - t * t);
    }
    dp[q] = s;
}

}  // namespace

namespace pnce {

size_t backward_workspace(long long A, int N, int KL) {
    (void)KL;
    const long long groups = (A + AGROUP - 1) / AGROUP;
    return round_up((size_t)groups * (size_t)round_up((size_t)N, 64) * sizeof(float), 256);
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
        const int num_qt = (N + QT - 1) / QT;
        const long long groups = (A + AGROUP - 1) / AGROUP;
        const long long blocks = groups * num_qt;
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
        const int pitch = (int)round_up((size_t)N, 64);
        float* partial = static_cast<float*>(ws);
        dp_partial_kernel<<<(unsigned)blocks, 256, 0, s>>>(G, Y, A, N, KL, num_qt, partial, pitch);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        dp_final_kernel<<<(N + 255) / 256, 256, 0, s>>>(partial, groups, N, pitch,
                                                        (float)(1.0 / (double)N),
                                                        tanh_map ? p : nullptr, dp);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

}  // namespace pnce
