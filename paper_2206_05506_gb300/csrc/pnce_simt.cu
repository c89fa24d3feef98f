// FP32 correlation on the CUDA cores: H[a][j] = (1/N) sum_n Y[a][n] p[(n - j) mod N]
// (Eq. 3 / Eq. 10 of the paper, the "plain FP32" estimator).  The same kernel, with the
// pilot read backwards, is the received-block half of the adjoint:
// dY[a][n] = (1/N) sum_j G[a][j] p[(n - j) mod N] = (1/N) sum_j G[a][j] p'[(j - n) mod N]
// with p'[x] = p[-x mod N].  In general: out[a][o] = scale * sum_{k < Kred} in[a][k] *
// pilot[(k - o) mod Nmod], o < Nout.
//
// Block tile: up to 32 antennas x 256 lags (for large grids the rows are split into
// balanced groups so that the grid fills whole waves); thread tile: 4 antennas x 8
// consecutive lags, so each received sample read from shared memory feeds 64 FMAs.  Grids
// smaller than half the GPU use 1 antenna per thread (8-row blocks, 4x shorter).  Because
// a thread's lags are consecutive, the pilot values it needs at sample n+1 are those of
// sample n shifted by one lag: a 15-entry register window slides along the pilot, one new
// shared load per sample.  The pilot window of the whole reduction is staged in shared
// memory once per block, and each warp double-buffers its own rows (cp.async); serving
// batches use an instantiation that reads the rows from, and writes the lags into, the
// requests' own buffers.
#include <algorithm>

#include "pnce_internal.h"

namespace {

constexpr int RJ = 8;             // consecutive lags per thread
constexpr int WARPS = 8;
constexpr int TJ = 32 * RJ;       // lags per block
constexpr int NC = 128;           // samples per chunk
constexpr int ELEN = NC + TJ + 8; // pilot entries staged per chunk
constexpr int EPAD = ELEN + ELEN / 32 + 4;

// Pilot entries are stored with one pad word per 32 so that lanes reading entries 8 apart
// hit distinct banks.
__device__ __forceinline__ int epos(int t) { return t + (t >> 5); }

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    int bytes = valid ? 8 : 0;          // 0 source bytes: zero fill
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// RA antennas per thread (4; 1 for small grids), WARPS * RA antennas per block
template <int RA>
struct Smem {
    float e[2][EPAD];
    float2 y[2][WARPS * RA][NC];
};
static_assert(offsetof(Smem<4>, y) % 16 == 0 && offsetof(Smem<1>, y) % 16 == 0 && NC % 2 == 0,
              "paired sample loads need 16-byte rows");

// FWD_BITS: +-1 pilot from packed bits.  FWD_REAL / ADJ_REAL: float pilot, read forwards
// or backwards.  *_TANH: the float argument is theta and the pilot is tanh(theta).
enum Mode { FWD_BITS = 0, FWD_REAL = 1, ADJ_REAL = 2, FWD_TANH = 3, ADJ_TANH = 4 };

template <int MODE>
__device__ __forceinline__ float pilot_value(const uint32_t* bits, const float* preal, int q,
                                             int nmod) {
    if constexpr (MODE == FWD_BITS) {
        uint32_t b = (__ldg(bits + (q >> 5)) >> (q & 31)) & 1u;
        return b ? -1.0f : 1.0f;
    } else {
        const int idx = (MODE == ADJ_REAL || MODE == ADJ_TANH) ? (q == 0 ? 0 : nmod - q) : q;
        const float v = __ldg(preal + idx);
        if constexpr (MODE == FWD_TANH || MODE == ADJ_TANH) return tanhf(v);
        return v;
    }
}

template <int MODE, int RA>
__global__ void __launch_bounds__(256, 2)
simt_corr_kernel(const uint32_t* __restrict__ bits, const float* __restrict__ preal,
                 const float2* __restrict__ Y, long long y_stride, long long A,
                 int N /* reduction length */, const pnce::LagMap lags, int nmod, int num_jt,
                 long long groups, float invN, float2* __restrict__ H) {
    constexpr int TA = WARPS * RA;    // antennas per block
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<RA>& sm = *reinterpret_cast<Smem<RA>*>(smem_raw);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long bid = blockIdx.x;
    long long j0;            // first lag of this block's tile
    int col0, valid;         // its first output column and number of lags kept
    pnce::lag_tile(lags, TJ, bid % num_jt, j0, col0, valid);
    // antenna group g of a balanced partition of the A rows into `groups` (<= TA rows each)
    const long long g = bid / num_jt, gbase = A / groups, grem = A % groups;
    const long long a0 = g * gbase + (g < grem ? g : grem);
    const int rows = (int)(gbase + (g < grem ? 1 : 0));
    const int nchunks = (N + NC - 1) / NC;
    // chunk-local pilot entry t holds p[(c*NC + t - (j0 + TJ - 1)) mod N]
    const long long eoff = j0 + TJ - 1;

    auto stage = [&](int c, int buf) {
        const int n0 = c * NC;
        for (int i = tid; i < TA * NC; i += 256) {
            const int aa = i / NC, nn = i % NC;
            const long long a = a0 + aa;
            const bool ok = (aa < rows) && (n0 + nn < N);
            const float2* src = ok ? (Y + a * y_stride + n0 + nn) : Y;
            cp_async8(&sm.y[buf][aa][nn], src, ok);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        for (int t = tid; t < ELEN; t += 256) {
            long long q = ((long long)n0 + t - eoff) % nmod;
            if (q < 0) q += nmod;
            sm.e[buf][epos(t)] = pilot_value<MODE>(bits, preal, (int)q, nmod);
        }
    };

    float2 acc[RA][RJ];
#pragma unroll
    for (int i = 0; i < RA; ++i)
#pragma unroll
        for (int r = 0; r < RJ; ++r) acc[i][r] = make_float2(0.f, 0.f);

    // lag of (lane, r) is j0 + 8*lane + r; chunk-local entry for sample n0+u is
    // u + base - r with base = TJ - 1 - 8*lane (>= 7)
    const int base = TJ - 1 - RJ * lane;

    stage(0, 0);
    cp_async_wait_all();
    __syncthreads();

    for (int c = 0; c < nchunks; ++c) {
        const int buf = c & 1;
        if (c + 1 < nchunks) stage(c + 1, buf ^ 1);

        if (warp * RA < rows) {                  // warps past the group's rows only stage
        const float* e = sm.e[buf];
        float w[15];
#pragma unroll
        for (int i = 0; i < 15; ++i) w[i] = e[epos(base - 7 + i)];

#pragma unroll 2   // the sliding window's shifts become register renames
        for (int s = 0; s < NC / 8; ++s) {
            float nw[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) nw[i] = e[epos(8 * s + 8 + base + i)];
#pragma unroll
            for (int u2 = 0; u2 < 8; u2 += 2) {
                // two consecutive samples per 16-byte load (rows of sm.y are 16-byte aligned)
                float4 yy[RA];
#pragma unroll
                for (int i = 0; i < RA; ++i)
                    yy[i] = *reinterpret_cast<const float4*>(&sm.y[buf][warp * RA + i][8 * s + u2]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int u = u2 + h;
#pragma unroll
                    for (int r = 0; r < RJ; ++r) {
                        const float pv = w[u - r + 7];
#pragma unroll
                        for (int i = 0; i < RA; ++i) {
                            const float yx = h ? yy[i].z : yy[i].x, yi = h ? yy[i].w : yy[i].y;
                            // both parts in one packed FMA (each part rounded as fmaf)
                            acc[i][r] = __ffma2_rn(make_float2(pv, pv), make_float2(yx, yi),
                                                   acc[i][r]);
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 7; ++i) w[i] = w[i + 8];
#pragma unroll
            for (int i = 0; i < 8; ++i) w[7 + i] = nw[i];
        }
        }
        cp_async_wait_all();
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < RA; ++i) {
        if (warp * RA + i >= rows) continue;
        const long long a = a0 + warp * RA + i;
        float2* hrow = H + a * lags.ldH + col0;
#pragma unroll
        for (int r = 0; r < RJ; ++r) {
            const int j = RJ * lane + r;
            if (j < valid) hrow[j] = make_float2(acc[i][r].x * invN, acc[i][r].y * invN);
        }
    }
}

// The same tile with no block-wide barrier in its main loop: the pilot window of the whole
// reduction is staged once per block (E[t] = pilot[(t - eoff) mod nmod] for t <
// win_len(Nred), every chunk's window included), and every warp double-buffers its own RA
// rows with cp.async and warp-level synchronisation only.  In the chunked kernel above,
// the per-chunk __syncthreads kept warps waiting on the slowest one (ncu: barrier stalls
// about a quarter of all stall cycles).  Used when the window fits (WIN_MAX entries).
constexpr int WIN_MAX = 8192 + TJ + 8;

template <int RA>
struct WSmem {
    float2 y[WARPS][2][RA][NC];
};

// entries of the whole window: the last chunk reads up to entry (nchunks - 1) * NC + ELEN - 1
__host__ __device__ constexpr int win_len(int nred) { return (nred + NC - 1) / NC * NC + TJ + 8; }
__host__ __device__ constexpr size_t win_bytes(int nred) {
    return ((size_t)win_len(nred) + (size_t)win_len(nred) / 32 + 1) * sizeof(float);
}

// Serving batches: row a of the launch is row a - row_offset of request dd[row_req[a]]
// (its Y has N samples per row, its H keeps the first K*L lags); rows with row_req < 0
// belong to no request.  The kernel writes each row's lags into its request's H, and reads
// the rows from the requests' Y when Y is null (else from Y, a batch copy at pitch N):
// no batch copy of H, and none of Y when one lag tile covers the lags (each row is then
// read by one block; with more, every block of a row would fetch it over the host link).
// Launched as a programmatic dependent of the kernel before it.  dd == nullptr: plain
// Y / H.
struct GroupedIO {
    const pnce_req_desc* dd = nullptr;
    const int* row_req = nullptr;
    bool pdl = false;
};

// The rows of one warp: NR (<= RA) received rows from row a_first of the group, the chunks
// of the reduction double-buffered in the warp's own shared buffers.  Every output is
// summed over n in the same order whatever NR, so results do not depend on the row split.
template <int MODE, int RA, int NR, bool GRP>
__device__ __forceinline__ void warp_rows(WSmem<RA>& sm, const float* __restrict__ E,
                                          const float2* __restrict__ Y, long long y_stride,
                                          long long a_first, int N, const pnce::LagMap& lags,
                                          int col0, int valid, float invN,
                                          float2* __restrict__ H, int warp, int lane,
                                          const GroupedIO& g) {
    const int nchunks = (N + NC - 1) / NC;
    // row i's samples (null: no request owns it), looked up when needed rather than kept
    // in registers through the main loop
    auto src_row = [&](int i) -> const float2* {
        const long long a = a_first + i;
        if (!GRP || Y != nullptr) return Y + a * y_stride;
        const int b = __ldg(g.row_req + a);
        if (b < 0) return nullptr;
        const pnce_req_desc& q = g.dd[b];
        return static_cast<const float2*>(q.Y) + (a - q.row_offset) * N;
    };
    // a valid address for the copies that only zero-fill
    const float2* zsrc = (!GRP || Y) ? Y : reinterpret_cast<const float2*>(g.row_req);
    auto stage = [&](int c, int buf) {
        const int n0 = c * NC;
#pragma unroll
        for (int aa = 0; aa < NR; ++aa) {
            const float2* sr = src_row(aa);
            for (int nn = lane; nn < NC; nn += 32) {
                const bool ok = sr != nullptr && n0 + nn < N;
                cp_async8(&sm.y[warp][buf][aa][nn], ok ? sr + n0 + nn : zsrc, ok);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    float2 acc[NR][RJ];
#pragma unroll
    for (int i = 0; i < NR; ++i)
#pragma unroll
        for (int r = 0; r < RJ; ++r) acc[i][r] = make_float2(0.f, 0.f);
    const int base = TJ - 1 - RJ * lane;

    stage(0, 0);
    for (int c = 0; c < nchunks; ++c) {
        const int buf = c & 1;
        if (c + 1 < nchunks) {
            stage(c + 1, buf ^ 1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncwarp();
        const int cb = c * NC + base;
        float w[15];
#pragma unroll
        for (int i = 0; i < 15; ++i) w[i] = E[epos(cb - 7 + i)];

#pragma unroll 2   // the sliding window's shifts become register renames
        for (int s = 0; s < NC / 8; ++s) {
            float nw[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) nw[i] = E[epos(cb + 8 * s + 8 + i)];
#pragma unroll
            for (int u2 = 0; u2 < 8; u2 += 2) {
                float4 yy[NR];
#pragma unroll
                for (int i = 0; i < NR; ++i)
                    yy[i] = *reinterpret_cast<const float4*>(&sm.y[warp][buf][i][8 * s + u2]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int u = u2 + h;
#pragma unroll
                    for (int r = 0; r < RJ; ++r) {
                        const float pv = w[u - r + 7];
#pragma unroll
                        for (int i = 0; i < NR; ++i) {
                            const float yx = h ? yy[i].z : yy[i].x, yi = h ? yy[i].w : yy[i].y;
                            acc[i][r] = __ffma2_rn(make_float2(pv, pv), make_float2(yx, yi),
                                                   acc[i][r]);
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 7; ++i) w[i] = w[i + 8];
#pragma unroll
            for (int i = 0; i < 8; ++i) w[7 + i] = nw[i];
        }
        __syncwarp();                          // buf is free for chunk c + 2
    }

    if constexpr (!GRP) {
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            float2* hrow = H + (a_first + i) * lags.ldH + col0;
#pragma unroll
            for (int r = 0; r < RJ; ++r) {
                const int j = RJ * lane + r;
                if (j < valid) hrow[j] = make_float2(acc[i][r].x * invN, acc[i][r].y * invN);
            }
        }
    } else {
        // Serving rows go out through the warp's (now idle) staging buffer, so that a store
        // instruction writes 256 contiguous bytes rather than 32 pieces of 8 bytes 64 bytes
        // apart: the same for L2, but over the host link (results in page-locked memory) every
        // partial piece would be a transfer of its own.
        float2* sbuf = &sm.y[warp][0][0][0];         // 2 * RA * NC >= TJ entries
        static_assert(2 * RA * NC >= TJ, "staging buffer too small for a row of results");
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            const long long a = a_first + i;
            const int b = __ldg(g.row_req + a);
            if (b < 0) continue;                     // warp-uniform: one row per iteration
            const pnce_req_desc& q = g.dd[b];
            const int kl = q.K * q.L;
            float2* drow = static_cast<float2*>(q.H) + (a - q.row_offset) * kl + col0;
            const int vrow = min(valid, kl - col0);  // lags of the tile kept for it
#pragma unroll
            for (int r = 0; r < RJ; ++r)
                sbuf[RJ * lane + r] = make_float2(acc[i][r].x * invN, acc[i][r].y * invN);
            __syncwarp();
#pragma unroll
            for (int k = 0; k < RJ; ++k) {
                const int j = lane + 32 * k;
                if (j < vrow) drow[j] = sbuf[j];
            }
            __syncwarp();                            // sbuf is rewritten for the next row
        }
    }
}

template <int MODE, int RA, bool GRP>
__global__ void __launch_bounds__(256, 2)
simt_corr_warp_kernel(const uint32_t* __restrict__ bits, const float* __restrict__ preal,
                      const float2* __restrict__ Y, long long y_stride, long long A,
                      int N /* reduction length */, const pnce::LagMap lags, int nmod,
                      int num_jt, long long groups, float invN, float2* __restrict__ H,
                      const GroupedIO gio) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WSmem<RA>& sm = *reinterpret_cast<WSmem<RA>*>(smem_raw);
    float* E = reinterpret_cast<float*>(smem_raw + sizeof(WSmem<RA>));

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long bid = blockIdx.x;
    long long j0;
    int col0, valid;
    pnce::lag_tile(lags, TJ, bid % num_jt, j0, col0, valid);
    const long long g = bid / num_jt, gbase = A / groups, grem = A % groups;
    const long long a0 = g * gbase + (g < grem ? g : grem);
    const int rows = (int)(gbase + (g < grem ? 1 : 0));     // <= WARPS * RA
    const long long eoff = j0 + TJ - 1;

    {   // the whole pilot window, once
        const int elen = win_len(N);
        long long q0 = ((long long)tid - eoff) % nmod;
        if (q0 < 0) q0 += nmod;
        int q = (int)q0;
        const int step = 256 % nmod;
        for (int t = tid; t < elen; t += 256) {
            E[epos(t)] = pilot_value<MODE>(bits, preal, q, nmod);
            q += step;
            if (q >= nmod) q -= nmod;
        }
    }
    __syncthreads();
    // as a programmatic dependent (serving batches) the pilot window above overlapped the
    // kernel before; the row map and the rows are read only after it has finished
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // The group's rows spread over the warps as evenly as possible (rows / WARPS or one
    // more each), so that the four SM sub-partitions, which take warps w, w + 4 of each
    // block, carry nearly the same number of rows (27 rows as 4+4+4+3+3+3+3+3 rather than
    // six warps of 4, one of 3 computed as 4, and one idle).  No block-wide barrier below.
    const int rbase = rows / WARPS, rextra = rows % WARPS;
    const int nrw = rbase + (warp < rextra ? 1 : 0);
    const long long a_first = a0 + (long long)warp * rbase + (warp < rextra ? warp : rextra);
    if (nrw == 4) {
        if constexpr (RA >= 4)
            warp_rows<MODE, RA, 4, GRP>(sm, E, Y, y_stride, a_first, N, lags, col0, valid, invN, H,
                                   warp, lane, gio);
    } else if (nrw == 3) {
        if constexpr (RA >= 3)
            warp_rows<MODE, RA, 3, GRP>(sm, E, Y, y_stride, a_first, N, lags, col0, valid, invN, H,
                                   warp, lane, gio);
    } else if (nrw == 2) {
        if constexpr (RA >= 2)
            warp_rows<MODE, RA, 2, GRP>(sm, E, Y, y_stride, a_first, N, lags, col0, valid, invN, H,
                                   warp, lane, gio);
    } else if (nrw == 1) {
        warp_rows<MODE, RA, 1, GRP>(sm, E, Y, y_stride, a_first, N, lags, col0, valid, invN, H,
                                    warp, lane, gio);
    }
}

// Few lags (K*L <= 32, lags contiguous): the block tile above would leave most lanes idle,
// and at ~2 K*L flops per 8-byte sample the work is close to the HBM roofline.  One warp
// per received row: lane l takes the sample pairs (2p, 2p+1) for p = l, l+32, ... (four
// pairs in flight per lane, each sample read once; one 16-byte load per pair when the
// row is 16-byte aligned, two 8-byte loads otherwise -- the pairs, and so the order of
// every sum, do not depend on where the row lies, so the same row gives the same bits in
// any buffer) and reads the pilot bits of each sample as one window of the wrapped bit
// table.  With
// p = 1 - 2b, sum_n y[n] p[n-j] = S - 2 B_j, S = sum_n y[n] and B_j the sum of the samples
// whose bit b[n-j] is set, so each lag costs one bit test and one predicated packed add.
// A butterfly reduction over the warp (the same sum on every lane) ends the row and lane
// j stores lag j.
template <int KLM>
__device__ __forceinline__ void few_lags_sample(const uint32_t* __restrict__ ext, int N, int KL,
                                                int n, float2 v, float2& all,
                                                float2 (&acc)[KLM]) {
    // bits of samples n-KL+1 .. n (mod N): bit i of w is pilot bit q + i, and lag j meets
    // bit n - j, i.e. bit KL-1-j of w; the table wraps past N, so q < N keeps the window
    // inside it
    int q = n - (KL - 1);
    if (q < 0) q += N;
    const uint32_t lo = __ldg(ext + (q >> 5)), hi = __ldg(ext + (q >> 5) + 1);
    const uint32_t w = (uint32_t)((((uint64_t)hi << 32) | lo) >> (q & 31));
    all = __fadd2_rn(all, v);
    const uint32_t wr = __brev(w) >> (32 - KL);     // bit j of wr = bit KL-1-j of w
#pragma unroll
    for (int j = 0; j < KLM; ++j)
        if ((wr >> j) & 1u) acc[j] = __fadd2_rn(acc[j], v);
}

// Two consecutive samples n, n + 1 (n even): their bit windows come from one 64-bit read
// of the table (window offset q & 31 <= 31 plus K*L + 1 <= 33 bits fit in 64).
template <int KLM>
__device__ __forceinline__ void few_lags_pair(const uint32_t* __restrict__ ext, int N, int KL,
                                              int n, float2 v0, float2 v1, float2& all,
                                              float2 (&acc)[KLM]) {
    int q = n - (KL - 1);
    if (q < 0) q += N;
    const uint32_t lo = __ldg(ext + (q >> 5)), hi = __ldg(ext + (q >> 5) + 1);
    const uint64_t win = (((uint64_t)hi << 32) | lo) >> (q & 31);
    const uint32_t wr0 = __brev((uint32_t)win) >> (32 - KL);          // sample n
    const uint32_t wr1 = __brev((uint32_t)(win >> 1)) >> (32 - KL);   // sample n + 1
    all = __fadd2_rn(all, v0);
#pragma unroll
    for (int j = 0; j < KLM; ++j)
        if ((wr0 >> j) & 1u) acc[j] = __fadd2_rn(acc[j], v0);
    all = __fadd2_rn(all, v1);
#pragma unroll
    for (int j = 0; j < KLM; ++j)
        if ((wr1 >> j) & 1u) acc[j] = __fadd2_rn(acc[j], v1);
}

template <int KLM>
__global__ void __launch_bounds__(256)
simt_few_lags_kernel(const uint32_t* __restrict__ ext, const float2* __restrict__ Y,
                     long long y_stride, long long A, int N, int KL, int ldH, float invN,
                     float2* __restrict__ H) {
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long a = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < A;
         a += nwarps) {
        const float2* y = Y + a * y_stride;
        float2 acc[KLM];                       // B_j
        float2 all = make_float2(0.f, 0.f);     // S
#pragma unroll
        for (int j = 0; j < KLM; ++j) acc[j] = make_float2(0.f, 0.f);
        const bool al16 = ((uintptr_t)y & 15u) == 0;
        const int npairs = N >> 1;
        for (int p0 = lane; p0 < npairs; p0 += 4 * 32) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {               // the loads first: latency to hide
                const int p = p0 + 32 * u;
                v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (p < npairs) {
                    if (al16) {
                        v[u] = __ldcs(reinterpret_cast<const float4*>(y) + p);
                    } else {
                        const float2 a0 = __ldcs(y + 2 * p), a1 = __ldcs(y + 2 * p + 1);
                        v[u] = make_float4(a0.x, a0.y, a1.x, a1.y);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p = p0 + 32 * u;
                if (p < npairs)
                    few_lags_pair<KLM>(ext, N, KL, 2 * p, make_float2(v[u].x, v[u].y),
                                       make_float2(v[u].z, v[u].w), all, acc);
            }
        }
        // an odd last sample: the lane whose turn pair npairs would be
        if ((N & 1) && lane == (npairs & 31))
            few_lags_sample<KLM>(ext, N, KL, N - 1, __ldcs(y + N - 1), all, acc);
        // S over the warp, and B_j over the warp by a reduce-scatter: at each exchange
        // distance o the lanes split the remaining lags in halves, keep one half and send
        // the other, so lane j ends with the warp's B_j after 31 exchanges per part (a
        // butterfly per lag would chain 5 * K*L of them)
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            all.x += __shfl_xor_sync(0xffffffffu, all.x, o);
            all.y += __shfl_xor_sync(0xffffffffu, all.y, o);
        }
        float bx[32], by[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            bx[j] = j < KLM ? acc[j].x : 0.f;
            by[j] = j < KLM ? acc[j].y : 0.f;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < o; ++i) {
                const float sx = upper ? bx[i] : bx[i + o], kx = upper ? bx[i + o] : bx[i];
                const float sy = upper ? by[i] : by[i + o], ky = upper ? by[i + o] : by[i];
                bx[i] = kx + __shfl_xor_sync(0xffffffffu, sx, o);
                by[i] = ky + __shfl_xor_sync(0xffffffffu, sy, o);
            }
        }
        if (lane < KL)
            H[a * ldH + lane] =
                make_float2((all.x - 2.f * bx[0]) * invN, (all.y - 2.f * by[0]) * invN);
    }
}

template <int KLM>
cudaError_t launch_few(const uint32_t* ext, const float2* Y, long long y_stride, long long A,
                       int N, int KL, int ldH, float2* H, cudaStream_t s) {
    long long blocks = (A + 7) / 8;                 // 8 rows (warps) per block
    if (blocks > 8LL * 1024 * 152) blocks = 8LL * 1024 * 152;
    simt_few_lags_kernel<KLM><<<(unsigned)blocks, 256, 0, s>>>(
        ext, Y, y_stride, A, N, KL, ldH, (float)(1.0 / (double)N), H);
    return cudaGetLastError();
}

cudaError_t launch_few_lags(const uint32_t* ext, const float2* Y, long long y_stride,
                            long long A, int N, int KL, int ldH, float2* H, cudaStream_t s) {
    if (A <= 0) return cudaSuccess;
    if (KL <= 8) return launch_few<8>(ext, Y, y_stride, A, N, KL, ldH, H, s);
    if (KL <= 16) return launch_few<16>(ext, Y, y_stride, A, N, KL, ldH, H, s);
    return launch_few<32>(ext, Y, y_stride, A, N, KL, ldH, H, s);
}

constexpr int FEW_LAGS = 32;    // largest K*L the few-lags kernel takes

template <int MODE, int RA>
cudaError_t launch_ra(const uint32_t* bits, const float* preal, const float2* Y,
                      long long y_stride, long long A, int N, const pnce::LagMap& lags, int nmod,
                      int num_jt, long long groups, float2* H, cudaStream_t s,
                      const GroupedIO& g) {
    const long long blocks = (long long)num_jt * groups;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (win_len(N) <= WIN_MAX) {
        const size_t wsmem = sizeof(WSmem<RA>) + win_bytes(N);
        auto kern = simt_corr_warp_kernel<MODE, RA, false>;
        if constexpr (MODE == FWD_BITS) {
            if (g.dd) kern = simt_corr_warp_kernel<MODE, RA, true>;
        } else {
            if (g.dd) return cudaErrorNotSupported;
        }
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)wsmem);
        if (e != cudaSuccess) return e;
        const float invN = (float)(1.0 / (double)nmod);
        if (g.pdl) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)blocks, 1, 1);
            cfg.blockDim = dim3(256, 1, 1);
            cfg.dynamicSmemBytes = wsmem;
            cfg.stream = s;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            at[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            return cudaLaunchKernelEx(&cfg, kern, bits, preal, Y, y_stride, A, N, lags, nmod,
                                      num_jt, groups, invN, H, g);
        }
        kern<<<(unsigned)blocks, 256, wsmem, s>>>(bits, preal, Y, y_stride, A, N, lags, nmod,
                                                  num_jt, groups, invN, H, g);
        return cudaGetLastError();
    }
    if (g.dd) return cudaErrorNotSupported;    // the row I/O exists in the warp kernel only
    const size_t smem = sizeof(Smem<RA>);
    cudaError_t e = cudaFuncSetAttribute(simt_corr_kernel<MODE, RA>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const float invN = (float)(1.0 / (double)nmod);
    simt_corr_kernel<MODE, RA><<<(unsigned)blocks, 256, smem, s>>>(bits, preal, Y, y_stride, A, N,
                                                                   lags, nmod, num_jt, groups,
                                                                   invN, H);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch(const uint32_t* bits, const float* preal, const float2* Y, long long y_stride,
                   long long A, int N, const pnce::LagMap& lags, int nmod, float2* H,
                   cudaStream_t s, const GroupedIO& g = GroupedIO{}) {
    const long long num_jt_ll = pnce::lag_tiles(lags, TJ);
    if (num_jt_ll > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const int num_jt = (int)num_jt_ll;
    if (A <= 0 || num_jt <= 0) return cudaSuccess;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(simt_corr_kernel<MODE, 4>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sizeof(Smem<4>))) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, simt_corr_kernel<MODE, 4>, 256,
                                                           sizeof(Smem<4>))) != cudaSuccess)
        return e;
    const long long slots = (long long)sms * per_sm;
    long long groups = (A + 4 * WARPS - 1) / (4 * WARPS);
    if (slots > 0 && 2 * groups * num_jt < slots) {
        // A small grid (less than half of the resident 32-row blocks): blocks of 8 rows, one
        // antenna per thread, so each block is 4x shorter and a small batch finishes sooner.
        return launch_ra<MODE, 1>(bits, preal, Y, y_stride, A, N, lags, nmod, num_jt,
                                  (A + WARPS - 1) / WARPS, H, s, g);
    }
    // Otherwise 32-row groups, raised so that the grid fills whole waves of the resident
    // blocks (tiles of 2^k rows leave the last wave partly empty on 152 SMs).  Neither choice
    // changes a result: every output is summed over n in the same order.
    if (slots > 0) {
        const long long waves = (groups * num_jt + slots - 1) / slots;
        const long long even = waves * slots / num_jt;
        groups = std::min(A, std::max(groups, even));
    }
    return launch_ra<MODE, 4>(bits, preal, Y, y_stride, A, N, lags, nmod, num_jt, groups, H, s,
                              g);
}

}  // namespace

namespace pnce {

cudaError_t launch_simt_bits(const pnce_pilot* pilot, const float2* Y, long long A, int N,
                             int KL, float2* H, cudaStream_t s) {
    if (KL <= FEW_LAGS) return launch_few_lags(pilot->ext_bits_dev, Y, N, A, N, KL, KL, H, s);
    return launch<FWD_BITS>(pilot->ext_bits_dev, nullptr, Y, N, A, N, lagmap_contiguous(KL), N,
                            H, s);
}

bool simt_grouped_ok(int N, int kl_max) { return kl_max > FEW_LAGS && win_len(N) <= WIN_MAX; }
bool simt_grouped_reads_rows(int kl_max) { return kl_max <= TJ; }

cudaError_t launch_simt_grouped(const pnce_pilot* pilot, const pnce_req_desc* dd,
                                const int* row_req, long long rows, int N, int kl_max,
                                const float2* Yb, cudaStream_t s, bool pdl) {
    if (!simt_grouped_ok(N, kl_max)) return cudaErrorNotSupported;
    GroupedIO g;
    g.dd = dd;
    g.row_req = row_req;
    g.pdl = pdl;
    return launch<FWD_BITS>(pilot->ext_bits_dev, nullptr, Yb, N, rows, N,
                            lagmap_contiguous(kl_max), N, nullptr, s, g);
}

cudaError_t launch_simt_bits_ex(const pnce_pilot* pilot, const float2* Y, long long y_stride,
                                long long A, int N, const LagMap& lags, float2* H,
                                cudaStream_t s) {
    if (lags.mode == 0 && lags.ldH <= FEW_LAGS)
        return launch_few_lags(pilot->ext_bits_dev, Y, y_stride, A, N, lags.ldH, lags.ldH, H, s);
    return launch<FWD_BITS>(pilot->ext_bits_dev, nullptr, Y, y_stride, A, N, lags, N, H, s);
}

cudaError_t launch_simt_real(const float* p, bool tanh_map, const float2* Y, long long A, int N,
                             int KL, float2* H, cudaStream_t s) {
    const LagMap lm = lagmap_contiguous(KL);
    return tanh_map ? launch<FWD_TANH>(nullptr, p, Y, N, A, N, lm, N, H, s)
                    : launch<FWD_REAL>(nullptr, p, Y, N, A, N, lm, N, H, s);
}

cudaError_t launch_adjoint_dy(const float* p, bool tanh_map, const float2* G, long long A, int N,
                              int KL, float2* dY, cudaStream_t s) {
    // reduction over the KL lags of G, N outputs per row, pilot read backwards
    const LagMap lm = lagmap_contiguous(N);
    return tanh_map ? launch<ADJ_TANH>(nullptr, p, G, KL, A, KL, lm, N, dY, s)
                    : launch<ADJ_REAL>(nullptr, p, G, KL, A, KL, lm, N, dY, s);
}

}  // namespace pnce
