// Tensor-core correlation (Sec. III-B: the correlator of Eq. 3 / Eq. 10 as a matrix
// product on the tensor cores) for sm_103a: tcgen05.mma with FP32 accumulators in TMEM.
//
//   C[r][j] = sum_n A[r][n] * B[n][j],  B[n][j] = p[(n - j) mod N]  (the circulant, Eq. 2)
//
// A: the quantised received block in 8-antenna groups of 16 rows (the 8 real parts, then
//    the 8 imaginary parts), staged by TMA with the 128-byte swizzle in boxes of 128 rows
//    x 128 B (one K block), one or two boxes per pipeline stage.
// B: never stored in HBM.  The lag order inside a tile is reversed (tile column i holds
//    lag j0 + BN - 1 - i, j0 the tile's first lag: k*L-contiguous tiles, or per-transmitter
//    tiles when the transmitters' cyclic shifts are spread out), which turns the Toeplitz
//    tile into a Hankel one: the value at
//    (column 8q + r, sample n0 + EPR*t + c) is p[(s + G*(QS*q + TS*t) + r + c) mod N].
//    Every 8-row x 16-byte core matrix of the canonical no-swizzle K-major layout is then
//    one of a short list indexed by D = QS*q + TS*t, so the pilot operand of a stage is
//    that list alone, and the shared-memory descriptor's two core-matrix strides (LBO
//    along K, SBO along the lags) point into it with overlap.  Successive K blocks of one
//    lag block only shift along that list, so when it fits, the whole list for every K
//    block of the CTA's lag block (N/8 + BN/8 core matrices for 16-bit types, ~70 KB at
//    N = 4095) is generated once at kernel start and stays resident ("resident pilot");
//    otherwise one warp regenerates each stage's list (<= 78 core matrices, <= 10 KB).
// Epilogue: tcgen05.ld in the 16x256b shape hands each thread the real and imaginary
//    accumulators of one antenna for two adjacent columns (the group layout puts the two
//    parts 8 TMEM lanes apart), so after the per-antenna factor 2^-s_a / N each thread
//    writes one complex lag pair (16 B; an antenna's 4 threads write 64 contiguous bytes)
//    with no shuffles and no shared-memory staging.  TMEM holds two 256-column
//    accumulators so the epilogue of one tile overlaps the products of the next.
//
// Warp roles (256 threads, persistent, one CTA per SM): warp 0 TMA producer, warp 1 pilot
// tile generator, warp 2 TMEM allocator + MMA issuer, warps 4-7 epilogue (TMEM lane
// quarter = warp % 4).  Tiles t = blockIdx.x + i*gridDim.x map to (row block t / num_jt,
// lag block t % num_jt); with a grid that is a multiple of num_jt a CTA keeps one lag block
// and the CTAs sharing a row block run together, so A is read from HBM about once.
//
// Every mbarrier wait is bounded in time; on expiry the CTA latches PNCE_ETIMEOUT, all
// roles leave their loops, in-flight TMA loads and MMAs are drained (bounded), TMEM is
// freed and the kernel returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "pnce_internal.h"

namespace {

constexpr int THREADS = 256;
constexpr int BM = 128;                   // accumulator rows (TMEM lanes) per tile
constexpr int STAGES = 8;                 // maximum pipeline depth
constexpr int MAX_KPS = 2;                // K blocks per pipeline stage (TMA boxes, 4 MMAs each):
                                          // two halve the issuing thread's per-stage work per
                                          // MMA, when shared memory leaves room for 3 stages
constexpr int A_BOX = BM * 128;           // one TMA box: 128 rows x 128 B = 16 KB
constexpr int ACC_COLS = 256;
constexpr int TMEM_COLS = 512;
constexpr int MAX_BN = 256;
constexpr double EPI_SPREAD = 0.5;        // share of a tile's MMA time the epilogue spans

struct TcParams {
    int N;
    pnce::LagMap lags;      // which lags each lag tile holds and where they go in H
    long long A;            // antennas
    int BN;                 // lags per tile (multiple of 32, <= 256)
    int num_jt;             // lag blocks
    long long num_tiles;
    int num_kb;             // K blocks of 128-byte rows per tile
    int kps;                // K blocks per stage (1 or 2)
    int a_stage;            // operand bytes per stage: kps * A_BOX
    int num_st;             // pipeline stages per tile: ceil(num_kb / kps)
    int stages;             // pipeline depth (<= STAGES)
    int b_region;           // bytes of the pilot operand region
    int res_rows;           // resident pilot: 16-byte rows to generate (0 otherwise)
    int ext_words;          // words of the wrapped pilot bit table
    int drop_first_arrive;  // test hook: the per-stage pilot generator withholds its first
                            // arrive, so the MMA issuer's bounded wait must run out
    unsigned long long wait_limit_ns;
    long long epi_spacing;  // SM cycles between the epilogue's 64-column chunks (0: none)
    int* err;
};

template <int DT> struct TcFmt;
// BK: elements per 128-byte A row; EPR: elements per 16-byte core-matrix row;
// G: pilot offset per core-matrix index step; QS/TS: index step per lag / K core matrix.
template <> struct TcFmt<PNCE_FP16> {
    static constexpr int BK = 64, EPR = 8, G = 8, QS = 1, TS = 1;
    static constexpr uint32_t AB = (0u << 7) | (0u << 10);
};
template <> struct TcFmt<PNCE_BF16> {
    static constexpr int BK = 64, EPR = 8, G = 8, QS = 1, TS = 1;
    static constexpr uint32_t AB = (1u << 7) | (1u << 10);
};
template <> struct TcFmt<PNCE_FP8E4M3> {
    static constexpr int BK = 128, EPR = 16, G = 8, QS = 1, TS = 2;
    static constexpr uint32_t AB = (0u << 7) | (0u << 10);
};
template <> struct TcFmt<PNCE_TF32> {
    static constexpr int BK = 32, EPR = 4, G = 4, QS = 2, TS = 1;
    static constexpr uint32_t AB = (2u << 7) | (2u << 10);
};

template <int DT>
__host__ __device__ constexpr int ncm(int bn, int kps) {   // core matrices of one stage's pilot
    using F = TcFmt<DT>;                                   // operand (kps K blocks)
    return (bn / 8 - 1) * F::QS + (kps * F::BK / F::EPR - 1) * F::TS + 1;
}
template <int DT>
constexpr int b_stage_bytes() { return (ncm<DT>(MAX_BN, MAX_KPS) * 128 + 1023) / 1024 * 1024; }

struct Ctl {
    unsigned long long full_a[STAGES];
    unsigned long long full_b[STAGES];
    unsigned long long empty[STAGES];
    unsigned long long tfull[2];
    unsigned long long tempty[2];
    uint32_t tmem_base;
    int abort_flag;
};

constexpr size_t smem_fixed() { return 1024 /* alignment slack */ + sizeof(Ctl); }

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t su32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)),
                 "r"(bytes)
                 : "memory");
}
// CL: acquire at cluster scope, for phases completed by arrivals from the peer CTA
template <bool CL = false>
__device__ __forceinline__ bool mbar_test(unsigned long long* b, uint32_t parity) {
    uint32_t ok;
    if constexpr (CL) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(su32(b)), "r"(parity)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(su32(b)), "r"(parity)
            : "memory");
    }
    return ok != 0;
}

// Bounded wait for the phase of parity `parity` of barrier b.  honor_abort: give up as
// soon as another role has latched an abort.  Returns false when the wait was abandoned.
// The first test is inlined (the common case on the issue path); the loop is not.
template <bool CL = false>
__device__ __noinline__ bool wait_bar_slow(unsigned long long* b, uint32_t parity, Ctl* ctl,
                                           const TcParams& prm, bool honor_abort) {
    const unsigned long long t0 = gtime();
    for (;;) {
        if (mbar_test<CL>(b, parity)) return true;
        if (honor_abort && *(volatile int*)&ctl->abort_flag) return false;
        if (gtime() - t0 > prm.wait_limit_ns) {
            *(volatile int*)&ctl->abort_flag = 1;
            atomicCAS(prm.err, 0, (int)PNCE_ETIMEOUT);
            return false;
        }
    }
}
template <bool CL = false>
__device__ __forceinline__ bool wait_bar(unsigned long long* b, uint32_t parity, Ctl* ctl,
                                         const TcParams& prm, bool honor_abort) {
    return mbar_test<CL>(b, parity) || wait_bar_slow<CL>(b, parity, ctl, prm, honor_abort);
}
// The same bounded wait for a role that is not on the issue path (the epilogue waiting
// for an accumulator, ~a tile's worth of MMAs): polls with a short sleep in between, so
// that the polling does not take issue slots and shared-memory cycles from the producer
// and the MMA issuer.
__device__ __noinline__ bool wait_bar_sleepy(unsigned long long* b, uint32_t parity, Ctl* ctl,
                                             const TcParams& prm) {
    const unsigned long long t0 = gtime();
    for (;;) {
        if (mbar_test(b, parity)) return true;
        if (*(volatile int*)&ctl->abort_flag) return false;
        if (gtime() - t0 > prm.wait_limit_ns) {
            *(volatile int*)&ctl->abort_flag = 1;
            atomicCAS(prm.err, 0, (int)PNCE_ETIMEOUT);
            return false;
        }
        __nanosleep(256);
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor (tcgen05 format: start >> 4 in bits 0-13, leading
// byte offset >> 4 in 16-29, stride byte offset >> 4 in 32-45, version 1 in 46-47,
// layout type in 61-63: 0 = no swizzle, 2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo,
                                          uint32_t layout) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)layout << 61;
    return d;
}

template <int DT>
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                     uint32_t accumulate) {
    if constexpr (DT == PNCE_FP16 || DT == PNCE_BF16) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
            : "memory");
    } else if constexpr (DT == PNCE_TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            su32(bar))
        : "memory");
}

// 16 TMEM lanes x 64 columns: thread t receives, for each block x < 8 of 8 columns,
// v[4x] v[4x+1] = lane t/4, columns 8x + 2(t%4) + {0,1}, and v[4x+2] v[4x+3] = lane 8 + t/4,
// the same columns
__device__ __forceinline__ void tmem_ld16x256b_x8(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x8.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
        "[%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
          "=r"(v[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Epilogue of one 128-row accumulator (TMEM columns [0, BN) at `tacc`) by epilogue warp q,
// which owns TMEM lanes 32q .. 32q+31: operand rows of the 8-antenna groups 2q and 2q+1
// of the row block (first antenna ant_base).  Column c of the tile holds tile-local lag
// BN-1-c.  Thread t keeps antenna t/4 of each group: from the 16x256b layout it holds the
// real (lane t/4) and imaginary (lane 8+t/4) parts of columns 2u, 2u+1, i.e. the complex
// estimates of two adjacent lags, scaled and stored as one 16-byte write (4 threads of an
// antenna write 64 contiguous bytes).  `release` runs once the last TMEM load is done, so
// the MMA issuer may reuse the accumulator while the stores drain.  The chunks start
// `spacing` SM cycles apart: a tile's stores (128 KB per CTA at BN = 256) issued in one
// burst take the L1 data path from the tensor cores' operand reads for a while, spread
// over the next tile's products they cost less (measured: ~4 % of the kernel in a burst).
// Chunks [c_lo, c_hi) of the 64-column chunks are drained (the last tile of a CTA with one
// or two tiles is split between the epilogue warps and the idle role warps).
template <typename Release>
__device__ __forceinline__ void drain_accumulator(uint32_t tacc, int q, int lane,
                                                  long long ant_base, const float* row_scale,
                                                  float2* __restrict__ H, long long A, int ldH,
                                                  int BN, int col0, int valid,
                                                  long long spacing, int c_lo, int c_hi,
                                                  Release release) {
    const long long c0 = clock64();
    const int g = lane >> 2, u4 = lane & 3;
    long long ant[2];
    float rs[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        ant[h] = ant_base + 16 * q + 8 * h + g;
        rs[h] = ant[h] < A ? __ldg(row_scale + ant[h]) : 0.f;
    }
    const int nch = BN / 64 + ((BN & 63) ? 1 : 0);     // chunks of 64 columns (BN % 32 == 0)
    const int ce = c_hi < nch ? c_hi : nch;
    for (int c = c_lo; c < ce; ++c) {
        if (c > c_lo && spacing > 0) {
            // bounded: the target lies at most nch * spacing cycles after c0
            while (clock64() - c0 < (c - c_lo) * spacing) __nanosleep(128);
        }
        uint32_t v[2][32];
#pragma unroll
        for (int h = 0; h < 2; ++h)
            tmem_ld16x256b_x8(tacc + ((uint32_t)(32 * q + 16 * h) << 16) + 64u * c, v[h]);
        tmem_wait_ld();
        if (c == ce - 1) release();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (ant[h] >= A) continue;
            const long long off = ant[h] * ldH + col0;
            float2* row = H + off;
#pragma unroll
            for (int x = 0; x < 8; ++x) {
                const int col = 64 * c + 8 * x + 2 * u4;        // even column of the pair
                const int j = BN - 2 - col;                     // lag of column col + 1
                if (j < 0 || j >= valid) continue;
                const float4 val = make_float4(
                    __uint_as_float(v[h][4 * x + 1]) * rs[h], __uint_as_float(v[h][4 * x + 3]) * rs[h],
                    __uint_as_float(v[h][4 * x]) * rs[h], __uint_as_float(v[h][4 * x + 2]) * rs[h]);
                if (j + 1 < valid && (off & 1) == 0) {
                    *reinterpret_cast<float4*>(row + j) = val;
                } else {
                    row[j] = make_float2(val.x, val.y);
                    if (j + 1 < valid) row[j + 1] = make_float2(val.z, val.w);
                }
            }
        }
    }
}

// --------------------------------------------------------- pilot operand tiles

// 16 bytes holding EPR consecutive +-1 pilot values in the operand format, from the low
// EPR bits of x (bit c -> element c; bit 0 -> +1, bit 1 -> -1).
template <int DT>
__device__ __forceinline__ uint4 pilot_row(uint32_t x) {
    uint32_t w[4];
    if constexpr (DT == PNCE_FP16 || DT == PNCE_BF16) {
        constexpr uint32_t one = (DT == PNCE_FP16) ? 0x3C00u : 0x3F80u;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t b0 = (x >> (2 * i)) & 1u, b1 = (x >> (2 * i + 1)) & 1u;
            w[i] = (one | (b0 << 15)) | ((one | (b1 << 15)) << 16);
        }
    } else if constexpr (DT == PNCE_FP8E4M3) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t nib = (x >> (4 * i)) & 0xFu;
            w[i] = 0x38383838u | ((nib & 1u) << 7) | ((nib & 2u) << 14) | ((nib & 4u) << 21) |
                   ((nib & 8u) << 28);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = 0x3F800000u | (((x >> i) & 1u) << 31);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Pilot operand: core matrix D, row r (byte offset 128 D + 16 r) holds the EPR pilot
// values starting at sequence index s_start + G*D + r (mod N).  Rows idx = 8 D + r are
// shared out over nthr threads (a multiple of 8), thread `tid` taking tid, tid+nthr, ...
template <int DT, bool SMEM_EXT = false>
__device__ __forceinline__ void gen_pilot_rows(unsigned char* dst, const uint32_t* __restrict__ ext,
                                               int N, long long s_start, int rows, int tid,
                                               int nthr) {
    using F = TcFmt<DT>;
    // row idx has sequence offset G*(idx >> 3) + (idx & 7); a step of nthr rows is a
    // step of nthr/8 core matrices
    long long w0 = s_start + (long long)F::G * (tid >> 3) + (tid & 7);
    int pos = (int)(((w0 % N) + N) % N);
    const int step = (int)(((long long)F::G * (nthr >> 3)) % N);
    for (int idx = tid; idx < rows; idx += nthr) {
        uint32_t lo, hi;
        if constexpr (SMEM_EXT) {             // a copy of the table in shared memory
            lo = ext[pos >> 5];
            hi = ext[(pos >> 5) + 1];
        } else {
            lo = __ldg(ext + (pos >> 5));
            hi = __ldg(ext + (pos >> 5) + 1);
        }
        const uint64_t win = (((uint64_t)hi << 32) | lo) >> (pos & 31);
        const uint4 v = pilot_row<DT>((uint32_t)win);
        *reinterpret_cast<uint4*>(dst + (idx >> 3) * 128 + (idx & 7) * 16) = v;
        pos += step;
        while (pos >= N) pos -= N;
    }
}

// ------------------------------------------------------------------- the kernel

template <int DT, bool RES, int KPS>
__global__ void __launch_bounds__(THREADS, 1)
tc_corr_kernel(const __grid_constant__ CUtensorMap tmap, const uint32_t* __restrict__ ext,
               const float* __restrict__ row_scale, float2* __restrict__ H, const TcParams prm) {
    using F = TcFmt<DT>;
    constexpr int BSTAGE = b_stage_bytes<DT>();
    constexpr int KSTEPS = 4;                  // MMAs per K block: 128 B of K, 32 B each
    constexpr uint32_t LBO = 128u * F::TS, SBO = 128u * F::QS;
    constexpr uint32_t KSTEP_B = 2u * 128u * F::TS;       // B bytes per MMA K step

    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int nst = prm.stages;
    unsigned char* sA = base;
    unsigned char* sB = sA + nst * prm.a_stage;
    Ctl* ctl = reinterpret_cast<Ctl*>(sB + prm.b_region);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int BN = prm.BN, num_jt = prm.num_jt, num_st = prm.num_st;
    // tiles t = blockIdx.x + i * gridDim.x of this CTA
    const long long my_tiles =
        blockIdx.x < prm.num_tiles ? (prm.num_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    constexpr int kps = KPS;                    // K blocks per stage (prm.kps)
    constexpr int a_stage = KPS * A_BOX;        // prm.a_stage

    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&ctl->full_a[s], 1);
            mbar_init(&ctl->full_b[s], 1);
            mbar_init(&ctl->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ctl->tfull[b], 1);
            mbar_init(&ctl->tempty[b], 4);
        }
        ctl->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap))
                     : "memory");
    }
    if constexpr (RES) {
        // the CTA's lag block never changes (grid is a multiple of num_jt): build the
        // pilot operand of all its K blocks once.  The bit table is first copied into the
        // (still unused) operand stages with one coalesced pass, so that the generator's
        // reads are shared-memory hits instead of a chain of global-load latencies -- the
        // difference matters for grids of a few tiles (serving batches), where the set-up
        // is a large part of the kernel.
        long long j0;
        int col0, valid;
        pnce::lag_tile(prm.lags, BN, blockIdx.x % num_jt, j0, col0, valid);
        if (prm.ext_words <= prm.stages * a_stage / 4) {
            uint32_t* sx = reinterpret_cast<uint32_t*>(sA);
            for (int i = threadIdx.x; i < prm.ext_words; i += THREADS) sx[i] = __ldg(ext + i);
            __syncthreads();
            gen_pilot_rows<DT, true>(sB, sx, prm.N, -j0 - BN + 1, prm.res_rows, threadIdx.x,
                                     THREADS);
        } else {
            gen_pilot_rows<DT>(sB, ext, prm.N, -j0 - BN + 1, prm.res_rows, threadIdx.x, THREADS);
        }
        // orders these generic accesses to shared memory (the pilot operand written, the
        // table copy in the stages read) before the tensor cores and TMA use it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(&ctl->tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = ctl->tmem_base;
    // Launched as a programmatic dependent (serving batches), the set-up above overlapped
    // the kernel before this one; the operand, factors and H are touched only after it has
    // finished.  Without that launch attribute this returns at once.
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t stage = 0, phase = 0;
            long long issued = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < prm.num_tiles && ok; t += gridDim.x) {
                const int y = (int)(t / num_jt) * BM;
                for (int st = 0; st < num_st; ++st) {
                    if (!wait_bar(&ctl->empty[stage], phase ^ 1u, ctl, prm, true)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_tx(&ctl->full_a[stage], a_stage);
                    // boxes past the last K block read the fill value (zeros)
#pragma unroll
                    for (int h = 0; h < KPS; ++h)
                        tma_load_2d(sA + stage * a_stage + h * A_BOX, &tmap,
                                    (kps * st + h) * F::BK, y, &ctl->full_a[stage]);
                    ++issued;
                    if (++stage == (uint32_t)nst) { stage = 0; phase ^= 1u; }
                }
            }
            // drain: the last loads issued must have landed before the CTA may exit
            const long long first = issued > nst ? issued - nst : 0;
            for (long long i = first; i < issued; ++i)
                wait_bar(&ctl->full_a[i % nst], (uint32_t)((i / nst) & 1), ctl, prm, false);
        }
    } else if (warp == 1 && !RES) {
        // ---------------------------------------------------- pilot operand generator
        const int rows = ncm<DT>(BN, kps) * 8;
        uint32_t stage = 0, phase = 0;
        bool ok = true;
        for (long long t = blockIdx.x; t < prm.num_tiles && ok; t += gridDim.x) {
            long long j0;
            int col0, valid;
            pnce::lag_tile(prm.lags, BN, t % num_jt, j0, col0, valid);
            for (int st = 0; st < num_st; ++st) {
                int got = 1;
                if (lane == 0) got = wait_bar(&ctl->empty[stage], phase ^ 1u, ctl, prm, true);
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) { ok = false; break; }
                const long long s_start = (long long)kps * st * F::BK - j0 - BN + 1;
                gen_pilot_rows<DT>(sB + stage * BSTAGE, ext, prm.N, s_start, rows, lane, 32);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                const bool drop = prm.drop_first_arrive && t == blockIdx.x && st == 0;
                if (lane == 0 && !drop) mbar_arrive(&ctl->full_b[stage]);
                if (++stage == (uint32_t)nst) { stage = 0; phase ^= 1u; }
            }
        }
    } else if (warp == 2) {
        // ------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | F::AB | ((uint32_t)(BN >> 3) << 17) |
                                   ((uint32_t)(BM >> 4) << 24);
            // a descriptor's start field is the byte address / 16 in its low 14 bits, and
            // every operand lies below 256 KB, so moving a descriptor by a byte offset is a
            // 64-bit add of offset / 16 (keeps the issue loop short)
            const uint64_t adesc0 = sdesc(su32(sA), 16u, 1024u, 2u);
            const uint64_t bdesc0 = sdesc(su32(sB), LBO, SBO, 0u);
            uint32_t stage = 0, phase = 0, acc = 0, acc_phase = 0;
            unsigned long long* last_bar = nullptr;
            uint32_t last_par = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < prm.num_tiles && ok; t += gridDim.x) {
                if (!wait_bar(&ctl->tempty[acc], acc_phase ^ 1u, ctl, prm, true)) break;
                fence_after();
                const uint32_t d = tmem + acc * ACC_COLS;
                for (int st = 0; st < num_st; ++st) {
                    if (!wait_bar(&ctl->full_a[stage], phase, ctl, prm, true) ||
                        (!RES && !wait_bar(&ctl->full_b[stage], phase, ctl, prm, true))) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint64_t ad = adesc0 + (uint64_t)((stage * (uint32_t)a_stage) >> 4);
                    // resident: K block kb starts BK/EPR core matrices (times TS) further on;
                    // a stage's second K block is one such step after its first
                    const uint64_t bd =
                        bdesc0 + (uint64_t)(RES ? (8u * F::TS * (uint32_t)(kps * st * (F::BK / F::EPR)))
                                                : ((stage * (uint32_t)BSTAGE) >> 4));
#pragma unroll
                    for (int h = 0; h < KPS; ++h)
#pragma unroll
                        for (int ks = 0; ks < KSTEPS; ++ks)
                            umma<DT>(d, ad + (uint64_t)(h * (A_BOX >> 4)) + 2u * ks,
                                     bd + (uint64_t)(h * 8 * F::TS * (F::BK / F::EPR)) +
                                         (KSTEP_B >> 4) * ks,
                                     idesc, (st | h | ks) != 0);
                    umma_commit(&ctl->empty[stage]);
                    last_bar = &ctl->empty[stage];
                    last_par = phase;
                    if (++stage == (uint32_t)nst) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                umma_commit(&ctl->tfull[acc]);
                last_bar = &ctl->tfull[acc];
                last_par = acc_phase;
                acc ^= 1u;
                if (acc == 0) acc_phase ^= 1u;
            }
            if (last_bar) wait_bar(last_bar, last_par, ctl, prm, false);   // drain the MMAs
        }
    } else if (warp >= 4) {
        // --------------------------------------------------------------- epilogue
        const int q = warp & 3;                 // TMEM lane quarter
        uint32_t acc = 0, acc_phase = 0;
        for (long long t = blockIdx.x; t < prm.num_tiles; t += gridDim.x) {
            const long long rb = t / num_jt;
            long long j0;                       // first lag of the tile (unused here)
            int col0, valid;                    // first output column, lags kept
            pnce::lag_tile(prm.lags, BN, t % num_jt, j0, col0, valid);
            int got = 1;
            if (lane == 0) got = wait_bar_sleepy(&ctl->tfull[acc], acc_phase, ctl, prm);
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) break;
            fence_after();
            unsigned long long* te = &ctl->tempty[acc];
            // pacing spreads the stores over the next tile's products; a CTA's last tile
            // has none to overlap, so its stores go out at once, and in a CTA of one or two
            // tiles the idle role warps drain the second half of its columns
            const bool last = t + gridDim.x >= prm.num_tiles;
            const long long spacing = last ? 0 : prm.epi_spacing;
            const int nch = (BN + 63) / 64;
            const int c_hi = last && my_tiles <= 2 ? (nch + 1) / 2 : nch;
            drain_accumulator(tmem + acc * ACC_COLS, q, lane, rb * (BM / 2), row_scale, H,
                              prm.A, prm.lags.ldH, BN, col0, valid, spacing, 0, c_hi, [&] {
                                  fence_before();
                                  __syncwarp();
                                  if (lane == 0) mbar_arrive(te);
                              });
            acc ^= 1u;
            if (acc == 0) acc_phase ^= 1u;
        }
    }

    if (warp < 4 && my_tiles >= 1 && my_tiles <= 2) {
        // Warps 0-3 have finished their roles (warps 0 and 2 only in lane 0) and drain the
        // second half of the columns of the CTA's last tile, with the epilogue warp of the
        // same TMEM lane quarter.  With one or two tiles per CTA the last tile is the first
        // use of its accumulator barrier, so the wait below cannot be satisfied by an
        // earlier phase.
        __syncwarp();
        const long long il = my_tiles - 1;
        const long long t = blockIdx.x + il * gridDim.x;
        const uint32_t acc = (uint32_t)(il & 1);
        const int nch = (BN + 63) / 64;
        const int c_lo = (nch + 1) / 2;
        if (c_lo < nch) {
            long long j0;
            int col0, valid;
            pnce::lag_tile(prm.lags, BN, t % num_jt, j0, col0, valid);
            int got = 1;
            if (lane == 0) got = wait_bar_sleepy(&ctl->tfull[acc], 0u, ctl, prm);
            got = __shfl_sync(0xffffffffu, got, 0);
            if (got) {
                fence_after();
                drain_accumulator(tmem + acc * ACC_COLS, warp & 3, lane, (t / num_jt) * (BM / 2),
                                  row_scale, H, prm.A, prm.lags.ldH, BN, col0, valid, 0, c_lo,
                                  nch, [] {});
            }
        }
    }

    fence_before();
    __syncthreads();
    if (warp == 2) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

// ------------------------------------------------ 2-SM variant (CTA pairs, opt-in)
//
// tcgen05.mma.cta_group::2 over a cluster of two CTAs: the pair computes a 256-row x BN-lag
// tile; each CTA stages its own 128 operand rows and holds the pilot list of its half of
// the BN lags (rank 0: tile columns [0, BN/2), rank 1: [BN/2, BN)), so each SM reads half
// the pilot operand per MMA.  Rank 0 issues the MMAs for both; the operand loads of both
// CTAs complete on rank 0's stage barrier, its commits arrive on the barriers of both CTAs
// (one commit per CTA), and each CTA drains its own 128 accumulator rows, the odd CTA
// releasing rank 0's accumulator barrier remotely.

struct PairCtl {
    unsigned long long full_a[STAGES];
    unsigned long long unused[STAGES];      // keeps the layout of Ctl
    unsigned long long empty[STAGES];
    unsigned long long tfull[2];
    unsigned long long tempty[2];           // rank 0: 4 local + 4 remote epilogue warps
    uint32_t tmem_base;
    int abort_flag;
};
// same layout as Ctl, so that wait_bar's abort flag is the pair's
static_assert(sizeof(PairCtl) == sizeof(Ctl) && offsetof(PairCtl, abort_flag) == offsetof(Ctl, abort_flag),
              "control block layout");

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}
// arrive on the barrier at the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ void mbar_arrive_remote(unsigned long long* local, uint32_t rank) {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(su32(local)), "r"(rank));
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote)
                 : "memory");
}
__device__ __forceinline__ uint32_t cluster_addr(const void* local, uint32_t rank) {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(su32(local)), "r"(rank));
    return remote;
}
// commit the issuing thread's MMAs to the barrier at this offset in each CTA of the pair
// (one commit per CTA; each tracks all MMAs the thread issued before it)
__device__ __forceinline__ void umma_commit_pair(unsigned long long* bar) {
#pragma unroll
    for (uint32_t r = 0; r < 2; ++r)
        asm volatile(
            "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                cluster_addr(bar, r))
            : "memory");
}

// TMA load into this CTA's shared memory whose completion is counted on the barrier at
// shared::cluster address `bar_cluster`, which may belong to the peer CTA of the pair
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, int x, int y,
                                                 uint32_t bar_cluster) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar_cluster)
        : "memory");
}
template <int DT>
__device__ __forceinline__ void umma_pair(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
    if constexpr (DT == PNCE_FP16 || DT == PNCE_BF16) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
            : "memory");
    } else if constexpr (DT == PNCE_TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

template <int DT, int KPS>
__global__ void __launch_bounds__(THREADS, 1)
tc_pair_kernel(const __grid_constant__ CUtensorMap tmap, const uint32_t* __restrict__ ext,
               const float* __restrict__ row_scale, float2* __restrict__ H, const TcParams prm) {
    using F = TcFmt<DT>;
    constexpr int KSTEPS = 4;
    constexpr uint32_t LBO = 128u * F::TS, SBO = 128u * F::QS;
    constexpr uint32_t KSTEP_B = 2u * 128u * F::TS;

    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int nst = prm.stages;
    unsigned char* sA = base;
    unsigned char* sB = sA + nst * prm.a_stage;
    PairCtl* ctl = reinterpret_cast<PairCtl*>(sB + prm.b_region);
    Ctl* wctl = reinterpret_cast<Ctl*>(ctl);    // abort flag shared with wait_bar

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int BN = prm.BN, num_jt = prm.num_jt, num_st = prm.num_st;
    constexpr int kps = KPS;                    // K blocks per stage (prm.kps)
    constexpr int a_stage = KPS * A_BOX;        // prm.a_stage
    const uint32_t rank = cluster_rank();
    const long long pair = cluster_id(), npairs = cluster_count();

    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&ctl->full_a[s], 1);
            mbar_init(&ctl->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ctl->tfull[b], 1);
            mbar_init(&ctl->tempty[b], 8);
        }
        ctl->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap))
                     : "memory");
    }
    {
        // this CTA's half of the pair's lag block: rank 0 the later lags (tile columns
        // [0, BN/2)), rank 1 the earlier ones; the pair keeps its lag block throughout
        long long j0;
        int col0, valid;
        pnce::lag_tile(prm.lags, BN, pair % num_jt, j0, col0, valid);
        const int bnc = BN / 2;
        const long long origin = j0 + (rank == 0 ? bnc : 0);
        gen_pilot_rows<DT>(sB, ext, prm.N, -origin - bnc + 1, prm.res_rows, threadIdx.x, THREADS);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(&ctl->tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    cluster_sync_all();      // barriers of both CTAs initialised, both pilot halves built
    fence_after();
    const uint32_t tmem = ctl->tmem_base;

    if (warp == 0) {
        // ------------------------------------------------- TMA producer (both CTAs)
        // both CTAs' loads of a stage complete on rank 0's full_a, which expects the bytes
        // of both; each CTA refills a stage when the pair's MMAs have released it (the
        // commit arrives on the empty barriers of both CTAs)
        if (lane == 0) {
            const uint32_t full0 = cluster_addr(&ctl->full_a[0], 0);
            uint32_t stage = 0, phase = 0;
            long long issued = 0;
            bool ok = true;
            for (long long t = pair; t < prm.num_tiles && ok; t += npairs) {
                const int y = (int)(2 * (t / num_jt) + rank) * BM;
                for (int st = 0; st < num_st; ++st) {
                    if (!wait_bar(&ctl->empty[stage], phase ^ 1u, wctl, prm, true)) {
                        ok = false;
                        break;
                    }
                    if (rank == 0) mbar_arrive_tx(&ctl->full_a[stage], 2 * a_stage);
#pragma unroll
                    for (int h = 0; h < KPS; ++h)
                        tma_load_2d_pair(sA + stage * a_stage + h * A_BOX, &tmap,
                                         (kps * st + h) * F::BK, y,
                                         full0 + stage * (uint32_t)sizeof(unsigned long long));
                    ++issued;
                    if (++stage == (uint32_t)nst) { stage = 0; phase ^= 1u; }
                }
            }
            // drain (rank 0): the last stages' loads of both CTAs must have landed before
            // the pair may exit; rank 1 leaves only after the closing cluster barrier
            if (rank == 0) {
                const long long first = issued > nst ? issued - nst : 0;
                for (long long i = first; i < issued; ++i)
                    wait_bar<true>(&ctl->full_a[i % nst], (uint32_t)((i / nst) & 1), wctl, prm,
                                   false);
            }
        }
    } else if (warp == 2) {
        // ------------------------------------------------ MMA issuer (rank 0 only)
        if (rank == 0 && lane == 0) {
            const uint32_t idesc = (1u << 4) | F::AB | ((uint32_t)(BN >> 3) << 17) |
                                   ((uint32_t)(2 * BM >> 4) << 24);
            const uint64_t adesc0 = sdesc(su32(sA), 16u, 1024u, 2u);
            const uint64_t bdesc0 = sdesc(su32(sB), LBO, SBO, 0u);
            uint32_t stage = 0, phase = 0, acc = 0, acc_phase = 0;
            unsigned long long* last_bar = nullptr;
            uint32_t last_par = 0;
            bool ok = true;
            for (long long t = pair; t < prm.num_tiles && ok; t += npairs) {
                if (!wait_bar<true>(&ctl->tempty[acc], acc_phase ^ 1u, wctl, prm, true)) break;
                fence_after();
                const uint32_t d = tmem + acc * ACC_COLS;
                for (int st = 0; st < num_st; ++st) {
                    if (!wait_bar<true>(&ctl->full_a[stage], phase, wctl, prm, true)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint64_t ad = adesc0 + (uint64_t)((stage * (uint32_t)a_stage) >> 4);
                    const uint64_t bd =
                        bdesc0 + (uint64_t)(8u * F::TS * (uint32_t)(kps * st * (F::BK / F::EPR)));
#pragma unroll
                    for (int h = 0; h < KPS; ++h)
#pragma unroll
                        for (int ks = 0; ks < KSTEPS; ++ks)
                            umma_pair<DT>(d, ad + (uint64_t)(h * (A_BOX >> 4)) + 2u * ks,
                                          bd + (uint64_t)(h * 8 * F::TS * (F::BK / F::EPR)) +
                                              (KSTEP_B >> 4) * ks,
                                          idesc, (st | h | ks) != 0);
                    umma_commit_pair(&ctl->empty[stage]);
                    last_bar = &ctl->empty[stage];
                    last_par = phase;
                    if (++stage == (uint32_t)nst) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                umma_commit_pair(&ctl->tfull[acc]);
                last_bar = &ctl->tfull[acc];
                last_par = acc_phase;
                acc ^= 1u;
                if (acc == 0) acc_phase ^= 1u;
            }
            if (last_bar) wait_bar(last_bar, last_par, wctl, prm, false);
        }
    } else if (warp >= 4) {
        // ------------------------------------------------------ epilogue (both CTAs)
        const int q = warp & 3;
        uint32_t acc = 0, acc_phase = 0;
        for (long long t = pair; t < prm.num_tiles; t += npairs) {
            const long long rb = 2 * (t / num_jt) + rank;
            long long j0;
            int col0, valid;
            pnce::lag_tile(prm.lags, BN, t % num_jt, j0, col0, valid);
            int got = 1;
            if (lane == 0) got = wait_bar_sleepy(&ctl->tfull[acc], acc_phase, wctl, prm);
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) break;
            fence_after();
            unsigned long long* te = &ctl->tempty[acc];
            drain_accumulator(tmem + acc * ACC_COLS, q, lane, rb * (BM / 2), row_scale, H,
                              prm.A, prm.lags.ldH, BN, col0, valid, prm.epi_spacing, 0,
                              (BN + 63) / 64, [&] {
                                  fence_before();
                                  __syncwarp();
                                  if (lane == 0) {
                                      if (rank == 0) mbar_arrive(te);
                                      else mbar_arrive_remote(te, 0);
                                  }
                              });
            acc ^= 1u;
            if (acc == 0) acc_phase ^= 1u;
        }
    }

    fence_before();
    __syncthreads();
    cluster_sync_all();      // the peer no longer reads this CTA's shared memory or barriers
    if (warp == 2) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------- lag-major variant (tiles of <= 128 lags)
//
// With the transmitters' cyclic shifts spread out (Eq. 8), a lag tile is one transmitter's
// L lags; at L = 128 the kernel above would issue MMAs of N = 128, whose operand reads
// (4 KB of received rows + 4 KB of pilot per 64 clocks) exceed the shared-memory data
// path.  Here the roles swap: the pilot tile (128 lags x K, the same Hankel core-matrix
// list, resident for all K blocks) is the A operand and 256 received operand rows
// (128 antennas, one 32 KB TMA box per K block) are the B operand, so every MMA is again
// M = 128 x N = 256 (4 KB + 8 KB per 128 clocks).  The accumulator then holds lags in its
// TMEM lanes and operand rows in its columns: a 32x32b load gives each epilogue thread one
// lag for 32 operand rows -- the real and imaginary parts of 16 antennas -- and a warp's
// store writes 32 consecutive lags (256 bytes) of one antenna.

constexpr int BR = 256;                   // operand rows per lag-major tile (the MMA's N)
constexpr int Y_BOX = BR * 128;           // one TMA box of them: 256 rows x 128 B = 32 KB

// 32 TMEM lanes x 32 columns: thread t receives lane (base + t), columns c .. c+31
__device__ __forceinline__ void tmem_ld32x32b_x32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
        "[%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
          "=r"(v[31])
        : "r"(taddr));
}

// Lag-major tiles on single CTAs: the pilot is the A operand (128 lags, M), the received
// rows the B operand (256 rows, N), so a warp of the epilogue stores 32 consecutive lags of
// one antenna.  A CTA streams a 256-row stage per 128 MMA clocks, twice the contiguous
// kernel's rate; the 2-SM pair kernel below halves that per SM and is the default.
template <int DT>
__global__ void __launch_bounds__(THREADS, 1)
tc_lagmajor_kernel(const __grid_constant__ CUtensorMap tmap, const uint32_t* __restrict__ ext,
                   const float* __restrict__ row_scale, float2* __restrict__ H,
                   const TcParams prm) {
    using F = TcFmt<DT>;
    constexpr int KSTEPS = 4;                  // MMAs per K block: 128 B of K, 32 B each
    constexpr int TL = 128;                    // lags per tile (the MMA's M)
    constexpr uint32_t LBO = 128u * F::TS, SBO = 128u * F::QS;
    constexpr uint32_t KSTEP_P = 2u * 128u * F::TS;       // pilot bytes per MMA K step

    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int nst = prm.stages;
    unsigned char* sY = base;
    unsigned char* sP = sY + nst * Y_BOX;
    Ctl* ctl = reinterpret_cast<Ctl*>(sP + prm.b_region);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int num_jt = prm.num_jt, num_kb = prm.num_kb;
    // Work units u = unit0 + i * nunits over (row block, lag tile); the CTA's lag tile is
    // fixed because the grid is a multiple of the lag tiles.
    const long long unit0 = blockIdx.x, nunits = gridDim.x;
    const int ngroups = num_jt;
    const long long total_units = prm.num_tiles;
    const int jt_own = (int)(unit0 % ngroups);

    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&ctl->full_a[s], 1);
            mbar_init(&ctl->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ctl->tfull[b], 1);
            mbar_init(&ctl->tempty[b], 4);
        }
        ctl->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap))
                     : "memory");
    }
    {
        // the CTA's lag block is fixed (the grid is a multiple of num_jt): its pilot operand
        // for every K block, generated once from a shared-memory copy of the bit table
        long long j0;
        int col0, valid;
        pnce::lag_tile(prm.lags, TL, jt_own, j0, col0, valid);
        if (prm.ext_words <= nst * Y_BOX / 4) {
            uint32_t* sx = reinterpret_cast<uint32_t*>(sY);
            for (int i = threadIdx.x; i < prm.ext_words; i += THREADS) sx[i] = __ldg(ext + i);
            __syncthreads();
            gen_pilot_rows<DT, true>(sP, sx, prm.N, -j0 - TL + 1, prm.res_rows, threadIdx.x,
                                     THREADS);
        } else {
            gen_pilot_rows<DT>(sP, ext, prm.N, -j0 - TL + 1, prm.res_rows, threadIdx.x, THREADS);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(&ctl->tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = ctl->tmem_base;
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t stage = 0, phase = 0;
            long long issued = 0;
            bool ok = true;
            for (long long u = unit0; u < total_units && ok; u += nunits) {
                const int y = (int)(u / ngroups) * BR;
                for (int kb = 0; kb < num_kb; ++kb) {
                    if (!wait_bar(&ctl->empty[stage], phase ^ 1u, ctl, prm, true)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_tx(&ctl->full_a[stage], Y_BOX);
                    tma_load_2d(sY + stage * Y_BOX, &tmap, kb * F::BK, y, &ctl->full_a[stage]);
                    ++issued;
                    if (++stage == (uint32_t)nst) { stage = 0; phase ^= 1u; }
                }
            }
            const long long first = issued > nst ? issued - nst : 0;
            for (long long i = first; i < issued; ++i)
                wait_bar(&ctl->full_a[i % nst], (uint32_t)((i / nst) & 1), ctl, prm, false);
        }
    } else if (warp == 2) {
        // ------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | F::AB | ((uint32_t)(BR >> 3) << 17) |
                                   ((uint32_t)(BM >> 4) << 24);
            const uint64_t pdesc0 = sdesc(su32(sP), LBO, SBO, 0u);      // A: pilot, Hankel list
            const uint64_t ydesc0 = sdesc(su32(sY), 16u, 1024u, 2u);    // B: rows, 128B swizzle
            uint32_t stage = 0, phase = 0, acc = 0, acc_phase = 0;
            unsigned long long* last_bar = nullptr;
            uint32_t last_par = 0;
            bool ok = true;
            for (long long u = unit0; u < total_units && ok; u += nunits) {
                if (!wait_bar(&ctl->tempty[acc], acc_phase ^ 1u, ctl, prm, true)) break;
                fence_after();
                const uint32_t d = tmem + acc * ACC_COLS;
                for (int kb = 0; kb < num_kb; ++kb) {
                    if (!wait_bar(&ctl->full_a[stage], phase, ctl, prm, true)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    // K block kb of the pilot starts BK/EPR core matrices (times TS) further on
                    const uint64_t pd =
                        pdesc0 + (uint64_t)(8u * F::TS * (uint32_t)(kb * (F::BK / F::EPR)));
                    const uint64_t yd = ydesc0 + (uint64_t)((stage * (uint32_t)Y_BOX) >> 4);
#pragma unroll
                    for (int ks = 0; ks < KSTEPS; ++ks)
                        umma<DT>(d, pd + (KSTEP_P >> 4) * ks, yd + 2u * ks, idesc,
                                 (kb | ks) != 0);
                    umma_commit(&ctl->empty[stage]);
                    last_bar = &ctl->empty[stage];
                    last_par = phase;
                    if (++stage == (uint32_t)nst) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                umma_commit(&ctl->tfull[acc]);
                last_bar = &ctl->tfull[acc];
                last_par = acc_phase;
                acc ^= 1u;
                if (acc == 0) acc_phase ^= 1u;
            }
            if (last_bar) wait_bar(last_bar, last_par, ctl, prm, false);   // drain the MMAs
        }
    } else if (warp >= 4) {
        // --------------------------------------------------------------- epilogue
        // Warp q owns TMEM lanes 32q .. 32q+31; lane i of the tile holds tile-local lag
        // TL - 1 - i (reversed order, which makes the pilot tile a Hankel one).
        const int q = warp & 3;
        const int o = TL - 1 - (32 * q + lane);          // this thread's lag in the tile
        uint32_t acc = 0, acc_phase = 0;
        for (long long u = unit0; u < total_units; u += nunits) {
            const long long ant0 = (u / ngroups) * (BR / 2);
            long long j0;
            int col0, valid;
            pnce::lag_tile(prm.lags, TL, jt_own, j0, col0, valid);
            int got = 1;
            if (lane == 0) got = wait_bar_sleepy(&ctl->tfull[acc], acc_phase, ctl, prm);
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) break;
            fence_after();
            const uint32_t tacc = tmem + acc * ACC_COLS + ((uint32_t)(32 * q) << 16);
            const long long spacing = u + nunits < total_units ? prm.epi_spacing : 0;
            const long long c0 = clock64();
            float2* hcol = H + col0 + o;
            for (int c = 0; c < BR / 32; ++c) {              // 32 operand rows = 16 antennas
                if (c > 0 && spacing > 0) {
                    // bounded: the target lies at most 8 * spacing cycles after c0
                    while (clock64() - c0 < c * spacing) __nanosleep(128);
                }
                uint32_t v[32];
                tmem_ld32x32b_x32(tacc + 32u * c, v);
                tmem_wait_ld();
                if (c == BR / 32 - 1) {
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&ctl->tempty[acc]);
                }
                if (o < valid) {
#pragma unroll
                    for (int g = 0; g < 2; ++g) {
#pragma unroll
                        for (int a = 0; a < 8; ++a) {
                            const long long ant = ant0 + 16 * c + 8 * g + a;
                            if (ant < prm.A) {
                                const float rs = __ldg(row_scale + ant);
                                hcol[ant * prm.lags.ldH] =
                                    make_float2(__uint_as_float(v[16 * g + a]) * rs,
                                                __uint_as_float(v[16 * g + 8 + a]) * rs);
                            }
                        }
                    }
                }
            }
            acc ^= 1u;
            if (acc == 0) acc_phase ^= 1u;
        }
    }

    fence_before();
    __syncthreads();
    if (warp == 2) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

// Lag-major tiles on CTA pairs with the 2-SM MMA (tcgen05.mma.cta_group::2, M = 256):
// each CTA of a cluster holds its own lag tile's pilot list (the A rows of its half of M)
// and TMA-loads its own half of the 256 received rows (the B columns of its half of N), so
// an SM writes 32 B/clock of rows into shared memory and its tensor core reads 64 B/clock
// of operands -- in the single-CTA lag-major kernel the 256-row stages alone asked for
// 64 B/clock of writes on top of 96 B/clock of reads, beyond the 128 B/clock data path.
// Rank 0 issues the MMAs of the pair; both CTAs' loads complete on rank 0's stage
// barrier; MMA completion arrives on the barriers of both; each CTA drains its own lags
// for all 256 rows, rank 1 releasing rank 0's accumulator barrier remotely.
template <int DT, int KPS>
__global__ void __launch_bounds__(THREADS, 1)
tc_lagmajor_pair_kernel(const __grid_constant__ CUtensorMap tmap, const uint32_t* __restrict__ ext,
                        const float* __restrict__ row_scale, float2* __restrict__ H,
                        const TcParams prm) {
    using F = TcFmt<DT>;
    constexpr int KSTEPS = 4;
    constexpr int TL = 128;
    constexpr uint32_t LBO = 128u * F::TS, SBO = 128u * F::QS;
    constexpr uint32_t KSTEP_P = 2u * 128u * F::TS;
    constexpr int a_stage = KPS * A_BOX;        // this CTA's 128 rows of KPS K blocks

    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int nst = prm.stages;
    unsigned char* sY = base;
    unsigned char* sP = sY + nst * a_stage;
    PairCtl* ctl = reinterpret_cast<PairCtl*>(sP + prm.b_region);
    Ctl* wctl = reinterpret_cast<Ctl*>(ctl);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int num_jt = prm.num_jt, num_st = prm.num_st;
    const uint32_t rank = cluster_rank();
    const long long unit0 = cluster_id(), nunits = cluster_count();
    const int ngroups = num_jt / 2;
    const long long total_units = prm.num_tiles / 2;
    const int jt_own = (int)(unit0 % ngroups) * 2 + (int)rank;

    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&ctl->full_a[s], 1);
            mbar_init(&ctl->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ctl->tfull[b], 1);
            mbar_init(&ctl->tempty[b], 8);
        }
        ctl->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap))
                     : "memory");
    }
    {
        long long j0;
        int col0, valid;
        pnce::lag_tile(prm.lags, TL, jt_own, j0, col0, valid);
        if (prm.ext_words <= nst * a_stage / 4) {
            uint32_t* sx = reinterpret_cast<uint32_t*>(sY);
            for (int i = threadIdx.x; i < prm.ext_words; i += THREADS) sx[i] = __ldg(ext + i);
            __syncthreads();
            gen_pilot_rows<DT, true>(sP, sx, prm.N, -j0 - TL + 1, prm.res_rows, threadIdx.x,
                                     THREADS);
        } else {
            gen_pilot_rows<DT>(sP, ext, prm.N, -j0 - TL + 1, prm.res_rows, threadIdx.x, THREADS);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(&ctl->tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    cluster_sync_all();      // barriers of both CTAs initialised, both pilot lists built
    fence_after();
    const uint32_t tmem = ctl->tmem_base;
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (warp == 0) {
        // ------------------------------------------------- TMA producer (both CTAs)
        if (lane == 0) {
            const uint32_t full0 = cluster_addr(&ctl->full_a[0], 0);
            uint32_t stage = 0, phase = 0;
            long long issued = 0;
            bool ok = true;
            for (long long u = unit0; u < total_units && ok; u += nunits) {
                const int y = (int)(u / ngroups) * BR + (int)rank * BM;
                for (int st = 0; st < num_st; ++st) {
                    if (!wait_bar(&ctl->empty[stage], phase ^ 1u, wctl, prm, true)) {
                        ok = false;
                        break;
                    }
                    if (rank == 0) mbar_arrive_tx(&ctl->full_a[stage], 2 * a_stage);
#pragma unroll
                    for (int h = 0; h < KPS; ++h)
                        tma_load_2d_pair(sY + stage * a_stage + h * A_BOX, &tmap,
                                         (KPS * st + h) * F::BK, y,
                                         full0 + stage * (uint32_t)sizeof(unsigned long long));
                    ++issued;
                    if (++stage == (uint32_t)nst) { stage = 0; phase ^= 1u; }
                }
            }
            if (rank == 0) {
                const long long first = issued > nst ? issued - nst : 0;
                for (long long i = first; i < issued; ++i)
                    wait_bar<true>(&ctl->full_a[i % nst], (uint32_t)((i / nst) & 1), wctl, prm,
                                   false);
            }
        }
    } else if (warp == 2) {
        // ------------------------------------------------ MMA issuer (rank 0 only)
        if (rank == 0 && lane == 0) {
            const uint32_t idesc = (1u << 4) | F::AB | ((uint32_t)(BR >> 3) << 17) |
                                   ((uint32_t)(2 * BM >> 4) << 24);
            const uint64_t pdesc0 = sdesc(su32(sP), LBO, SBO, 0u);     // A: pilot lists
            const uint64_t ydesc0 = sdesc(su32(sY), 16u, 1024u, 2u);   // B: row halves
            uint32_t stage = 0, phase = 0, acc = 0, acc_phase = 0;
            unsigned long long* last_bar = nullptr;
            uint32_t last_par = 0;
            bool ok = true;
            for (long long u = unit0; u < total_units && ok; u += nunits) {
                if (!wait_bar<true>(&ctl->tempty[acc], acc_phase ^ 1u, wctl, prm, true)) break;
                fence_after();
                const uint32_t d = tmem + acc * ACC_COLS;
                for (int st = 0; st < num_st; ++st) {
                    if (!wait_bar<true>(&ctl->full_a[stage], phase, wctl, prm, true)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint64_t yd = ydesc0 + (uint64_t)((stage * (uint32_t)a_stage) >> 4);
                    const uint64_t pd =
                        pdesc0 + (uint64_t)(8u * F::TS * (uint32_t)(KPS * st * (F::BK / F::EPR)));
#pragma unroll
                    for (int h = 0; h < KPS; ++h)
#pragma unroll
                        for (int ks = 0; ks < KSTEPS; ++ks)
                            umma_pair<DT>(d,
                                          pd + (uint64_t)(h * 8 * F::TS * (F::BK / F::EPR)) +
                                              (KSTEP_P >> 4) * ks,
                                          yd + (uint64_t)(h * (A_BOX >> 4)) + 2u * ks, idesc,
                                          (st | h | ks) != 0);
                    umma_commit_pair(&ctl->empty[stage]);
                    last_bar = &ctl->empty[stage];
                    last_par = phase;
                    if (++stage == (uint32_t)nst) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                umma_commit_pair(&ctl->tfull[acc]);
                last_bar = &ctl->tfull[acc];
                last_par = acc_phase;
                acc ^= 1u;
                if (acc == 0) acc_phase ^= 1u;
            }
            if (last_bar) wait_bar(last_bar, last_par, wctl, prm, false);
        }
    } else if (warp >= 4) {
        // ------------------------------------------------------ epilogue (both CTAs)
        // lanes: this CTA's 128 lags (lane i holds tile-local lag TL - 1 - i); columns:
        // the pair's 256 operand rows (128 antennas)
        const int q = warp & 3;
        const int o = TL - 1 - (32 * q + lane);
        uint32_t acc = 0, acc_phase = 0;
        long long j0;
        int col0, valid;
        pnce::lag_tile(prm.lags, TL, jt_own, j0, col0, valid);
        for (long long u = unit0; u < total_units; u += nunits) {
            const long long ant0 = (u / ngroups) * (BR / 2);
            int got = 1;
            if (lane == 0) got = wait_bar_sleepy(&ctl->tfull[acc], acc_phase, wctl, prm);
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) break;
            fence_after();
            const uint32_t tacc = tmem + acc * ACC_COLS + ((uint32_t)(32 * q) << 16);
            const long long spacing = u + nunits < total_units ? prm.epi_spacing : 0;
            const long long c0 = clock64();
            float2* hcol = H + col0 + o;
            for (int c = 0; c < BR / 32; ++c) {
                if (c > 0 && spacing > 0) {
                    // bounded: the target lies at most 8 * spacing cycles after c0
                    while (clock64() - c0 < c * spacing) __nanosleep(128);
                }
                uint32_t v[32];
                tmem_ld32x32b_x32(tacc + 32u * c, v);
                tmem_wait_ld();
                if (c == BR / 32 - 1) {
                    fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        if (rank == 0) mbar_arrive(&ctl->tempty[acc]);
                        else mbar_arrive_remote(&ctl->tempty[acc], 0);
                    }
                }
                if (o < valid) {
#pragma unroll
                    for (int g = 0; g < 2; ++g) {
#pragma unroll
                        for (int a = 0; a < 8; ++a) {
                            const long long ant = ant0 + 16 * c + 8 * g + a;
                            if (ant < prm.A) {
                                const float rs = __ldg(row_scale + ant);
                                hcol[ant * prm.lags.ldH] =
                                    make_float2(__uint_as_float(v[16 * g + a]) * rs,
                                                __uint_as_float(v[16 * g + 8 + a]) * rs);
                            }
                        }
                    }
                }
            }
            acc ^= 1u;
            if (acc == 0) acc_phase ^= 1u;
        }
    }

    fence_before();
    __syncthreads();
    cluster_sync_all();      // the peer no longer reads this CTA's shared memory or barriers
    if (warp == 2) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

// ------------------------------------------------------------------------- host

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Bound on every device-side wait (PNCE_WAIT_LIMIT_MS, default 2000 ms), read per launch.
unsigned long long wait_limit_ns() {
    const char* e = getenv("PNCE_WAIT_LIMIT_MS");
    long long ms = e ? atoll(e) : 2000;
    if (ms < 1) ms = 1;
    return (unsigned long long)ms * 1000000ull;
}

template <typename Kern>
pnce_status launch_kernel(Kern kern, long long grid, size_t smem, cudaStream_t s, bool pdl,
                          const CUtensorMap& map, const uint32_t* ext, const float* factors,
                          float2* H, const TcParams& prm, int cluster = 1) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return PNCE_ECUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    int na = 0;
    if (cluster > 1) {
        at[na].id = cudaLaunchAttributeClusterDimension;
        at[na].val.clusterDim.x = (unsigned)cluster;
        at[na].val.clusterDim.y = 1;
        at[na].val.clusterDim.z = 1;
        ++na;
    }
    if (pdl) {
        at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    cfg.attrs = at;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, kern, map, ext, factors, H, prm) == cudaSuccess ? PNCE_OK
                                                                                  : PNCE_ECUDA;
}

// The lag-major kernel for tiles of <= 128 lags; PNCE_EUNSUPPORTED when the shape does not
// suit it (the caller then takes the lag-column kernel).
template <int DT>
pnce_status launch_lagmajor(const pnce_handle* h, const pnce_pilot* pilot, long long A, int N,
                            const pnce::LagMap& lags, const void* operand, const float* factors,
                            float2* H, cudaStream_t s, bool pdl) {
    using F = TcFmt<DT>;
    auto enc = encode_fn();
    if (!enc) return PNCE_ECUDA;
    const long long njt = pnce::lag_tiles(lags, 128);
    if (njt < 1 || njt > h->num_sms) return PNCE_EUNSUPPORTED;
    TcParams prm{};
    prm.N = N;
    prm.lags = lags;
    prm.A = A;
    prm.BN = 128;
    prm.num_jt = (int)njt;
    prm.num_tiles = (pnce::operand_rows(A) + BR - 1) / BR * njt;
    prm.num_kb = (N + F::BK - 1) / F::BK;
    prm.wait_limit_ns = wait_limit_ns();
    prm.err = h->status_dev;
    prm.ext_words = pilot->ext_words;
    prm.drop_first_arrive = 0;
    // CTA pairs with the 2-SM MMA, each CTA loading half of the rows, when the lag tiles
    // pair up; single CTAs otherwise, or with PNCE_TC_LAGMAJOR_CL=1 (to compare the two)
    const char* cl_env = getenv("PNCE_TC_LAGMAJOR_CL");
    const bool pairable = njt % 2 == 0 && njt / 2 <= h->num_sms / 2;
    const int cl = pairable && !(cl_env && cl_env[0] == '1') ? 2 : 1;
    const bool mma2 = cl == 2;
    // every CTA keeps one lag block: the number of work units (CTAs, or pairs) in flight is
    // a multiple of the lag groups, and at most the number of units of work
    const long long groups = njt / cl;
    long long units = (h->num_sms / cl) / groups * groups;
    if (units > prm.num_tiles / cl) units = prm.num_tiles / cl;
    const long long grid = units * cl;
    const long long avail = (long long)h->max_smem_optin - (long long)smem_fixed();
    // The resident pilot list must cover every K block the MMAs read: with kps K blocks per
    // stage that is the K blocks rounded up to a multiple of kps (a last stage past N reads
    // zero rows, but its pilot core matrices must still lie inside the list).
    auto list_cm = [&](int kps_) {
        const long long kb = ((long long)prm.num_kb + kps_ - 1) / kps_ * kps_;
        return (128 / 8 - 1) * F::QS + (kb * (F::BK / F::EPR) - 1) * F::TS + 1;
    };
    auto region = [](long long cm_) { return (cm_ * 128 + 1023) / 1024 * 1024; };
    // stage bytes per CTA: the whole 256-row box, or (2-SM pairs) this CTA's 128 rows of
    // two K blocks when three such stages fit, else of one K block
    int kps = 1;
    long long stage_bytes = Y_BOX;
    if (mma2) {
        kps = (avail - region(list_cm(2))) / (2 * A_BOX) >= 3 ? 2 : 1;
        stage_bytes = kps * A_BOX;
    }
    const long long cm = list_cm(kps);
    const long long bregion = region(cm);
    long long st = (avail - bregion) / stage_bytes;
    if (st < (kps == 2 ? 3 : (mma2 ? 4 : 3))) return PNCE_EUNSUPPORTED;
    if (st > STAGES) st = STAGES;
    if ((prm.num_tiles + grid - 1) / grid <= 1 && st > 4) st = 4;
    prm.kps = kps;
    prm.a_stage = (int)stage_bytes;
    prm.num_st = (prm.num_kb + kps - 1) / kps;
    prm.stages = (int)st;
    prm.b_region = (int)bregion;
    prm.res_rows = (int)(cm * 8);
    // a tile's products: num_kb * 4 MMAs of 128 clocks (M = 128, N = 256); the epilogue's
    // eight 32-column chunks are spread over EPI_SPREAD of that
    prm.epi_spacing = (long long)(EPI_SPREAD * (double)(prm.num_kb * 4LL * 128)) / 8;

    CUtensorMap map;
    CUtensorMapDataType ty = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    if (DT == PNCE_BF16) ty = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (DT == PNCE_FP8E4M3) ty = CU_TENSOR_MAP_DATA_TYPE_UINT8;
    if (DT == PNCE_TF32) ty = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)pnce::operand_rows(A)};
    const cuuint64_t strides[1] = {(cuuint64_t)pnce::row_pitch(N) * pnce::elem_bytes(DT)};
    // a pair's CTAs load half of the 256 rows each
    const cuuint32_t box[2] = {(cuuint32_t)F::BK, (cuuint32_t)(BR / cl)};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&map, ty, 2, const_cast<void*>(operand), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return PNCE_ECUDA;
    const size_t smem = smem_fixed() + (size_t)prm.stages * prm.a_stage + prm.b_region;
    if ((long long)smem > h->max_smem_optin) return PNCE_EUNSUPPORTED;
    if (mma2)
        return kps == 2 ? launch_kernel(tc_lagmajor_pair_kernel<DT, 2>, grid, smem, s, pdl, map,
                                        pilot->ext_bits_dev, factors, H, prm, 2)
                        : launch_kernel(tc_lagmajor_pair_kernel<DT, 1>, grid, smem, s, pdl, map,
                                        pilot->ext_bits_dev, factors, H, prm, 2);
    return launch_kernel(tc_lagmajor_kernel<DT>, grid, smem, s, pdl, map, pilot->ext_bits_dev,
                         factors, H, prm);
}

template <int DT>
pnce_status launch_dt(const pnce_handle* h, const pnce_pilot* pilot, long long A, int N,
                      const pnce::LagMap& lags, const void* operand, const float* factors,
                      float2* H, cudaStream_t s, bool pdl) {
    using F = TcFmt<DT>;
    auto enc = encode_fn();
    if (!enc) return PNCE_ECUDA;

    CUtensorMap map;
    CUtensorMapDataType ty = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    if (DT == PNCE_BF16) ty = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (DT == PNCE_FP8E4M3) ty = CU_TENSOR_MAP_DATA_TYPE_UINT8;
    if (DT == PNCE_TF32) ty = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)pnce::operand_rows(A)};
    const cuuint64_t strides[1] = {(cuuint64_t)pnce::row_pitch(N) * pnce::elem_bytes(DT)};
    const cuuint32_t box[2] = {(cuuint32_t)F::BK, (cuuint32_t)BM};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&map, ty, 2, const_cast<void*>(operand), dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return PNCE_ECUDA;

    TcParams prm;
    prm.N = N;
    prm.lags = lags;
    prm.A = A;
    // lag tile width: as few tiles of <= 256 lags as cover a run, split evenly (a run is
    // all K*L lags when they are contiguous, one transmitter's L lags otherwise)
    const int run = lags.mode == 0 ? lags.ldH : lags.L;
    // A launch of few tiles (a serving batch) leaves most SMs idle, and a CTA's epilogue
    // drains its 128 x 256 accumulator at the rate one SM's stores reach (~4 us per tile):
    // there, tiles of <= 128 lags give twice the CTAs and half the drain each, for MMAs of
    // N = 128 (which the shared-memory data path makes ~1.5x dearer per flop).
    // The width halves while the tiles still fill at most half the SMs, down to
    // PNCE_TC_SMALL_GRID_BN (default 128; 0 keeps 256, to compare).
    int max_bn = MAX_BN;
    if (lags.mode == 0) {
        const long long rb = (pnce::operand_rows(A) + BM - 1) / BM;
        const char* sg = getenv("PNCE_TC_SMALL_GRID_BN");
        const int floor_bn = sg ? atoi(sg) : 128;
        while (floor_bn > 0 && max_bn / 2 >= floor_bn &&
               2 * rb * ((run + max_bn - 1) / max_bn) <= h->num_sms)
            max_bn /= 2;
    }
    const int tiles_per_run = (run + max_bn - 1) / max_bn;
    const int per = (run + tiles_per_run - 1) / tiles_per_run;
    prm.BN = (per + 31) / 32 * 32;
    // Lag tiles of at most 128 lags each (a transmitter's lags under the spread shift rule)
    // go to the lag-major kernel, whose MMAs stay N = 256 wide; PNCE_TC_LAGMAJOR=0 keeps
    // them on this kernel (to compare the two).
    const char* lm_env = getenv("PNCE_TC_LAGMAJOR");
    if (lags.mode == 1 && prm.BN <= 128 && !(lm_env && lm_env[0] == '0')) {
        const pnce_status st = launch_lagmajor<DT>(h, pilot, A, N, lags, operand, factors, H, s,
                                                   pdl);
        if (st != PNCE_EUNSUPPORTED) return st;
    }
    const long long njt = pnce::lag_tiles(lags, prm.BN);
    if (njt > (1 << 30)) return PNCE_EUNSUPPORTED;
    prm.num_jt = (int)njt;
    const long long num_rb = (pnce::operand_rows(A) + BM - 1) / BM;
    prm.num_tiles = num_rb * prm.num_jt;
    prm.num_kb = (N + F::BK - 1) / F::BK;
    prm.wait_limit_ns = wait_limit_ns();
    prm.err = h->status_dev;
    prm.ext_words = pilot->ext_words;

    long long grid = h->num_sms;
    if (grid >= prm.num_jt) grid = grid / prm.num_jt * prm.num_jt;
    if (grid > prm.num_tiles) grid = prm.num_tiles;
    if (grid < 1) return PNCE_OK;

    // Pipeline shape.  Resident pilot operand when every CTA keeps one lag block and the
    // list for all K blocks fits beside the stages: two K blocks per stage when that still
    // leaves 3 stages (32 KB each), else one K block per stage with at least 4 (16 KB).
    // Otherwise the per-stage pilot generator, two K blocks per stage.
    const long long avail = (long long)h->max_smem_optin - (long long)smem_fixed();
    auto res_cm_for = [&](int bn, int kps) {   // core matrices of the resident list
        const long long nst = (prm.num_kb + kps - 1) / kps;
        return (long long)(bn / 8 - 1) * F::QS + (nst * kps * (F::BK / F::EPR) - 1) * F::TS + 1;
    };
    auto kbytes = [](long long cm) { return (cm * 128 + 1023) / 1024 * 1024; };
    // PNCE_TC_STAGED_PILOT=1 forces the per-stage pilot path (used to test both paths);
    // PNCE_TC_TEST_DROP_ARRIVE=1 (staged path only) withholds one arrive so that the test of
    // the bounded waits sees PNCE_ETIMEOUT latched and the context still usable
    const char* force = getenv("PNCE_TC_STAGED_PILOT");
    const char* drop = getenv("PNCE_TC_TEST_DROP_ARRIVE");
    prm.drop_first_arrive = (drop && drop[0] == '1') ? 1 : 0;
    const bool may_res = !(force && force[0] == '1') && (grid % prm.num_jt == 0);
    bool res = false;
    for (int kps = MAX_KPS; kps >= 1 && may_res && !res; --kps) {
        const long long cm = res_cm_for(prm.BN, kps);
        const long long st = (avail - kbytes(cm)) / (kps * A_BOX);
        if (st >= (kps == 2 ? 3 : 4)) {
            res = true;
            prm.kps = kps;
            prm.stages = (int)std::min<long long>(STAGES, st);
            prm.b_region = (int)kbytes(cm);
            prm.res_rows = (int)(cm * 8);
        }
    }
    if (!res) {
        prm.kps = MAX_KPS;
        prm.stages = (int)std::min<long long>(
            STAGES, avail / (MAX_KPS * A_BOX + b_stage_bytes<DT>()));
        prm.b_region = prm.stages * b_stage_bytes<DT>();
        prm.res_rows = 0;
    }
    // A CTA with a single tile needs no deep pipeline; four stages keep its shared memory
    // small enough to become resident beside the blocks of the kernel before it, so that
    // a programmatic dependent launch overlaps its set-up with that kernel.
    if ((prm.num_tiles + grid - 1) / grid <= 1 && prm.stages > 4) {
        prm.stages = 4;
        if (!res) prm.b_region = prm.stages * b_stage_bytes<DT>();
    }
    prm.a_stage = prm.kps * A_BOX;
    prm.num_st = (prm.num_kb + prm.kps - 1) / prm.kps;
    // a tile's products take ~num_kb * 4 MMAs of BN/2 cycles (M = 128, any operand type);
    // the epilogue's chunks are spread over EPI_SPREAD of that
    {
        const long long nch = (prm.BN + 63) / 64;
        const long long tile_cycles = (long long)prm.num_st * prm.kps * 2LL * prm.BN;
        prm.epi_spacing = nch > 1 ? (long long)(EPI_SPREAD * (double)tile_cycles) / nch : 0;
    }
    // 2-SM variant (opt-in while it is being evaluated): CTA pairs, each CTA with half of a
    // BN-lag tile's pilot list; pairs stay on one lag block, so their count is a multiple
    // of num_jt
    const char* pairs_env = getenv("PNCE_TC_PAIRS");
    if (pairs_env && pairs_env[0] == '1' && !(force && force[0] == '1')) {
        const long long num_prb = (pnce::operand_rows(A) + 2 * BM - 1) / (2 * BM);
        const long long ptiles = num_prb * prm.num_jt;
        long long pairs = h->num_sms / 2;
        if (pairs >= prm.num_jt) pairs = pairs / prm.num_jt * prm.num_jt;
        if (pairs > ptiles) pairs = ptiles;
        TcParams pp = prm;
        bool ok2 = false;
        for (int kps = MAX_KPS; kps >= 1 && !ok2; --kps) {
            const long long cm = res_cm_for(prm.BN / 2, kps);
            const long long st = (avail - kbytes(cm)) / (kps * A_BOX);
            if (st >= (kps == 2 ? 3 : 4)) {
                ok2 = true;
                pp.kps = kps;
                pp.a_stage = kps * A_BOX;
                pp.num_st = (prm.num_kb + kps - 1) / kps;
                pp.stages = (int)std::min<long long>(STAGES, st);
                pp.b_region = (int)kbytes(cm);
                pp.res_rows = (int)(cm * 8);
            }
        }
        if (pairs >= 1 && pairs % prm.num_jt == 0 && prm.BN % 32 == 0 && ok2) {
            pp.num_tiles = ptiles;
            const size_t smem2 = smem_fixed() + (size_t)pp.stages * pp.a_stage + pp.b_region;
            auto pk = pp.kps == 2 ? tc_pair_kernel<DT, 2> : tc_pair_kernel<DT, 1>;
            if (cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem2) != cudaSuccess)
                return PNCE_ECUDA;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)(2 * pairs), 1, 1);
            cfg.blockDim = dim3(THREADS, 1, 1);
            cfg.dynamicSmemBytes = smem2;
            cfg.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            const cudaError_t le =
                cudaLaunchKernelEx(&cfg, pk, map, pilot->ext_bits_dev, factors, H, pp);
            return le == cudaSuccess ? PNCE_OK : PNCE_ECUDA;
        }
    }

    const size_t smem = smem_fixed() + (size_t)prm.stages * prm.a_stage + prm.b_region;
    if ((long long)smem > h->max_smem_optin) return PNCE_EUNSUPPORTED;
    // the staged path always takes two K blocks per stage
    auto kern = !res ? tc_corr_kernel<DT, false, 2>
                     : (prm.kps == 2 ? tc_corr_kernel<DT, true, 2> : tc_corr_kernel<DT, true, 1>);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return PNCE_ECUDA;
    if (pdl) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid, 1, 1);
        cfg.blockDim = dim3(THREADS, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const cudaError_t le =
            cudaLaunchKernelEx(&cfg, kern, map, pilot->ext_bits_dev, factors, H, prm);
        return le == cudaSuccess ? PNCE_OK : PNCE_ECUDA;
    }
    kern<<<(unsigned)grid, THREADS, smem, s>>>(map, pilot->ext_bits_dev, factors, H, prm);
    return cudaGetLastError() == cudaSuccess ? PNCE_OK : PNCE_ECUDA;
}

}  // namespace

namespace pnce {

pnce_status launch_tc_ex(const pnce_handle* h, const pnce_pilot* pilot, long long A, int N,
                         const LagMap& lm, int dtype, const void* operand, const float* factors,
                         float2* H, cudaStream_t s, bool pdl) {
    if (!(h->cc_major == 10 && h->cc_minor == 3)) return PNCE_EUNSUPPORTED;
    switch (dtype) {
        case PNCE_FP16:
            return launch_dt<PNCE_FP16>(h, pilot, A, N, lm, operand, factors, H, s, pdl);
        case PNCE_BF16:
            return launch_dt<PNCE_BF16>(h, pilot, A, N, lm, operand, factors, H, s, pdl);
        case PNCE_FP8E4M3:
            return launch_dt<PNCE_FP8E4M3>(h, pilot, A, N, lm, operand, factors, H, s, pdl);
        case PNCE_TF32:
            return launch_dt<PNCE_TF32>(h, pilot, A, N, lm, operand, factors, H, s, pdl);
        default: return PNCE_EINVAL;
    }
}

pnce_status launch_tc(const pnce_handle* h, const pnce_pilot* pilot, long long A, int N, int KL,
                      int dtype, const void* operand, const float* factors, float2* H,
                      cudaStream_t s, bool pdl) {
    return launch_tc_ex(h, pilot, A, N, lagmap_contiguous(KL), dtype, operand, factors, H, s,
                        pdl);
}

}  // namespace pnce
