/*
 * pnce.h -- C ABI of libpnce, PN-sequence correlation channel estimation on GB300.
 *
 * What is computed (Sec. II, Eq. 2, 3 and 10 of "Channel Estimation for Massive MIMO
 * systems using Tensor Cores in GPU"): K transmitters send cyclic shifts k*L of one
 * length-N m-sequence pilot p; after cyclic-prefix removal every receive antenna
 * correlates its N complex samples with every cyclic shift of p,
 *
 *     H[f][m][k][l] = (1/N) * sum_{n<N} Y[f][m][n] * p[(n - l - k*L) mod N],
 *
 * which is the circulant (Eq. 2) correlator (1/N) S^T Y of Eq. 3 / Eq. 10 restricted
 * to the lags j = k*L + l < K*L.  p[n] = +1 for pilot bit 0 and -1 for bit 1.
 *
 * Conventions shared by every entry point
 *  - Complex data are interleaved float32 pairs (re, im) ("complex64").
 *    Y is [F][M][N] and H is [F][M][K][L] (equivalently [F*M][K*L], lag j = k*L + l),
 *    both dense row-major.
 *  - Pointers named *_dev are device pointers on the device that was current when the
 *    handle was created; *_host are host pointers (page-locked memory recommended).
 *    The caller owns Y, H, gradients and workspaces; the library owns only what its
 *    own create functions return.  No estimate/backward call allocates memory.
 *  - stream is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Calls only enqueue work; results are ready when the stream reaches them.
 *  - Every function returns a pnce_status and never aborts or prints.  Arguments are
 *    validated before anything is launched; an invalid call launches nothing.
 *  - A handle may be used from several host threads: the sections that enqueue work on
 *    the handle's own streams (large-batch overlap in pnce_estimate, pnce_estimate_host)
 *    and the trace record are serialised inside the library.  Such sections of different
 *    calls then also run one after the other on the GPU.
 *    Errors raised on the device after launch (a bounded wait that ran out inside a
 *    kernel) are latched in the handle and reported by pnce_get_status().
 *  - Shape rules: F, M >= 1; N >= 2; K, L >= 1 and K*L <= N (Eq. 7 with C = L: the
 *    cyclic shifts must not alias).  Device pointers must be 16-byte aligned.
 */
#ifndef PNCE_H
#define PNCE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PNCE_OK = 0,
    PNCE_EINVAL = 1,        /* bad argument: shape, null or misaligned pointer, small workspace */
    PNCE_EUNSUPPORTED = 2,  /* valid request the library or device cannot serve */
    PNCE_ENOMEM = 3,        /* a create function could not allocate */
    PNCE_ECUDA = 4,         /* a CUDA runtime call failed */
    PNCE_ETIMEOUT = 5,      /* a device-side bounded wait ran out (latched, see pnce_get_status) */
    PNCE_ESTATE = 6         /* wrong device current, or handle/pilot mismatch */
} pnce_status;

/* Arithmetic of the correlation.  FP32_SIMT: exact FP32 on the CUDA cores.  The others
 * quantise Y (per antenna, power-of-two scale) and run on the tensor cores with FP32
 * accumulation; +-1 pilots are exact in every one of these formats (Sec. III-B uses FP16
 * operands).  AUTO lets the library choose from the shape, see pnce_auto_dtype. */
typedef enum {
    PNCE_FP32_SIMT = 0,
    PNCE_TF32 = 1,
    PNCE_FP16 = 2,
    PNCE_BF16 = 3,
    PNCE_FP8E4M3 = 4,
    PNCE_AUTO = 5
} pnce_dtype;

/*
 * The arithmetic PNCE_AUTO stands for at this shape: PNCE_FP32_SIMT when K*L <= 16, else
 * PNCE_FP16 (the paper's tensor-core operand format, Sec. III-B).  With few lags the
 * correlation is bound by reading Y once (8 bytes per sample), which the FP32 kernel does
 * at about the rate of the quantiser pass that every tensor-core estimate starts with, so
 * exact FP32 costs nothing there; with more lags the tensor cores win by far.  Host only;
 * returns -1 for an invalid shape.  pnce_workspace_size, pnce_estimate, pnce_estimate_ex,
 * pnce_host_workspace_size, pnce_estimate_host, pnce_grouped_workspace_size and
 * pnce_estimate_grouped (with K*L = kl_max) accept PNCE_AUTO and resolve it by this rule;
 * pnce_quantize, pnce_correlate_quantized and pnce_estimate_static, which name one
 * tensor-core step or format, do not.
 */
int pnce_auto_dtype(int N, int K, int L);

typedef struct pnce_handle pnce_handle;   /* per-device context: latched device status */
typedef struct pnce_pilot pnce_pilot;     /* device-resident pilot bit table of one sequence */

/* Library version, major*10000 + minor*100 + patch. */
int pnce_version(void);

/* Human-readable name of a status code (static string, never NULL). */
const char* pnce_status_string(pnce_status s);

/* Create a handle bound to the current device.  Allocates one small device status word. */
pnce_status pnce_create(pnce_handle** out);
pnce_status pnce_destroy(pnce_handle* h);

/* Read (and clear) the status latched by kernels of this handle.  Synchronises stream. */
pnce_status pnce_get_status(pnce_handle* h, void* stream);

/*
 * Pilot table (Sec. II-A: the m-sequence pilot, Eq. 1).  bits_host: ceil(N/32) uint32
 * words, bit n of the sequence in word n/32 at bit n%32 (LSB first).  The library
 * uploads a wrapped copy (bit t = bit (t mod N)) to device memory once; the call is
 * synchronous.  N in [2, 2^24).
 */
pnce_status pnce_pilot_create(pnce_handle* h, const uint32_t* bits_host, int N, pnce_pilot** out);
pnce_status pnce_pilot_destroy(pnce_pilot* p);

/*
 * Workspace bytes pnce_estimate needs for this shape and dtype (0 for FP32_SIMT).  The
 * tensor-core dtypes keep the quantised operand there: 16*ceil(F*M/8) rows of
 * ceil(N/64)*64 elements (row order as in pnce_quantize), plus per-antenna scales.
 * Returns 0 for invalid shapes.
 */
size_t pnce_workspace_size(int F, int M, int N, int K, int L, int dtype);

/*
 * Channel estimate, Eq. 3 / Eq. 10 (definition at the top of this file).
 * Y_dev: complex64 [F][M][N]; H_dev: complex64 [F][M][K][L] (fully overwritten).
 * dtype: a pnce_dtype.  For the tensor-core dtypes Y is first quantised per antenna
 * (pnce_quantize) into workspace_dev, then correlated on the tensor cores; the FP32 SIMT
 * path ignores the workspace (may be NULL).  With the environment variable
 * PNCE_OVERLAP_CHUNKS=n (2..8), a large tensor-core batch is cut into n frame chunks whose
 * quantisation overlaps the previous chunk's correlation on the handle's own streams
 * (the call still behaves as if enqueued on `stream`); by default the two run in order.
 */
pnce_status pnce_estimate(pnce_handle* h, const pnce_pilot* pilot, const void* Y_dev,
                          int F, int M, int N, int K, int L, int dtype,
                          void* workspace_dev, size_t workspace_bytes, void* H_dev,
                          void* stream);

/* Cyclic-shift rule of the multiplexed transmitters (Sec. II-B). */
typedef enum {
    PNCE_SHIFT_KL = 0,      /* transmitter k at cyclic shift k*L: lags 0 .. K*L-1 contiguous */
    PNCE_SHIFT_SPREAD = 1   /* transmitter k at cyclic shift k*floor(N/K) (Eq. 8, spread evenly) */
} pnce_shift_rule;

/* Frame layout options of pnce_estimate_ex. */
typedef struct {
    int cp_len;             /* cyclic-prefix samples at the head of every received row */
    int shift_rule;         /* a pnce_shift_rule */
} pnce_frame_opts;

/*
 * pnce_estimate with the pilot-slot layout spelled out (Sec. II-A/B):
 *  - Y_dev rows hold cp_len + N samples, the cyclic prefix first; the prefix is skipped
 *    (Sec. II-A: the CP is removed and only the PN part is correlated);
 *  - transmitter k uses the cyclic shift s_k given by opts->shift_rule, and
 *    H[f][m][k][l] = (1/N) sum_n Y[f][m][cp_len + n] p[(n - s_k - l) mod N].
 * Requires L <= floor(N/K) for PNCE_SHIFT_SPREAD (shifted copies must not alias, Eq. 7),
 * K*L <= N for PNCE_SHIFT_KL.  opts == NULL is pnce_estimate.  Workspace as
 * pnce_workspace_size(F, M, N, K, L, dtype).
 */
pnce_status pnce_estimate_ex(pnce_handle* h, const pnce_pilot* pilot, const void* Y_dev,
                             int F, int M, int N, int K, int L, int dtype,
                             const pnce_frame_opts* opts, void* workspace_dev,
                             size_t workspace_bytes, void* H_dev, void* stream);

/*
 * Reduced-precision operand (Sec. III-B: conversion of the received block to the
 * tensor-core input format).  For antenna a = f*M + m: A_a = max_n max(|Re y|, |Im y|)
 * (exact in FP32), E_a = sum_n |y|^2 (FP64); scale 2^s_a with s_a = t - e where
 * A_a = mant * 2^e, mant in [0.5, 1), t = 15 (fp16) or 8 (e4m3), s_a = 0 for bf16,
 * tf32 and A_a = 0; s_a clamped to [-100, 100].  Writes, into workspace_dev, the rows
 * of round(y * 2^s_a) in dtype (round to nearest even; e4m3 saturates at 448; tf32
 * rounds ties away): antennas in groups of 8, 16 rows per group, the real parts of the
 * group's antennas first, so row 16*(a/8) + (a%8) holds the real part of antenna a and
 * row 16*(a/8) + 8 + (a%8) its imaginary part; the rows of antennas >= F*M in the last
 * group are zero.  Rows hold ceil(N/64)*64 elements (the tail past N is not written).
 * Also writes the per-antenna output factor 2^-s_a / N (float32) after the rows and, if
 * power_dev != NULL, E_a / N (float64 [F*M]).
 * exps_dev (int32 [F*M], may be NULL) receives s_a.  dtype must not be FP32_SIMT.
 */
pnce_status pnce_quantize(pnce_handle* h, const void* Y_dev, int F, int M, int N, int dtype,
                          void* workspace_dev, size_t workspace_bytes, int32_t* exps_dev,
                          double* power_dev, void* stream);

/*
 * Tensor-core correlation of an operand already quantised into workspace_dev by
 * pnce_quantize (same F, M, N, dtype): the contraction and epilogue of pnce_estimate
 * alone.  Lets callers time or overlap the quantisation separately.
 */
pnce_status pnce_correlate_quantized(pnce_handle* h, const pnce_pilot* pilot,
                                     int F, int M, int N, int K, int L, int dtype,
                                     const void* workspace_dev, size_t workspace_bytes,
                                     void* H_dev, void* stream);

/* How pnce_estimate_real_pilot / pnce_backward read their float pilot argument. */
typedef enum {
    PNCE_PILOT_REAL = 0,    /* the argument is the pilot p itself */
    PNCE_PILOT_TANH = 1     /* the argument is theta and the pilot is p = tanh(theta) */
} pnce_pilot_map;

/*
 * Estimate with a real-valued pilot (float32 [N], device) in place of the +-1 sequence:
 * H = (1/N) sum_n Y[n] p[(n - j) mod N], FP32 on the CUDA cores.  With PNCE_PILOT_TANH
 * the argument is theta and p = tanh(theta) is formed inside the kernel: the forward of
 * the relaxed pilot used for end-to-end pilot optimisation.
 */
pnce_status pnce_estimate_real_pilot(pnce_handle* h, const float* pilot_dev, int pilot_map,
                                     const void* Y_dev, int F, int M, int N, int K, int L,
                                     void* H_dev, void* stream);

/*
 * Adjoint of pnce_estimate_real_pilot for a real loss.  G_dev = dLoss/dRe(H) +
 * i dLoss/dIm(H), complex64 [F][M][K][L].  Outputs (either may be NULL to skip):
 *   dY_dev[f][m][n] = (1/N) sum_{j<KL} G[f][m][j] p[(n - j) mod N]      complex64
 *   dpilot_dev[q]   = (1/N) sum_{f,m,j} Re(conj(G[f][m][j]) Y[f][m][(q + j) mod N])
 * and with PNCE_PILOT_TANH, dpilot_dev is the gradient with respect to theta,
 * dp[q] * (1 - tanh(theta[q])^2).  The pilot sum is reduced deterministically in two
 * stages through workspace_dev (pnce_backward_workspace_size bytes), so repeated calls
 * give identical bits.
 */
size_t pnce_backward_workspace_size(int F, int M, int N, int K, int L);
pnce_status pnce_backward(pnce_handle* h, const float* pilot_dev, int pilot_map,
                          const void* Y_dev, const void* G_dev, int F, int M, int N, int K,
                          int L, void* dY_dev, float* dpilot_dev, void* workspace_dev,
                          size_t workspace_bytes, void* stream);

/*
 * End-to-end estimate from host memory (the paper's frame latency includes the host to
 * device transfer, Sec. IV-C): copies Y_host (complex64 [F][M][N]) to the device,
 * estimates as pnce_estimate, and copies H back to H_host (complex64 [F][M][K][L]).
 * Frames go through in chunks, triple buffered, on three streams owned by the handle
 * (copy-in, kernels, copy-out), so both copy directions overlap the kernels.  The
 * pipeline starts after the work already queued on `stream`, and `stream` waits for its
 * end: to the caller the call behaves as if it were enqueued on `stream`.  All device
 * buffers live in workspace_dev (pnce_host_workspace_size bytes, caller-owned).  Host
 * buffers should be page-locked for the copies to be asynchronous.  Y comes in by
 * cudaMemcpyAsync; H goes out by a copy kernel storing into H_host when H_host is
 * page-locked memory known to CUDA (it shares the host link with the inbound copy better
 * than a second DMA does), by cudaMemcpyAsync otherwise.  Calls on the same handle are
 * serialised on the handle's pipeline streams.
 */
size_t pnce_host_workspace_size(int F, int M, int N, int K, int L, int dtype);
pnce_status pnce_estimate_host(pnce_handle* h, const pnce_pilot* pilot, const void* Y_host,
                               int F, int M, int N, int K, int L, int dtype,
                               void* workspace_dev, size_t workspace_bytes, void* H_host,
                               void* stream);

/*
 * Tracing.  While enabled, the estimate entry points (pnce_estimate, pnce_estimate_ex,
 * pnce_quantize, pnce_correlate_quantized, pnce_estimate_grouped, pnce_estimate_fmt,
 * pnce_estimate_real_pilot, pnce_backward, pnce_estimate_static) record a CUDA event before and after every
 * quantiser / correlation / adjoint launch, on the stream it runs on (internal streams
 * included), up to 8192 launches.  Each such launch is also an NVTX range named
 * "pnce.<kind>" (always on; a no-op unless a profiler is attached).
 * pnce_trace_enable creates the events on first use (allocates host and event resources,
 * not device memory) and clears the record; pnce_trace_read waits for the recorded kernels,
 * returns up to max_entries (kind, milliseconds) pairs -- kind 0 quantiser, 1 tensor-core
 * correlation, 2 FP32 SIMT correlation, 3 fast m-sequence transform, 4 adjoint (dY and
 * dp together) -- in launch order, and
 * clears the record.  Do not enable it while capturing a CUDA graph.
 */
pnce_status pnce_trace_enable(pnce_handle* h, int on);
pnce_status pnce_trace_read(pnce_handle* h, int* kinds, float* ms, int max_entries, int* count);

/*
 * Row movement for batched serving (the frames of many requests estimated as one batch;
 * no counterpart in the paper, which processes one frame at a time).  Pointer tables are
 * arrays of 64-bit addresses that the GPU can dereference: device memory, or page-locked
 * host memory, which the kernels then read or write directly over the host link.  The
 * tables themselves may also live in page-locked host memory.  A NULL row address skips
 * that row.  Both calls only enqueue one kernel on `stream`.
 *
 * pnce_gather_rows: dst_dev[r][0..nelem) = src_rows[r][0..nelem) for r < rows, with
 *   8-byte elements (one complex64 sample) and a row pitch of dst_pitch elements.
 * pnce_scatter_rows: dst_rows[r][0..counts[r]) = src_dev[r][0..counts[r]) for r < rows,
 *   source row pitch src_pitch elements (counts are clamped to src_pitch).
 */
/*
 * Grouped estimate for continuous-batching serving (the paper processes one frame at a
 * time, so this has no counterpart there): the antennas of nreq requests that share one
 * pilot (same N) are estimated as one batch of `rows` rows with kl_max lags.  descs is a
 * table of nreq <= rows descriptors in device memory or page-locked host memory, copied
 * to the workspace by the call's first operation (a copy node when captured, so the table
 * can be rewritten between replays of a captured graph).  Request b moves its
 * received rows Y (complex64 [M][N]) into batch rows row_offset .. row_offset+M-1 (the
 * requests' row ranges must not overlap), and
 * gets back H (complex64 [M][K*L]) = the first K*L lags of those rows, with lag
 * j = k*L + l as in pnce_estimate.  Y and H may be device memory or page-locked host
 * memory (read and written by the GPU over the host link), 8-byte aligned.  M = 0 marks
 * an empty slot.  A descriptor with row_offset + M > rows, K*L > kl_max, or a NULL or
 * misaligned buffer is skipped and latches PNCE_EINVAL (pnce_get_status), as does a row
 * claimed by two descriptors (which of the two then gets it is not defined).  Batch rows
 * no request covers are estimated from zeros or whatever the workspace holds, and
 * discarded.  workspace_dev: 256-byte aligned, pnce_grouped_workspace_size(rows, N,
 * kl_max, dtype) bytes (0 for invalid shapes).  Enqueues on `stream`, each kernel a
 * programmatic dependent of the one before it: a table / row-map kernel, then for the
 * tensor-core dtypes the quantiser (reading each row from its request's Y), the
 * correlation and a scatter into the requests' H; for FP32 with kl_max > 32 the SIMT
 * correlation reading the rows from the requests' Y (after a row gather into the
 * workspace when kl_max > 256) and writing each row's lags into its request's H; for
 * FP32 with kl_max <= 32 a row gather, the correlation and a scatter.  Allocates nothing.
 */
typedef struct {
    const void* Y;          /* complex64 [M][N] */
    void* H;                /* complex64 [M][K*L] */
    int M, K, L;
    int row_offset;         /* first batch row of the request */
} pnce_req_desc;
size_t pnce_grouped_workspace_size(int rows, int N, int kl_max, int dtype);
pnce_status pnce_estimate_grouped(pnce_handle* h, const pnce_pilot* pilot,
                                  const pnce_req_desc* descs, int nreq, int rows, int kl_max,
                                  int dtype, void* workspace_dev, size_t workspace_bytes,
                                  void* stream);

/* Native serving loop (continuous batching of uneven requests, built on
 * pnce_estimate_grouped; the paper has no counterpart).  A run replays a trace open loop:
 * request i is submitted t_arrival seconds after the run starts (t_arrival non-decreasing).
 * Admission: in arrival order while the footprint of admitted, unfinished requests stays
 * within mem_cap_bytes (a request is admitted regardless when nothing is in flight; the
 * footprint of a request is M * (8 N + 2 e pitch(N) + 8 kl_class) bytes, e the operand
 * element bytes of dtype (0 for FP32, 2 for PNCE_AUTO), pitch(N) = N rounded up to 64).
 * Admitted requests wait in buckets keyed by (N, kl_class), kl_class the smallest of
 * 64, 256, 1024 that holds K*L, capped at N (above 1024: K*L rounded up to 1024, capped
 * at N).  Whenever one of the
 * `slots` streams is free the bucket whose oldest request arrived first (ties: smaller N,
 * then smaller class) is launched as one grouped batch, packing its requests in order while
 * their antennas fit max_batch_rows (always at least one).  A batch runs as one replay of a
 * CUDA graph captured per (slot, N, class, capacity), capacity the smallest of 64, 256,
 * 1024, 4096 antennas that holds it (larger: a multiple of 4096).  Completion = its event,
 * polled in launch order.  The run busy-polls on the calling thread; a server is used by
 * one thread at a time.
 *
 * pnce_server_create: dtype as pnce_estimate_grouped (PNCE_AUTO resolved per bucket);
 *   1 <= slots <= 64.  Creates the streams and events; the caller keeps h alive.
 * pnce_server_add_pilot: the pilot for one PN length N (not owned: keep it alive while
 *   the server may run batches of that N).  A request whose N has no pilot fails (status
 *   PNCE_EINVAL).  Adding another pilot for an N drops the graphs captured with the
 *   previous one (after the server's streams are idle), so that one may then be destroyed.
 * pnce_server_prepare: captures the graphs of one (N, kl_class, capacity) shape on every
 *   slot ahead of a run (a run captures missing shapes when it first needs them, inside
 *   its timed loop).  Allocates the shape's workspace and page-locked descriptor table.
 * pnce_server_run: reqs[n] in host memory; each request's Y (complex64 [M][N]) and H
 *   (complex64 [M][K*L]) as in pnce_req_desc.  out[n]: per request the admission, launch
 *   and completion times (seconds from the start of the run), the batch index and a
 *   status (PNCE_OK, or the status that failed its batch: PNCE_ECUDA for a launch or an
 *   event error, PNCE_EINVAL for a missing pilot, PNCE_ENOMEM for a shape that could not be
 *   allocated; -1 for a request the run never got to, when it gave up part-way).  Returns PNCE_EINVAL for invalid arguments (nothing run), else, after every
 *   batch completed, the status latched on the device by the run's kernels (PNCE_OK when
 *   none; otherwise some results may be wrong).
 * Online use (a session of requests submitted as they come, results collected as they
 * finish; the same rules, the arrival time of a request being its submission):
 * pnce_server_start begins a session (its clock starts at 0; PNCE_ESTATE while requests of
 *   the previous session are still open).
 * pnce_server_submit queues one request (req->t_arrival is ignored) and returns its ticket
 *   (0, 1, ... in submission order); PNCE_EINVAL for an invalid request, PNCE_ESTATE with
 *   no session.  The request's buffers must stay valid until it is reported.
 * pnce_server_poll runs one scheduling pass (completions, admissions, launches) and
 *   reports up to max_out finished requests -- tickets[k] with outs[k] as in
 *   pnce_server_run -- in *n_out; the others are reported by later polls.  Results latched
 *   on the device by the kernels are read with pnce_get_status.
 * pnce_server_open: requests of the session not yet reported.  pnce_server_run returns
 *   PNCE_ESTATE while any are open (the two share the slots).
 * pnce_sched_simulate: the same scheduling rules on a virtual clock, no GPU: the clock
 *   advances by clock_dt at every pass of the loop, a batch of r antennas completes
 *   base_s + per_row_s * r seconds after its launch, a request's footprint is
 *   M * row_bytes.  Faults made on the host: every fail_launch_every-th launch is refused
 *   and every fail_done_every-th batch that started fails at completion (0: never); their
 *   requests get PNCE_ECUDA.  Fills out[n] and *batches as pnce_server_run does.
 */
typedef struct pnce_server pnce_server;
typedef struct {
    const void* Y;          /* complex64 [M][N] */
    void* H;                /* complex64 [M][K*L] */
    int M, N, K, L;
    double t_arrival;       /* seconds from the start of the run */
} pnce_serve_req;
typedef struct {
    double t_admit, t_launch, t_done;   /* seconds from the start of the run */
    int batch;
    int status;
} pnce_serve_out;
pnce_status pnce_server_create(pnce_handle* h, int dtype, int slots, double mem_cap_bytes,
                               int max_batch_rows, pnce_server** out);
pnce_status pnce_server_destroy(pnce_server* server);
pnce_status pnce_server_add_pilot(pnce_server* server, const pnce_pilot* pilot);
pnce_status pnce_server_prepare(pnce_server* server, int N, int kl_class, int capacity);
pnce_status pnce_server_run(pnce_server* server, const pnce_serve_req* reqs, int n,
                            pnce_serve_out* out, int* batches);
pnce_status pnce_server_start(pnce_server* server);
pnce_status pnce_server_submit(pnce_server* server, const pnce_serve_req* req,
                               long long* ticket);
pnce_status pnce_server_poll(pnce_server* server, long long* tickets, pnce_serve_out* outs,
                             int max_out, int* n_out);
pnce_status pnce_server_open(pnce_server* server, int* n_open);
pnce_status pnce_sched_simulate(const pnce_serve_req* reqs, int n, int slots,
                                double mem_cap_bytes, int max_batch_rows, double row_bytes,
                                double base_s, double per_row_s, double clock_dt,
                                int fail_launch_every, int fail_done_every,
                                pnce_serve_out* out, int* batches);

pnce_status pnce_gather_rows(const uint64_t* src_rows, int rows, int nelem, void* dst_dev,
                             long long dst_pitch, void* stream);
pnce_status pnce_scatter_rows(const void* src_dev, long long src_pitch, const uint64_t* dst_rows,
                              const int* counts, int rows, void* stream);

/*
 * Allocation-free estimate (no counterpart in the paper; an interface addition).  Same
 * result as pnce_estimate for the tensor-core dtypes, but the call takes no workspace and
 * allocates nothing: the quantised operand and factors live in one device array of
 * PNCE_STATIC_SCRATCH_BYTES that is part of the library image.  It is for callers that
 * cannot call cudaMalloc: a real-time receive chain whose per-slot deadline cannot absorb
 * the allocator's unbounded latency (cudaMalloc may also synchronise the device), and
 * hosts that run the library inside a fixed, pre-reserved memory budget with no allocator
 * to hand it.
 *  - Every device that loads the library keeps the array until the process exits.
 *  - Shapes whose operand does not fit (pnce_workspace_size(...) > PNCE_STATIC_SCRATCH_BYTES,
 *    i.e. 16*ceil(A/8) rows of ceil(N/64)*64 elements of the dtype's size, 256-byte
 *    rounded, plus 4*A bytes of factors, for A = F*M antennas: about 4000 antennas at
 *    N = 4095 in fp16 or bf16, 8000 in e4m3, 2000 in tf32) return PNCE_EINVAL and launch
 *    nothing; FP32_SIMT needs no scratch and is rejected here too (use pnce_estimate), as
 *    is PNCE_AUTO.
 *  - The first call on a device looks up the array's device address; make that first call
 *    before any stream capture.
 *  - All calls share the one array and it keeps the last call's contents (nothing in it
 *    needs to start at zero).  Calls whose work overlaps on the GPU -- other streams, other
 *    threads, other handles -- race on it: the caller must serialise them.
 */
#define PNCE_STATIC_SCRATCH_BYTES (64u << 20)
pnce_status pnce_estimate_static(pnce_handle* h, const pnce_pilot* pilot, const void* Y_dev,
                                 int F, int M, int N, int K, int L, int dtype, void* H_dev,
                                 void* stream);

/*
 * Fast m-sequence transform: a yardstick beside the paper's method, not part of it (the
 * paper correlates with the dense circulant, Sec. III-B).  For an m-sequence pilot of
 * degree r (N = 2^r - 1) the same estimate, H[f][m][k][l] = (1/N) sum_n Y[f][m][n]
 * p[(n - l - kL) mod N], is a permutation of each received row into a vector of 2^r
 * entries, a Walsh-Hadamard transform and a gather of the K*L lags: O(N log N) per row
 * instead of O(N K L), in FP32 on the CUDA cores.
 *
 * pnce_fmt_tables (host only, no device use): for bits_host packed as for
 * pnce_pilot_create, fills pos[n] (n < N) with the r-bit window
 * s_n = sum_{i<r} bit[(n+i) mod N] 2^i and lagvec[j] (j < N) with the vector u_j for which
 * bit[(n - j) mod N] = parity(u_j & s_n) for every n.  Both arrays are caller-owned,
 * N entries each.  Returns PNCE_EINVAL unless N = 2^r - 1 with 2 <= r <= 14 and the bits
 * are an m-sequence (distinct nonzero windows, and the order-r linear recurrence they
 * imply holds over the whole period).
 * pnce_fmt_create builds the tables and uploads them to the handle's device (synchronous);
 * pnce_fmt_destroy frees them.
 * pnce_estimate_fmt: Y_dev complex64 [F][M][N], H_dev complex64 [F][M][K][L] (fully
 * overwritten), K*L <= N, both 16-byte aligned; enqueued on `stream`, no workspace.
 */
typedef struct pnce_fmt pnce_fmt;
pnce_status pnce_fmt_tables(const uint32_t* bits_host, int N, uint16_t* pos, uint16_t* lagvec);
pnce_status pnce_fmt_create(pnce_handle* h, const uint32_t* bits_host, int N, pnce_fmt** out);
pnce_status pnce_fmt_destroy(pnce_fmt* f);
pnce_status pnce_estimate_fmt(pnce_handle* h, const pnce_fmt* f, const void* Y_dev, int F,
                              int M, int N, int K, int L, void* H_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PNCE_H */
