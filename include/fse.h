/*
 * fse.h -- C-ABI of the GB300 (sm_103a) implementation of Frequency Selective
 * Extrapolation (FSE) block-loss concealment with the line-scan or the
 * optimized, parallelizable processing order of Seiler & Kaup, "Optimized
 * and Parallelized Processing Order for Improved Frequency Selective Signal
 * Extrapolation".
 *
 * Every entry point returns an int status (FSE_OK = 0 or an FSE_E* code)
 * and never aborts the process.  No torch types appear here: buffers are
 * plain host or device pointers, sizes are ints.
 *
 * Method summary (what the library computes for every lost block b):
 *   1. Extrapolation area L = block b plus a frame of `border` samples
 *      (Sec. 2, Fig. 1): (B + 32) x (B + 32) samples for B x B blocks and
 *      d = 16 (48 x 48 for B = 16).  With B < d the area reaches blocks
 *      beyond the 8-neighbourhood; blocks of one group still read the frame
 *      as of the group start.
 *      Sub-areas: A (originally known), R (lost, concealed earlier),
 *      B_i (lost, inside b), B_o (lost, outside b, still open), and
 *      samples outside the image.
 *   2. Weighting, Eq. (2): rho^dist on A, delta * rho^dist on R, 0 on
 *      B_i, B_o and outside; dist from the area centre ((M-1)/2, (N-1)/2).
 *   3. Model, Eq. (1): g = sum_k c_k phi_k with 2-D DFT basis functions
 *      phi_k[m,n] = exp(+j 2 pi (k_m m + k_n n) / 64) (Sec. 4).  Each of K
 *      iterations selects u = argmax_k |R_w[k]|^2 (largest decrease of the
 *      weighted residual energy; ties to the smallest k_m * 64 + k_n),
 *      adds dc = gamma * R_w[u] / W[0] to c_u (orthogonality deficiency
 *      compensation, gamma = 0.5 in Sec. 4) and updates the weighted
 *      residual spectrum R_w[k] -= dc * W[(k - u) mod 64] (transform-domain
 *      form, Sec. 4), where W is the DFT of the weights.
 *   4. The real part of the model, clamped to [0, 255], is inserted into
 *      the lost samples of b (Sec. 2); the 8-bit output is rounded half to
 *      even.  Later blocks read the clamped, unrounded value.
 *   5. Blocks are processed in line-scan order, or in the groups of
 *      Algorithm 1 (Sec. 3): all blocks of a group are extrapolated in
 *      parallel from the frame state at the start of the group.
 */
#ifndef FSE_H
#define FSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FSE_OK 0
#define FSE_EINVAL 1     /* bad argument: NULL, size, stride, parameter     */
#define FSE_ENOMEM 2     /* device/host allocation failed or over budget    */
#define FSE_EAGAIN 3     /* admission refused for now; retry later          */
#define FSE_ETIMEDOUT 4  /* a bounded device-side wait gave up              */
#define FSE_ECUDA 5      /* a CUDA runtime call failed                      */
#define FSE_ENOTFOUND 6  /* unknown ticket                                  */
#define FSE_ETOOBIG 7    /* frame larger than fse_conceal_frame_noalloc's
                            fixed scratch (1920 x 1088 samples)            */

/* ---- parameters ---------------------------------------------------------- */
#define FSE_ORDER_LINESCAN 0   /* conventional raster order, one block at a time */
#define FSE_ORDER_OPTIMIZED 1  /* Algorithm 1 groups (Sec. 3)                   */

/* Arithmetic of the initial weighted projection (DFT of w*f and of w).  The
 * iterations always run in FP32.  FSE_PREC_FP32 computes the projection on
 * the FP32 pipes; the others run it as DFT-as-GEMM on the tensor cores with
 * FP32 accumulation and the named operand type. */
#define FSE_PREC_FP32 0
#define FSE_PREC_TF32 1
#define FSE_PREC_BF16 2
#define FSE_PREC_FP16 3
#define FSE_PREC_BF16X3 4      /* split-BF16 operands (hi*hi + hi*lo + lo*hi) */
#define FSE_PREC_TF32X3 5      /* split-TF32 operands, FP32-grade accuracy    */

/* How the groups are dispatched on the device. */
#define FSE_EXEC_GROUPS 0      /* one launch per dependency level (blocks of a
                                  level are independent), or per group with
                                  FSE_OPT_GROUP_LAUNCHES (the plain path)      */
#define FSE_EXEC_PERSISTENT 1  /* one persistent launch over all frames; a block
                                  starts once every earlier-group block whose
                                  samples lie in its area has published its
                                  completion flag (bounded device waits)      */

#define FSE_MAX_ITERS 1024

typedef struct fse_params {
    int block;      /* block size B: 16, 8, 4 or 2 (Sec. 4 uses all four)  */
    int border;     /* frame width d around the block; 16 supported        */
    int dft;        /* DFT size per dimension; 64 supported                */
    int iters;      /* K, 0 .. FSE_MAX_ITERS (the paper uses 200)          */
    float rho;      /* weighting decay rho-hat, 0 < rho < 1 (paper: 0.8)   */
    float delta;    /* weight factor of R, 0 <= delta <= 1 (paper: 0.2)    */
    float gamma;    /* ODC factor, 0 < gamma <= 1 (paper: 0.5)             */
    int order;      /* FSE_ORDER_*                                         */
    int precision;  /* FSE_PREC_*                                          */
    int executor;   /* FSE_EXEC_*                                          */
} fse_params;

/* One frame of 8-bit luma.  luma, out and loss_mask are [height][stride]
 * row-major bytes; loss_mask[y*stride+x] != 0 marks a lost sample.  out may
 * alias luma.  stride >= width.  A block is lost when any of its in-image
 * samples is lost.  Limits (FSE_EINVAL beyond them): width x height <= 2^30,
 * height x stride < 2^31 and height x (width rounded up to 32) < 2^31, so
 * that every sample offset fits 32 bits. */
typedef struct fse_frame {
    const uint8_t *luma;
    uint8_t *out;
    const uint8_t *loss_mask;
    int width, height, stride;
} fse_frame;

typedef struct fse_ctx fse_ctx;

typedef struct fse_stats {
    int status;          /* FSE_OK or the error of this request              */
    int lost_blocks;     /* blocks concealed                                  */
    int groups;          /* processing-order groups                           */
    int batch_requests;  /* requests in the device batch that carried it      */
    int inflight;        /* other device batches in flight when it started    */
    double queue_ms;     /* submit -> start of its device batch               */
    double latency_ms;   /* submit -> result copied back                      */
} fse_stats;

/* Processing order (Sec. 3, Algorithm 1; or line scan).  Host only.
 * block_lost: [bh*bw] bytes, non-zero = block has lost samples.
 * Outputs, caller-owned: group_of_block [bh*bw] (-1 = nothing to do, else
 * the 0-based group), group_ptr [bh*bw + 1], block_ids [bh*bw] (each group
 * lists its blocks in raster order; group g is block_ids[group_ptr[g] ..
 * group_ptr[g+1])), n_groups.  Readings: neighbours are the 8 adjacent
 * blocks; a corner block gets +5, another margin block +3; N_min is the
 * minimum over blocks with N >= 0; S is filled in raster order.
 * Errors: FSE_EINVAL on NULL pointers, bw/bh <= 0 or an unknown order. */
int fse_plan_order(int bw, int bh, const uint8_t *block_lost, int order,
                   int32_t *group_of_block, int32_t *group_ptr,
                   int32_t *block_ids, int32_t *n_groups);

/* Claim order of the lost blocks of n_frames frames for the executors (host
 * only; no counterpart in the paper, which states the groups' order only).
 * Lost block s depends on lost block d when d lies within the area footprint
 * of s (+-16/B blocks) and has a smaller group: s reads d's concealed samples
 * (class R, Sec. 2).  Every order with dependencies first gives the result of
 * the group order (Sec. 3).
 * Inputs: per frame bw[i], bh[i]; group_of_block = the frames' group maps
 * (as from fse_plan_order) concatenated, frame i's [bh[i]*bw[i]] after
 * frame i-1's; block = B (16, 8, 4 or 2).
 * mode 0 (one launch per level): level = 1 + the largest level of the
 *   block's dependencies, 0 without; items sorted by level, then frame, then
 *   group order; level_start [lost blocks + 1] receives the first item of
 *   each level and the total, n_levels the number of levels.
 * mode 1 (for comparison): list schedule of `workers` CTAs with unit block
 *   times, longest chain of dependants first (ties: ready first; initially
 *   frame by frame in group order, later in order of release); each round
 *   starts up to `workers` ready blocks, whose dependants become ready in
 *   the next round.
 * mode 2: longest chain of dependants first (height, counting the block),
 *   then frame, then group order; topological because a block's height
 *   exceeds its dependants'.
 * mode 3 (persistent executor with `workers` CTAs): the mode-2 order cut
 *   into rounds of `workers` claims; each block's round is raised to one past
 *   the latest round of its dependencies (taken in group order); items are
 *   then sorted by round, within a round by frame, then group order.
 * level_start / n_levels are used in mode 0 only.
 * Output, caller-owned: items [2 * lost blocks] (frame, block) pairs.
 * Errors: FSE_EINVAL on NULL pointers, a dimension <= 0, an unsupported
 * block size, an unknown mode or workers <= 0 in mode 1 or 3. */
int fse_plan_claims(int n_frames, const int32_t *bw, const int32_t *bh,
                    const int32_t *group_of_block, int block, int workers, int mode,
                    int32_t *items, int32_t *level_start, int32_t *n_levels);

/* Measured ceilings of the units the iteration loop runs on (no counterpart
 * in the paper; used as roofline denominators): *smem_gbs = shared-memory
 * load bandwidth of 16-byte conflict-free loads on every SM (GB/s),
 * *fp32_tflops = packed FP32 FMA throughput on every SM (TFLOP/s).  Runs two
 * short kernels (a few ms) on `device`, which becomes the current device.
 * Errors: FSE_EINVAL (NULL output, bad device), FSE_ENOMEM, FSE_ECUDA. */
int fse_measure_peaks(int device, double *smem_gbs, double *fp32_tflops);

/* Microbenchmark of the iteration loop alone (Sec. 4: K selections and
 * transform-domain residual updates of a 64x64 spectrum per block; no
 * gather, projection or synthesis), so that the cost of each loop design
 * can be measured apart from the rest of the per-block kernel.  Runs
 * ctas_per_sm x (SM count) CTAs of 256 threads, each extrapolating
 * blocks_per_cta synthetic spectra for `iters` iterations, twice (the
 * first as warm-up).  variant: the selection step of the loop, 0 = two
 * block barriers per iteration (warp maxima, then the search of the
 * winning warp), 1 = one barrier (row maxima reduced during the update,
 * one candidate slot per warp), 2 = one barrier (every warp searches its
 * maximum), 3 = two barriers (the winning warp named from the warp maxima,
 * which alone searches and publishes the pre-packed update step; the form
 * the block kernels use), 4 = as 3
 * with the search by a match mask and a selection tree.  All variants
 * select the same indices.  Two calibration forms make no selection (the
 * index sequence is a fixed hash of the iteration): 5 = the update alone,
 * 6 = the update with a warp reduction and one block barrier.  7 = as 0,
 * the candidates read once after the second barrier and the winner's value
 * taken by shuffles; 8 = as 7, the block maximum gathered by a shared
 * atomic maximum into one word; 9 = as 7 with W kept once, as planes of
 * real and imaginary parts (4 CTAs per SM fit); 10 = as 9 with 128-thread
 * CTAs whose threads hold 32 entries.
 * Outputs: *ns_per_block_iter = kernel time x SMs / (blocks x iters), i.e.
 * nanoseconds per block-iteration per SM; *checksum = a hash of every
 * selected index (equal across variants).
 * Errors: FSE_EINVAL (NULL output, bad device, variant, iters outside
 * 1..FSE_MAX_ITERS, blocks_per_cta outside 1..4096, or more CTAs per SM
 * than can be resident), FSE_ENOMEM, FSE_ECUDA. */
int fse_loop_microbench(int device, int variant, int ctas_per_sm, int iters,
                        int blocks_per_cta, double *ns_per_block_iter, uint32_t *checksum);

/* Create a context on CUDA device `device`.  mem_budget bounds the device
 * workspace the context may hold (0 = no limit).  The context owns its
 * workspace (FP32 working frames, plans, status words) and a serving
 * thread started on the first fse_submit. */
int fse_ctx_create(fse_ctx **ctx, int device, size_t mem_budget);
void fse_ctx_destroy(fse_ctx *ctx);

/* Conceal n frames whose luma/out/loss_mask are DEVICE pointers.
 * Stream-ordered on `cuda_stream` (a cudaStream_t, NULL = legacy default
 * stream).  The call plans on the host: it reads the block-loss maps back
 * and synchronises the stream once before it enqueues the extrapolation;
 * it returns once the work is enqueued, so buffers must stay valid until
 * the stream passes it.  Not thread-safe per context.
 * Errors: FSE_EINVAL (params, sizes, NULL), FSE_ENOMEM, FSE_ECUDA,
 * FSE_ETIMEDOUT (reported by the next call that synchronises). */
int fse_conceal_batch(fse_ctx *ctx, const fse_frame *frames, int n,
                      const fse_params *params, void *cuda_stream);

/* Same as fse_conceal_batch for frames in HOST memory: copies the inputs to
 * the device, conceals, copies `out` back and returns when `out` holds the
 * result (so it reports FSE_ETIMEDOUT directly).  The block-loss maps come
 * from the host masks.  The inputs are copied in on a stream of the
 * context, the extrapolation runs on `cuda_stream`, the outputs are copied
 * back on another stream of the context.  Host buffers should be
 * page-locked for the copies to run asynchronously. */
int fse_conceal_batch_host(fse_ctx *ctx, const fse_frame *frames, int n,
                           const fse_params *params, void *cuda_stream);

/* Asynchronous form of fse_conceal_batch_host: enqueues the copies, plans
 * the batch on the host and enqueues its launch, then returns; *ticket
 * names the batch for fse_wait_batch.  Two batches can be in flight: the
 * host planning and the copies of one overlap the extrapolation of the
 * other.  A call made while two are in flight first waits for the older
 * one (its status is kept for its fse_wait_batch; the statuses of the 64
 * most recent unwaited batches are kept).  The frames' host buffers (luma,
 * loss_mask, out) must stay valid and unmodified (out: unread) until
 * fse_wait_batch(ticket) returns; they should be page-locked, since a copy
 * to or from pageable memory makes the call wait for it.
 * Errors: as fse_conceal_batch_host, FSE_EINVAL for a NULL ticket. */
int fse_conceal_batch_host_async(fse_ctx *ctx, const fse_frame *frames, int n,
                                 const fse_params *params, void *cuda_stream,
                                 uint64_t *ticket);

/* Wait until the batch `ticket` of fse_conceal_batch_host_async has written
 * its outputs to host memory and return its status (FSE_ETIMEDOUT if a
 * device wait of its launch failed, FSE_ECUDA).  A ticket can be waited for
 * once.  Errors: FSE_ENOTFOUND for an unknown or already waited ticket. */
int fse_wait_batch(fse_ctx *ctx, uint64_t ticket);

/* FSE of n pre-gathered areas (DEVICE pointers), for inspection and parity
 * tests of the per-block computation alone.  The area is M x M with
 * M = params->block + 32, stored in the top-left of a 48x48 array.
 *   area_f   [n][48][48] float: sample values (ignored where weight is 0)
 *   area_cls [n][48][48] uint8: 0 = A, 1 = R, 2 = B_i, 3 = B_o, 4 = outside
 *                               (entries beyond M x M are ignored)
 *   g_out    [n][16][16] float: real part of the model at area positions
 *                               (16 + i, 16 + j); the block is the top-left
 *                               B x B, unclamped
 *   u_out    [n][K] int32 (optional): selected index 64*k_m + k_n, -1 if
 *                               the area has no support
 *   dc_out   [n][K][2] float (optional): coefficient increments
 *   r_out    [n][64][64][2] float (optional): weighted residual spectrum
 *                               after K iterations
 * Stream-ordered, asynchronous. */
int fse_extrapolate_areas(fse_ctx *ctx, const float *area_f,
                          const uint8_t *area_cls, int n,
                          const fse_params *params, float *g_out,
                          int32_t *u_out, float *dc_out, float *r_out,
                          void *cuda_stream);

/* Serving.  fse_submit queues one request whose luma/out/loss_mask are
 * HOST pointers; they are borrowed until fse_poll reports done.  Requests
 * are admitted into device batches as workspace memory frees up; batches
 * overlap on the device (continuous batching).  Page-locked buffers are
 * copied to and from the device directly; pageable ones through staging
 * buffers of the library.  Non-blocking.
 * Errors: FSE_EINVAL, FSE_EAGAIN (queue full; retry later). */
int fse_submit(fse_ctx *ctx, const fse_frame *frame, const fse_params *params,
               uint64_t *ticket);

/* Non-blocking.  *done = 1 once the request finished (out written); then
 * *out (optional) receives its statistics and the ticket is released.
 * Errors: FSE_ENOTFOUND for an unknown or already released ticket. */
int fse_poll(fse_ctx *ctx, uint64_t ticket, int *done, fse_stats *out);

/* Block until every submitted request has finished (or timeout_ms passes;
 * returns FSE_ETIMEDOUT then).  timeout_ms < 0 waits without limit. */
int fse_drain(fse_ctx *ctx, int timeout_ms);

/* Device-side statistics of the last fse_conceal_batch / _host call:
 * lost blocks, groups (max over frames) and kernel launches enqueued (the
 * extrapolation launches, plus one for the block-loss map kernel when the
 * maps were built on the device). */
int fse_last_batch_info(fse_ctx *ctx, int *lost_blocks, int *groups,
                        int *launches);

/* Device times of the extrapolation launches of the last min(n, 64) device
 * batches of the synchronous API that launched any (ms[0] the most recent),
 * from the same CUDA events as fse_last_kernel_ms; *count receives how many
 * were written.  Waits for their end events.  Lets a caller time a run of
 * batches without synchronising between them.  Errors: FSE_EINVAL, FSE_ECUDA. */
int fse_recent_kernel_ms(fse_ctx *ctx, int n, float *ms, int *count);

/* Launch configuration the last fse_conceal_batch / _host call ran with:
 * *executor (FSE_EXEC_*) and *ctas_per_sm (persistent CTAs per SM; 0 for
 * FSE_EXEC_GROUPS).  Either pointer may be NULL.  Errors: FSE_EINVAL. */
int fse_last_batch_config(fse_ctx *ctx, int *executor, int *ctas_per_sm);

/* The full launch shape of the last fse_conceal_batch / _host call: as
 * fse_last_batch_config, plus *claim_order (FSE_CLAIM_*, the persistent
 * executor's claim order; 0 for FSE_EXEC_GROUPS), *threads_per_cta (256:
 * one thread owns 16 spectrum entries) and *blocks_per_cta (1).  Any pointer
 * may be NULL.  Errors: FSE_EINVAL. */
int fse_last_batch_shape(fse_ctx *ctx, int *executor, int *ctas_per_sm, int *claim_order,
                         int *threads_per_cta, int *blocks_per_cta);

/* Where a block's time goes (tracing; no counterpart in the paper): with
 * FSE_OPT_PHASE_CLOCKS set, the persistent executor records the SM clock of
 * its first thread at the phase boundaries of every block, and this call
 * returns, for the last synchronous persistent batch, the mean SM clocks per
 * block of each phase: clk[0] dependency wait, [1] TMA staging of the area,
 * [2] gather (classes, weights), [3] projection (and W: copied from its
 * table or computed), [4] the K iterations, [5] synthesis, [6] store and
 * release (n values, at most 7).  Three blocks share an SM, so a phase's
 * clocks include the issue slots other blocks take.  *blocks receives the
 * blocks averaged (0: nothing recorded).  Synchronises `cuda_stream`.
 * Errors: FSE_EINVAL, FSE_ECUDA. */
int fse_last_phase_clocks(fse_ctx *ctx, void *cuda_stream, double *clk, int n, int *blocks);

/* Device time of the extrapolation launches of the last fse_conceal_batch
 * or fse_conceal_batch_host call (the persistent kernel, or all group
 * launches), from CUDA events recorded on the call's stream around them.
 * Waits for the end event.  *ms = 0 when the batch had nothing to do.
 * Errors: FSE_EINVAL (NULL), FSE_ECUDA. */
int fse_last_kernel_ms(fse_ctx *ctx, float *ms);

/* Copy the FP32 working frame of frame `frame` of the last fse_conceal_batch
 * or fse_conceal_batch_host call into dst (DEVICE pointer, [height][dst_stride]
 * floats).  Values are defined at lost samples only: the clamped, unrounded
 * model values that later blocks read; other samples are unspecified.
 * Valid until the next batch call.  Stream-ordered, asynchronous.
 * Errors: FSE_EINVAL for a bad index, NULL dst or dst_stride < width. */
int fse_copy_work(fse_ctx *ctx, int frame, float *dst, int dst_stride,
                  void *cuda_stream);

/* Copy the selection trace of frame `frame` of the last batch into dst
 * (DEVICE pointer, [bh*bw][iters] int16, blocks in raster order): for every
 * concealed block the K selected indices 64*k_m + k_n in iteration order,
 * -1 when its area had no support; rows of blocks without loss are
 * unspecified.  Only recorded while FSE_OPT_KEEP_TRACE is 1.
 * Errors: FSE_EINVAL for a bad index, NULL dst or no recorded trace. */
int fse_copy_trace(fse_ctx *ctx, int frame, int16_t *dst, void *cuda_stream);

/* Conceal one frame without allocating anything.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc, for example a plug-in whose host application owns all device
 * memory through its own pool or budget, or code running where a stray
 * allocation would break a memory plan fixed in advance.
 *
 * frame: luma, out and loss_mask are DEVICE pointers (as for
 * fse_conceal_batch); at most 1920 x 1088 samples, else FSE_ETOOBIG.
 * params: as for fse_conceal_batch; precision must be FSE_PREC_FP32; the
 * executor field is ignored (one launch per processing-order group).
 *
 * Scratch: one fixed array of about 8.5 MB in device memory, declared in the
 * library, that every GPU which loads the library holds until the process
 * exits.  No context is needed and the call makes no device or host
 * allocation (host staging is static too).  Every call looks up the current
 * device's address of the array (the first lookup on a device loads the
 * library's module there), so make the first call before any stream
 * capture.  Every call shares the array: calls whose GPU work overlaps
 * (other host threads, other streams) race and must be serialised by the
 * caller; host-side staging is serialised internally.
 * Stream-ordered on `cuda_stream`; the call synchronises that stream twice
 * (to read the block-loss map and to release its staging) and returns with
 * the extrapolation launches enqueued.
 * Cost: this is not the fast path.  Areas are gathered with plain loads
 * (no TMA staging) and every processing-order group is its own launch, so
 * the line-scan order (one block per group) is bound by launch latency:
 * about 2,400 serial launches for a 1080p frame with 30% of its blocks lost.
 * The processing order is planned by the same code as fse_plan_order.
 * Errors: FSE_EINVAL, FSE_ETOOBIG, FSE_ECUDA. */
int fse_conceal_frame_noalloc(const fse_frame *frame, const fse_params *params,
                              void *cuda_stream);

/* Weight-spectrum table of one class pattern (inspection; what
 * FSE_OPT_W_TABLES gives the blocks of that pattern): W = DFT64 of the 48x48
 * weights of Eq. (2) (Sec. 2 sub-areas: the 16x16 centre is B_i, each of the
 * eight neighbour cells is A, R, B_o or outside as the key says; see
 * FSE_OPT_W_TABLES), written to dst (DEVICE pointer, 16-byte aligned,
 * 72,704 bytes) as 71 rows of 64 float4 (Re W[r][c], Re W[r][c ^ 32],
 * Im W[r][c], Im W[r][c ^ 32]), rows 64..70 repeating rows 0..6.
 * key: 16 bits, two per neighbour in raster order (dy, dx) = (-1,-1),
 * (-1,0), (-1,1), (0,-1), (0,1), (1,-1), (1,0), (1,1); 0 = A (not lost),
 * 1 = R (concealed earlier), 2 = B_o (lost, later), 3 = outside the image.
 * builder: 1 = the FP32 split DFTs of the block kernels, 2 = DFT-as-GEMM on
 * the tcgen05 tensor cores (split-TF32 operands, FP32 accumulation).
 * Synchronises `cuda_stream`.
 * Errors: FSE_EINVAL (bad key, rho outside (0, 1), delta outside [0, 1],
 * builder, NULL or unaligned dst), FSE_ENOMEM, FSE_ECUDA, FSE_ETIMEDOUT (a
 * tensor-core product did not complete within its bounded wait). */
int fse_weight_table(fse_ctx *ctx, int key, float rho, float delta, int builder, void *dst,
                     void *cuda_stream);

/* Context options (host-side settings; take effect on the next batch).
 *   FSE_OPT_SPIN_LIMIT       polls a device-side dependency wait makes
 *                            before it gives up with FSE_ETIMEDOUT
 *                            (default 2^23, about a second)
 *   FSE_OPT_PERSISTENT_CTAS  CTAs per SM of the persistent launch
 *                            (0 = as many as fit)
 *   FSE_OPT_SERVE_SLOTS      concurrent device batches of the server (1..16;
 *                            before the first fse_submit)
 *   FSE_OPT_SERVE_MAX_BATCH  requests per device batch (>= 1)
 *   FSE_OPT_TEST_STUCK_DEP   test hook: 1 adds a dependency that nothing
 *                            releases to the last work item of the next
 *                            persistent batch, so its bounded wait runs out
 *   FSE_OPT_KEEP_TRACE       1 records the selection trace of every block
 *                            (see fse_copy_trace); 0 (default) does not
 *   FSE_OPT_GROUP_LAUNCHES   1: FSE_EXEC_GROUPS launches once per group of
 *                            the processing order (Sec. 3, the plain path),
 *                            0 (default): once per dependency level
 *   FSE_OPT_AUTOTUNE         1: fse_conceal_batch calls with
 *                            FSE_EXEC_PERSISTENT choose, per batch shape
 *                            (frames, samples, K, B, order, precision), the
 *                            fastest of the launch configurations whose
 *                            results are identical: the persistent launch
 *                            with 1 .. (occupancy limit) CTAs per SM and
 *                            each claim order (FSE_CLAIM_*), or one launch
 *                            per dependency level.  The first call of a
 *                            shape runs one untimed pass, then times every
 *                            candidate twice (same output bytes); later
 *                            calls reuse the choice (fse_last_batch_shape
 *                            reports it).
 *                            0 (default): as requested.
 *   FSE_OPT_INPUTS_READY     1: the loss masks of each fse_conceal_batch call
 *                            are complete when the call is made (no work
 *                            still queued on its stream writes them); the
 *                            call copies them to the host on a side stream
 *                            and plans the batch while the stream's earlier
 *                            work (a previous batch) still runs.  A failed
 *                            device wait of a batch is then reported by a
 *                            later call.  0 (default): the masks are read in
 *                            stream order.
 *   FSE_OPT_SERVE_LATENCY_MS latency-aware admission of fse_submit: while
 *                            the oldest request not yet on the GPU has
 *                            waited longer than this many milliseconds,
 *                            new requests are refused with FSE_EAGAIN, so
 *                            past saturation the queueing delay stays near
 *                            the budget instead of growing without bound.
 *                            0 (default): admission by queue length and
 *                            memory only.
 *   FSE_OPT_CLAIM_ORDER      order in which the persistent executor's CTAs
 *                            claim blocks (every order gives the same
 *                            bytes: a block waits only for the
 *                            earlier-group blocks in its area):
 *                            FSE_CLAIM_DELAYED (default) the longest chain
 *                            of dependants first, cut into rounds of one
 *                            claim per CTA, each block moved past its
 *                            dependencies' round; FSE_CLAIM_HEIGHT the
 *                            longest chain first; FSE_CLAIM_LIST a list
 *                            schedule of rounds of ready blocks.
 *   FSE_OPT_PHASE_CLOCKS     1: the persistent executor records the phase
 *                            clocks of every block (fse_last_phase_clocks;
 *                            FP32 projections only; an instrumented build of
 *                            the kernel, not the one that serves requests);
 *                            0 (default): it does not.
 *   FSE_OPT_W_TABLES         blocks whose sub-area classes are fixed by
 *                            their eight neighbours (16x16 blocks lost as a
 *                            whole, FP32 projection) take the spectrum of
 *                            their weights, W, from a table per class
 *                            pattern, computed once per context and
 *                            (rho, delta) and kept in device memory within
 *                            the memory budget (72,704 bytes per pattern);
 *                            the block kernels then project only w f.
 *                            2 (default): tables by DFT-as-GEMM on the
 *                            tcgen05 tensor cores (split-TF32, FP32
 *                            accumulation; FP32-grade); 1: tables by the
 *                            blocks' own FP32 split DFTs (byte-identical to
 *                            0); 0: every block computes W.
 * Errors: FSE_EINVAL for an unknown option or value. */
#define FSE_OPT_SPIN_LIMIT 1
#define FSE_OPT_PERSISTENT_CTAS 2
#define FSE_OPT_SERVE_SLOTS 3
#define FSE_OPT_SERVE_MAX_BATCH 4
#define FSE_OPT_TEST_STUCK_DEP 5
#define FSE_OPT_KEEP_TRACE 6
#define FSE_OPT_GROUP_LAUNCHES 7
#define FSE_OPT_AUTOTUNE 8
#define FSE_OPT_INPUTS_READY 9
#define FSE_OPT_SERVE_LATENCY_MS 10
#define FSE_OPT_W_TABLES 11
#define FSE_OPT_CLAIM_ORDER 12
#define FSE_OPT_PHASE_CLOCKS 13
#define FSE_CLAIM_DELAYED 0
#define FSE_CLAIM_HEIGHT 1
#define FSE_CLAIM_LIST 2
int fse_ctx_set_option(fse_ctx *ctx, int option, long long value);

const char *fse_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif
