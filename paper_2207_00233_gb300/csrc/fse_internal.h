// Internal declarations shared by the library's translation units
// (device kernels in fse_kernels.cu, host runtime in fse_api.cpp).
#pragma once

#include <cstddef>
#include <cstdint>
#include <functional>
#include <vector>

#include <cuda_runtime.h>

namespace fse {

// Fixed geometry of the supported configuration: 16x16 blocks, a 16-sample
// frame around the block (Sec. 4: d = 16), a 48x48 extrapolation area and a
// 64x64 DFT basis.
constexpr int kBlock = 16;
constexpr int kBorder = 16;
constexpr int kArea = kBlock + 2 * kBorder;  // 48
constexpr int kDft = 64;
constexpr int kThreads = 256;                // one CTA per lost block
constexpr int kWarps = kThreads / 32;

// Shared-memory layout of the per-block CTA (bytes).  The weight spectrum W
// is stored as W4[row][j] = (Re W[row][j], Re W[row][j^32], Im W[row][j],
// Im W[row][j^32]) so that one 16-byte load gives a thread both columns it
// owns; rows 0..6 are repeated as rows 64..70 so that the eight consecutive
// rows a thread reads never wrap.  Before the iterations the same region
// holds the area tiles and the first projection stage.
constexpr int kW4Rows = kDft + 7;
constexpr int kW4Bytes = kW4Rows * kDft * 16;          // 72704
constexpr int kTwOff = kW4Bytes;                       // 64 x float2
constexpr int kRedOff = kTwOff + kDft * 8;             // reduction scratch
constexpr int kRedBytes = 8 * 4 + 8 * 16 + 64;         // smax[8], cand[8], misc
constexpr int kXrwOff = kRedOff + kRedBytes;           // W's real columns (FP32 projection)
constexpr int kXrwBytes = 2 * 33 * 8;                  // columns k_n = 0, 32; rows 0..32
constexpr int kListOff = kXrwOff + kXrwBytes;          // dc list, then u list
// misc[2..3]: TMA mbarrier, misc[4]: its next phase parity, misc[5..6]: the
// persistent executor's claimed item and wait result; misc[8..15]: thread
// 0's clock at the phase boundaries of the current block (kPhaseStamps)
constexpr int kMbarOff = kRedOff + 8 * 4 + 8 * 16 + 8;
static_assert(kMbarOff % 8 == 0 && kMbarOff + 20 <= kListOff, "mbarrier placement");
constexpr int kPhaseStamps = 8;
constexpr int kStampOff = kRedOff + 8 * 4 + 8 * 16 + 32;
static_assert(kStampOff + 4 * kPhaseStamps <= kRedOff + kRedBytes, "phase stamps placement");
inline int smem_bytes(int iters) {
    return kListOff + iters * 8 + ((iters * 2 + 15) / 16) * 16;
}

// Scratch inside the W4 region before the iterations.  The area tiles have
// a row stride of 49 floats so that 32 consecutive rows of one column fall
// into 32 different banks.
constexpr int kTileStride = kArea + 1;                          // 49
constexpr int kXTileOff = 0;                                    // 48x49 float: w*f
constexpr int kWTileOff = kXTileOff + kArea * kTileStride * 4;  // 48x49 float: w
constexpr int kHalfCols = kDft / 2 + 1;                         // 33 (real input)
constexpr int kYxOff = kWTileOff + kArea * kTileStride * 4;     // 48x33 float2
constexpr int kYwOff = kYxOff + kArea * kHalfCols * 8;          // 48x33 float2
static_assert(kYwOff + kArea * kHalfCols * 8 <= kW4Bytes, "scratch overflow");
// Column-DFT intermediates of the FP32 projection (33 x 132 floats each):
// the x input's in the (then free) tile region, the w input's after the
// half spectra.
constexpr int kTswOff = kYwOff + kArea * kHalfCols * 8;         // 44160
static_assert(kTswOff + 33 * 132 * 4 <= kW4Bytes, "column-DFT scratch overflow");
// Row-DFT intermediates (64 planes x 96 rows floats), before the column DFTs
// reuse the space.
constexpr int kZsOff = kTswOff;
static_assert(kZsOff + 64 * 2 * kArea * 4 <= kW4Bytes, "row-DFT scratch overflow");
// After the iterations the W4 region holds the synthesis tables, in chunks
// of kSynChunk iterations: P[it][i] = dc_it exp(+j 2 pi u_m (16+i) / 64) as
// (Re, Re, -Im, -Im) and E[it][j] = exp(+j 2 pi u_n (16+j) / 64) as 16 real
// then 16 imaginary parts; then the eight warps' partial 16x16 sums.
constexpr int kSynChunk = 128;
constexpr int kSynPartOff = kSynChunk * 16 * 16 + kSynChunk * 32 * 4;
static_assert(kSynPartOff + kWarps * 256 * 4 <= kW4Bytes, "synthesis tables overflow");

struct KParams {
    float rho, delta, gamma;
    int iters;
    const uint4 *frags;  // packed DFT operand fragments of the tensor-core
                         // projection (null for FSE_PREC_FP32)
    int lb;              // log2 of the block size B; the area is (B + 32)^2
    int *error;          // status word for a failed TMA wait (group launches;
                         // null: frames are gathered with plain loads)
    uint32_t *clocks;    // persistent executor: [items][kPhaseStamps] phase
                         // stamps of every block (FSE_OPT_PHASE_CLOCKS), or null
};

// Block sizes: B = 16 (the 48x48 area fills the tile) or B = 8, 4, 2 with the
// same 16-sample frame: the (B + 32)^2 area occupies the top-left of the
// 48x48 tile and the rest weighs 0 (the zero-extended DFT is unchanged).
inline int block_log2(int block) {
    return block == 16 ? 4 : block == 8 ? 3 : block == 4 ? 2 : block == 2 ? 1 : -1;
}

// Tensor-core projection (warp-level mma.sync).  Stage 1 multiplies the
// stacked area tiles [w*f; w] (96 x 48) by [cos | -sin] (48 x 80, half
// spectrum k_n = 0..32, padded to 40 columns each); stage 2 multiplies
// [cos | sin](k_m) (64 x 96) by [[Y_re, Y_im]; [Y_im, -Y_re]] (96 x 80 per
// input), which gives Re and Im of the spectrum directly.
constexpr int kYRows = 2 * kArea;           // 96
constexpr int kYCols = 80;                  // 40 real + 40 imaginary
constexpr int kYStride = kYCols + 4;        // conflict-free fragment loads
constexpr int kYOff = 2 * kArea * kTileStride * 4;                 // after the tiles
constexpr int kR0Off = kYOff + kYRows * kYStride * 4;              // 64 x 33 float2
static_assert(kR0Off + kDft * kHalfCols * 8 <= kW4Bytes, "projection scratch overflow");

// TMA staging of a frame area, before the gather: the luma and loss-mask
// tiles of 48 x 48 samples, starting at the sample row of the area and at
// the 16-byte boundary at or below its first column (the copy must start on
// a 16-byte boundary).  With the 16-sample frame the area's first column is
// at most 14 samples past that boundary and M = B + 32 <= 34 + 14 for
// B < 16, so 48 columns always cover it.  The tiles share the (not yet
// used) projection scratch at kYOff.  Samples of the working frame are read
// only where the area holds concealed samples (class R), with plain loads.
constexpr int kStageCols = 48, kStageRows = 48;
constexpr int kStageLumaOff = kYOff;
constexpr int kStageMaskOff = kStageLumaOff + kStageCols * kStageRows;
constexpr int kStageBytes = kStageCols * kStageRows * 2;  // 4608
static_assert(kStageLumaOff % 128 == 0 && kStageMaskOff % 128 == 0,
              "TMA destinations must be 128-byte aligned");
static_assert(kStageMaskOff + kStageCols * kStageRows <= kW4Bytes, "staging overflow");
constexpr int kTensorMapBytes = 128;       // one CUtensorMap
constexpr int kMapsPerFrame = 2;           // luma, mask
size_t frag_bytes(int precision);
cudaError_t launch_build_frags(int precision, const float2 *tw, uint4 *out,
                               cudaStream_t stream);

// Device-side description of one frame of a batch.
struct FrameDesc {
    const uint8_t *luma;     // [H][stride]
    const uint8_t *mask;     // [H][stride], non-zero = lost
    uint8_t *out;            // [H][stride]
    float *work;             // [H][wstride] FP32 working frame
    const int32_t *gob;      // [bh][bw] group of each block, -1 = no loss
    int H, W, stride, wstride, bh, bw;
    int16_t *trace;          // [bh*bw][iters] selected indices, or null
    uint32_t *done;          // [bh*bw] completion flags (persistent executor)
    int lb;                  // log2 of the block size B (1..4)
    int pad0;
    const void *tmaps;       // 2 tensor maps (luma, mask), 64-byte aligned,
                             // or null: gather with plain loads
    const uint64_t *wtab;    // [bh*bw] device address of the block's weight-
                             // spectrum table (W4 layout, kW4Bytes), 0: the
                             // block computes W itself; null: no tables
};

// Weight-spectrum tables.  W = DFT64(w) depends only on the sub-area classes
// of the area (Sec. 2: A, R, B_i, B_o, outside) and on rho and delta.  With
// B = 16 and a block that is lost as a whole, those classes follow from the
// states of its eight neighbour blocks: 0 = A (not lost), 1 = R (lost as a
// whole, earlier group), 2 = B_o (lost as a whole, same or later group),
// 3 = outside the image.  The key packs them, 2 bits each, neighbours in
// raster order (dy, dx) = (-1,-1), (-1,0), (-1,1), (0,-1), (0,1), (1,-1),
// (1,0), (1,1).  A table holds W in the W4 layout of the shared-memory
// region, kW4Bytes bytes, so that a block copies it in with one bulk copy.
constexpr int kWKeyStates = 4;
constexpr int kWKeys = 1 << 16;
// Fills the tables of `n` keys (FP32 split DFTs, the arithmetic of the
// in-kernel projection): keys [n] (device), dst [n] table addresses (device).
cudaError_t launch_wtables(const int32_t *keys, const uint64_t *dst, int n, float delta,
                           const float *rho_tab, const float2 *tw_tab, cudaStream_t stream);
// The same tables as two DFT-as-GEMM stages on the tcgen05 tensor cores with
// split-TF32 operands and FP32 accumulation (fse_wtable_tc.cu); image: the
// constant DFT operands (wtable_tc_image, uploaded once); error: status word
// for a product that did not complete in time.
void wtable_tc_image(std::vector<float> &img);
int wtable_tc_image_floats();
cudaError_t launch_wtables_tc(const int32_t *keys, const uint64_t *dst, int n, float delta,
                              const float *rho_tab, const float4 *image, int *error,
                              cudaStream_t stream);

// Work of the persistent executor: items are (frame, block) pairs in a claim
// order in which every block follows its dependencies (the earlier-group lost
// blocks within its area footprint).  A claimed item waits until those have
// set their completion flags; each was claimed earlier by a running CTA.
struct WorkQueue {
    const int2 *items;       // [n] (frame, block)
    int *head;               // work counter
    int *error;              // status word: 0 ok, else FSE_ETIMEDOUT
    int n;
    int stuck_item;          // test hook: this item also waits on its own
                             // flag, which nothing sets (-1: none)
    long long spin_limit;    // polls before a wait gives up
};

// Launchers (fse_kernels.cu).  All are asynchronous on `stream`.
// lost_out[b] = 1 when any in-image sample of block b is lost; part_out
// (optional) [b] = 1 when some in-image sample of b is not lost.  Both start
// zeroed by the caller.
cudaError_t launch_block_loss(const FrameDesc *frames_dev, int n_frames,
                              int max_blocks, uint8_t *lost_out, uint8_t *part_out,
                              const int *lost_off_dev, cudaStream_t stream);
cudaError_t launch_group(const FrameDesc *frames_dev, const int2 *items,
                         int n_items, const KParams &kp, const float *rho_tab,
                         const float2 *tw_tab, int precision,
                         cudaStream_t stream);
cudaError_t launch_persistent(const FrameDesc *frames_dev, const WorkQueue &wq,
                              const KParams &kp, const float *rho_tab,
                              const float2 *tw_tab, int precision, int grid,
                              cudaStream_t stream);
cudaError_t launch_areas(const float *area_f, const uint8_t *area_cls, int n,
                         const KParams &kp, const float *rho_tab,
                         const float2 *tw_tab, int precision, float *g_out,
                         int32_t *u_out, float *dc_out, float *r_out,
                         cudaStream_t stream);
int max_resident_ctas(int iters);   // CTAs of the block kernel per SM

// Claim order of a batch (host, fse_sched.cpp).  Per frame: the block grid,
// the group of each block and the lost blocks in group order; frame_depths
// fills, per block, the dependency level, the height (longest chain of
// dependants, counting the block) and the number of dependencies, for the
// footprint radius rad = 16 / B blocks.  The per-block arrays live in a grid
// padded by rad blocks of group -1 (no bounds tests in the footprint scans).
struct FrameDepths {
    int bw = 0, bh = 0;
    const int32_t *gob = nullptr;
    const int32_t *ids = nullptr;
    int n = 0;
    std::vector<int32_t> own_ids;               // storage of ids, when owned
    int rad = 0, pw = 0;                        // padding, padded row length
    std::vector<int32_t> gp;                    // padded group map
    std::vector<int32_t> nbr;                   // footprint offsets (no centre)
    std::vector<int32_t> pid;                   // padded cell of ids[j]
    std::vector<int32_t> level, height, indeg;  // per padded cell
    std::vector<int32_t> key;                   // claim round (delay_claims)
    int block_of(int c) const { return (c / pw - rad) * bw + (c % pw - rad); }
};
void frame_depths(FrameDepths &f, int rad);
// Items by level (independent sets); level_start[l] .. level_start[l + 1].
void level_claims(const std::vector<FrameDepths> &frames, std::vector<int2> &items,
                  std::vector<int> &level_start);
// Items by height, descending (persistent executor).
void height_claims(const std::vector<FrameDepths> &frames, std::vector<int2> &items);
// Items in the height order cut into rounds of `workers` claims, each block
// moved to no earlier than the round after its latest dependency's;
// pfor(n, fn) runs fn(0..n-1), possibly in parallel (one call per frame).
void delay_claims(std::vector<FrameDepths> &frames, int workers, std::vector<int2> &items,
                  const std::function<void(int, const std::function<void(int)> &)> &pfor);
// Items in list-schedule order for `workers` CTAs (consumes indeg).
void schedule_claims(std::vector<FrameDepths> &frames, int workers, std::vector<int2> &items);
bool precision_supported(int precision);

// Processing order of one frame (fse_plan.cpp): line scan or Algorithm 1,
// with the outputs of fse_plan_order, in caller-provided scratch of
// plan_scratch_bytes(bw, bh) bytes (4-byte aligned; unused for line scan).
// Allocates nothing.
constexpr size_t plan_scratch_bytes(int bw, int bh) {
    return (size_t)(bw + 2) * (bh + 2) * 5 + (size_t)14 * bw * bh * 4 + 14 * 4;
}
int plan_order_core(int bw, int bh, const uint8_t *block_lost, int order,
                    int32_t *group_of_block, int32_t *group_ptr, int32_t *block_ids,
                    int32_t *n_groups, void *scratch);

}  // namespace fse
