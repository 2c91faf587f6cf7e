// fse_conceal_frame_noalloc: concealment of one frame for callers that
// cannot allocate device memory (for example code that runs inside a
// memory-pool-managed or externally budgeted process where every cudaMalloc
// is forbidden, or a plug-in whose host framework owns all allocations).
//
// All scratch the frame path needs (frame descriptor, tables, block-loss
// map, processing-order plan, FP32 working frame) lives in one file-scope
// __device__ array of fixed size; every GPU that loads the library holds it
// until the process exits.  Host staging uses static arrays as well, so the
// call performs no device or host allocation.  The kernels are the ones of
// the regular frame path (block-loss map, one launch per processing-order
// group), given pointers into the fixed array.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/fse.h"
#include "fse_ctx.h"
#include "fse_internal.h"

namespace fse {
namespace {

// Fixed limits: frames up to 1920 x 1088 samples (1080p luma).
constexpr int kNaMaxW = 1920;
constexpr int kNaMaxH = 1088;
constexpr int kNaMaxBw = kNaMaxW / kBlock;   // 120
constexpr int kNaMaxBh = kNaMaxH / kBlock;   // 68
constexpr int kNaMaxBlocks = kNaMaxBw * kNaMaxBh;
constexpr int kNaWStride = kNaMaxW;          // floats per working-frame row

// Layout of the scratch array (byte offsets, each 256-aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffDesc = 0;
constexpr size_t kOffTw = align256(kOffDesc + sizeof(FrameDesc));
constexpr size_t kOffRho = align256(kOffTw + kDft * sizeof(float2));
constexpr size_t kOffLostOff = align256(kOffRho + kArea * kArea * sizeof(float));
constexpr size_t kOffLost = align256(kOffLostOff + 2 * sizeof(int));
constexpr size_t kOffGob = align256(kOffLost + kNaMaxBlocks);
constexpr size_t kOffItems = align256(kOffGob + kNaMaxBlocks * sizeof(int32_t));
constexpr size_t kOffWork = align256(kOffItems + kNaMaxBlocks * sizeof(int2));
constexpr size_t kScratchBytes = align256(kOffWork + (size_t)kNaMaxH * kNaWStride * sizeof(float));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;  // guards the static host staging below

// Static host staging.
FrameDesc h_desc;
float2 h_tw[kDft];
float h_rho[kArea * kArea];
int h_lost_off[2];
uint8_t h_lost[kNaMaxBlocks];
int32_t h_gob[kNaMaxBlocks];
int32_t h_ids[kNaMaxBlocks];
int32_t h_group_ptr[kNaMaxBlocks + 1];
int2 h_items[kNaMaxBlocks];
// scratch of the processing-order planner (the one fse_plan_order uses)
int32_t h_plan_scratch[(plan_scratch_bytes(kNaMaxBw, kNaMaxBh) + 3) / 4];

// cos / sin of 2 pi t / 64 with exact symmetries (t and 64 - t mirror each
// other; axis values exact).
void na_twiddles(float2 *tw) {
    double c[kDft], s[kDft];
    const double step = 2.0 * 3.14159265358979323846 / kDft;
    for (int t = 0; t <= kDft / 8; ++t) {
        c[t] = std::cos(step * t);
        s[t] = std::sin(step * t);
    }
    for (int t = kDft / 8 + 1; t <= kDft / 4; ++t) {
        c[t] = s[kDft / 4 - t];
        s[t] = c[kDft / 4 - t];
    }
    c[kDft / 4] = 0.0;
    s[kDft / 4] = 1.0;
    for (int t = kDft / 4 + 1; t <= kDft / 2; ++t) {
        c[t] = -c[kDft / 2 - t];
        s[t] = s[kDft / 2 - t];
    }
    s[0] = 0.0;
    s[kDft / 2] = 0.0;
    for (int t = kDft / 2 + 1; t < kDft; ++t) {
        c[t] = c[kDft - t];
        s[t] = -s[kDft - t];
    }
    for (int t = 0; t < kDft; ++t) tw[t] = make_float2((float)c[t], (float)s[t]);
}

#define NA_CK(call)                    \
    do {                               \
        if ((call) != cudaSuccess) {   \
            cudaGetLastError();        \
            return FSE_ECUDA;          \
        }                              \
    } while (0)

}  // namespace
}  // namespace fse

using namespace fse;

extern "C" int fse_conceal_frame_noalloc(const fse_frame *frame, const fse_params *params,
                                         void *cuda_stream) {
    if (!frame) return FSE_EINVAL;
    int rc = check_params(params);
    if (rc) return rc;
    if (params->precision != FSE_PREC_FP32 || params->block != kBlock) return FSE_EINVAL;
    if (!frame->luma || !frame->out || !frame->loss_mask || frame->width <= 0 ||
        frame->height <= 0 || frame->stride < frame->width)
        return FSE_EINVAL;
    if (frame->width > kNaMaxW || frame->height > kNaMaxH) return FSE_ETOOBIG;

    std::lock_guard<std::mutex> lk(g_mu);
    // The array's name is a host-side stand-in: its address on the current
    // device is looked up on every call (cheap next to the call's two stream
    // synchronisations), so it stays right if the device's context has been
    // reset and the module reloaded elsewhere.
    void *sym = nullptr;
    NA_CK(cudaGetSymbolAddress(&sym, g_noalloc_scratch));
    unsigned char *base = static_cast<unsigned char *>(sym);
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

    FrameDesc *d_desc = reinterpret_cast<FrameDesc *>(base + kOffDesc);
    float2 *d_tw = reinterpret_cast<float2 *>(base + kOffTw);
    float *d_rho = reinterpret_cast<float *>(base + kOffRho);
    int *d_lost_off = reinterpret_cast<int *>(base + kOffLostOff);
    uint8_t *d_lost = base + kOffLost;
    int32_t *d_gob = reinterpret_cast<int32_t *>(base + kOffGob);
    int2 *d_items = reinterpret_cast<int2 *>(base + kOffItems);
    float *d_work = reinterpret_cast<float *>(base + kOffWork);

    const int W = frame->width, H = frame->height;
    const int bw = (W + kBlock - 1) / kBlock, bh = (H + kBlock - 1) / kBlock;
    h_desc.luma = frame->luma;
    h_desc.mask = frame->loss_mask;
    h_desc.out = frame->out;
    h_desc.work = d_work;
    h_desc.gob = d_gob;
    h_desc.H = H;
    h_desc.W = W;
    h_desc.stride = frame->stride;
    h_desc.wstride = kNaWStride;
    h_desc.bh = bh;
    h_desc.bw = bw;
    h_desc.trace = nullptr;
    h_desc.done = nullptr;
    h_desc.lb = block_log2(kBlock);
    h_desc.pad0 = 0;
    h_desc.tmaps = nullptr;  // plain-load gather
    h_desc.wtab = nullptr;   // every block computes its weight spectrum
    na_twiddles(h_tw);
    const double cm = 0.5 * (kArea - 1);
    for (int m = 0; m < kArea; ++m)
        for (int n = 0; n < kArea; ++n)
            h_rho[m * kArea + n] = (float)std::pow((double)params->rho,
                                                   std::sqrt((m - cm) * (m - cm) + (n - cm) * (n - cm)));
    h_lost_off[0] = 0;
    h_lost_off[1] = bw * bh;

    // Tables and descriptor; the loss map starts at zero on every call.
    NA_CK(cudaMemcpyAsync(d_desc, &h_desc, sizeof(h_desc), cudaMemcpyHostToDevice, stream));
    NA_CK(cudaMemcpyAsync(d_tw, h_tw, sizeof(h_tw), cudaMemcpyHostToDevice, stream));
    NA_CK(cudaMemcpyAsync(d_rho, h_rho, sizeof(h_rho), cudaMemcpyHostToDevice, stream));
    NA_CK(cudaMemcpyAsync(d_lost_off, h_lost_off, sizeof(h_lost_off), cudaMemcpyHostToDevice,
                          stream));
    NA_CK(cudaMemsetAsync(d_lost, 0, (size_t)bw * bh, stream));
    NA_CK(launch_block_loss(d_desc, 1, H * bw, d_lost, nullptr, d_lost_off, stream));
    NA_CK(cudaMemcpyAsync(h_lost, d_lost, (size_t)bw * bh, cudaMemcpyDeviceToHost, stream));
    NA_CK(cudaStreamSynchronize(stream));

    int32_t n_groups = 0;
    rc = plan_order_core(bw, bh, h_lost, params->order, h_gob, h_group_ptr, h_ids, &n_groups,
                         h_plan_scratch);
    if (rc) return rc;
    const int n_items = h_group_ptr[n_groups];
    for (int i = 0; i < n_items; ++i) h_items[i] = make_int2(0, h_ids[i]);
    NA_CK(cudaMemcpyAsync(d_gob, h_gob, sizeof(int32_t) * bw * bh, cudaMemcpyHostToDevice,
                          stream));
    if (n_items > 0)
        NA_CK(cudaMemcpyAsync(d_items, h_items, sizeof(int2) * n_items, cudaMemcpyHostToDevice,
                              stream));
    // The static host staging is reused by the next call: wait for the
    // uploads before releasing it.
    NA_CK(cudaStreamSynchronize(stream));
    if (frame->out != frame->luma)
        NA_CK(cudaMemcpy2DAsync(frame->out, frame->stride, frame->luma, frame->stride, W, H,
                                cudaMemcpyDeviceToDevice, stream));
    const KParams kp{params->rho, params->delta, params->gamma, params->iters, nullptr,
                     block_log2(kBlock)};
    for (int g = 0; g < n_groups; ++g)
        NA_CK(launch_group(d_desc, d_items + h_group_ptr[g], h_group_ptr[g + 1] - h_group_ptr[g],
                           kp, d_rho, d_tw, FSE_PREC_FP32, stream));
    return FSE_OK;
}
