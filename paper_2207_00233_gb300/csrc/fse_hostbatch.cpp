// Batches of frames in host memory: fse_conceal_batch_host (synchronous) and
// fse_conceal_batch_host_async / fse_wait_batch.
//
// Each batch owns one of two slots of device frame copies.  Its frames are
// copied in on one stream and out on another, the extrapolation runs on the
// caller's stream between them, and the block-loss maps are built from the
// host masks while the copies run.  With two batches in flight the copies
// and the host planning of one overlap the extrapolation of the other.
#include <algorithm>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fse.h"
#include "fse_ctx.h"
#include "fse_internal.h"

using namespace fse;

namespace {

constexpr size_t kMaxResults = 64;  // finished batches kept for fse_wait_batch

// Device rows are padded to 16 bytes (TMA row pitch).
int device_pitch(const fse_frame &f) { return (f.width + 15) & ~15; }

int ensure_streams(fse_ctx *ctx) {
    if (!ctx->h2d) CK(cudaStreamCreateWithFlags(&ctx->h2d, cudaStreamNonBlocking));
    if (!ctx->d2h) CK(cudaStreamCreateWithFlags(&ctx->d2h, cudaStreamNonBlocking));
    for (HostBatch &b : ctx->hb) {
        if (!b.loaded) CK(cudaEventCreateWithFlags(&b.loaded, cudaEventDisableTiming));
        if (!b.launched) CK(cudaEventCreateWithFlags(&b.launched, cudaEventDisableTiming));
        if (!b.done) CK(cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming));
    }
    if (!ctx->hb_status.ptr) {
        const int rc = ctx->host_reserve(ctx->hb_status, 2 * sizeof(int));
        if (rc) return rc;
        std::memset(ctx->hb_status.ptr, 0, 2 * sizeof(int));
    }
    return FSE_OK;
}

// Waits until slot k's outputs are in host memory, frees the slot and
// returns the batch's status.
int finish_slot(fse_ctx *ctx, int k) {
    HostBatch &b = ctx->hb[k];
    int rc = FSE_OK;
    if (cudaEventSynchronize(b.done) != cudaSuccess) {
        cudaGetLastError();
        rc = FSE_ECUDA;
    } else if (static_cast<volatile int *>(ctx->hb_status.ptr)[k] != 0) {
        rc = FSE_ETIMEDOUT;
    }
    b.ticket = 0;
    return rc;
}

// Enqueues one batch of host frames (ctx->api_mu held).
int enqueue(fse_ctx *ctx, const fse_frame *frames, int n, const fse_params *params,
            cudaStream_t stream, uint64_t *ticket) {
    int rc = ensure_streams(ctx);
    if (rc) return rc;
    const int k = ctx->hb_next;
    HostBatch &b = ctx->hb[k];
    if (b.ticket) {
        // the older of two batches in flight: its slot is needed now, its
        // status is kept for fse_wait_batch
        const uint64_t t = b.ticket;
        ctx->hb_results[t] = finish_slot(ctx, k);
        while (ctx->hb_results.size() > kMaxResults) ctx->hb_results.erase(ctx->hb_results.begin());
    }
    std::vector<size_t> off(n + 1, 0);
    for (int i = 0; i < n; ++i)
        off[i + 1] = off[i] + (((size_t)frames[i].height * device_pitch(frames[i]) + 255) &
                               ~(size_t)255);
    rc = ctx->dev_reserve(b.d_luma, off[n]);
    if (!rc) rc = ctx->dev_reserve(b.d_mask, off[n]);
    if (!rc) rc = ctx->dev_reserve(b.d_out, off[n]);
    if (rc) return rc;

    // ---- copy in ----
    std::vector<fse_frame> dev(n);
    for (int i = 0; i < n; ++i) {
        const fse_frame &h = frames[i];
        const int pitch = device_pitch(h);
        uint8_t *dl = static_cast<uint8_t *>(b.d_luma.ptr) + off[i];
        uint8_t *dm = static_cast<uint8_t *>(b.d_mask.ptr) + off[i];
        uint8_t *dout = static_cast<uint8_t *>(b.d_out.ptr) + off[i];
        CK(cudaMemcpy2DAsync(dl, pitch, h.luma, h.stride, h.width, h.height,
                             cudaMemcpyHostToDevice, ctx->h2d));
        CK(cudaMemcpy2DAsync(dm, pitch, h.loss_mask, h.stride, h.width, h.height,
                             cudaMemcpyHostToDevice, ctx->h2d));
        dev[i] = fse_frame{dl, dout, dm, h.width, h.height, pitch};
    }
    CK(cudaEventRecord(b.loaded, ctx->h2d));

    // ---- plan from the host masks while the copies run, then launch ----
    std::vector<std::vector<uint8_t>> lost(n);
    ctx->pool.run(n, [&](int i) { lost[i] = host_block_loss(frames[i], params->block); });
    CK(cudaStreamWaitEvent(stream, b.loaded, 0));
    rc = run_batch(ctx, ctx->ws, dev.data(), n, params, stream, &lost);
    ctx->last_lost_blocks = ctx->ws.lost_blocks;
    ctx->last_groups = ctx->ws.groups;
    ctx->last_launches = ctx->ws.launches;
    ctx->last_executor = ctx->ws.executor;
    ctx->last_ctas = ctx->ws.ctas_per_sm;
    ctx->last_claim = ctx->ws.claim;
    if (rc) return rc;
    // the launch's status word, read back in stream order (the slot's
    // previous batch has finished, so its word is free)
    int *st = static_cast<int *>(ctx->hb_status.ptr) + k;
    *st = 0;
    if (ctx->ws.status_live) {
        CK(cudaMemcpyAsync(st, static_cast<int *>(ctx->ws.status.ptr) + 1, sizeof(int),
                           cudaMemcpyDeviceToHost, stream));
        ctx->ws.status_live = false;
    }
    CK(cudaEventRecord(b.launched, stream));

    // ---- copy out ----
    CK(cudaStreamWaitEvent(ctx->d2h, b.launched, 0));
    for (int i = 0; i < n; ++i) {
        const fse_frame &h = frames[i];
        CK(cudaMemcpy2DAsync(h.out, h.stride, dev[i].out, dev[i].stride, h.width, h.height,
                             cudaMemcpyDeviceToHost, ctx->d2h));
    }
    CK(cudaEventRecord(b.done, ctx->d2h));
    b.ticket = ctx->hb_ticket++;
    ctx->hb_next = k ^ 1;
    *ticket = b.ticket;
    return FSE_OK;
}

int check_batch(fse_ctx *ctx, const fse_frame *frames, int n, const fse_params *params) {
    if (!ctx || !frames || n <= 0) return FSE_EINVAL;
    int rc = check_params(params);
    for (int i = 0; i < n && !rc; ++i) rc = check_frame(frames[i]);
    return rc;
}

int wait_ticket(fse_ctx *ctx, uint64_t ticket) {
    for (int k = 0; k < 2; ++k)
        if (ticket != 0 && ctx->hb[k].ticket == ticket) return finish_slot(ctx, k);
    const auto it = ctx->hb_results.find(ticket);
    if (it == ctx->hb_results.end()) return FSE_ENOTFOUND;
    const int rc = it->second;
    ctx->hb_results.erase(it);
    return rc;
}

}  // namespace

void fse::release_host_batches(fse_ctx *ctx) {
    for (HostBatch &b : ctx->hb) {
        if (b.done) cudaEventSynchronize(b.done);
        ctx->dev_release(b.d_luma);
        ctx->dev_release(b.d_mask);
        ctx->dev_release(b.d_out);
        for (cudaEvent_t *e : {&b.loaded, &b.launched, &b.done}) {
            if (*e) cudaEventDestroy(*e);
            *e = nullptr;
        }
        b.ticket = 0;
    }
    for (cudaStream_t *s : {&ctx->h2d, &ctx->d2h}) {
        if (*s) cudaStreamDestroy(*s);
        *s = nullptr;
    }
    ctx->host_release(ctx->hb_status);
    ctx->hb_results.clear();
}

extern "C" int fse_conceal_batch_host(fse_ctx *ctx, const fse_frame *frames, int n,
                                      const fse_params *params, void *cuda_stream) {
    int rc = check_batch(ctx, frames, n, params);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    cudaSetDevice(ctx->device);
    uint64_t t = 0;
    rc = enqueue(ctx, frames, n, params, static_cast<cudaStream_t>(cuda_stream), &t);
    return rc ? rc : wait_ticket(ctx, t);
}

extern "C" int fse_conceal_batch_host_async(fse_ctx *ctx, const fse_frame *frames, int n,
                                            const fse_params *params, void *cuda_stream,
                                            uint64_t *ticket) {
    int rc = check_batch(ctx, frames, n, params);
    if (rc) return rc;
    if (!ticket) return FSE_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    cudaSetDevice(ctx->device);
    return enqueue(ctx, frames, n, params, static_cast<cudaStream_t>(cuda_stream), ticket);
}

extern "C" int fse_wait_batch(fse_ctx *ctx, uint64_t ticket) {
    if (!ctx) return FSE_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    cudaSetDevice(ctx->device);
    return wait_ticket(ctx, ticket);
}
