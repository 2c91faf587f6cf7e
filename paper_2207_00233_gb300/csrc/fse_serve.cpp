// Serving: fse_submit / fse_poll with continuous batching.
//
// Admission: a request is refused (FSE_EAGAIN) when the queue is full, or,
// with FSE_OPT_SERVE_LATENCY_MS, while the oldest queued request has waited
// longer than the latency budget; a batch is admitted onto a slot when its
// workspace fits the memory budget.
//
// A server thread owns `n_slots` CUDA streams, each with its own workspace.
// Pending requests (FIFO) are admitted into a batch on a free slot when the
// workspace for the batch fits the context's memory budget; requests that
// arrive while other batches are on the GPU go into the next free slot, so
// their work overlaps on the device with the batches already running.
// Frames travel through pinned staging buffers: the caller's host buffers
// are copied on the server thread, so the device copies are asynchronous.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fse.h"
#include "fse_ctx.h"
#include "fse_internal.h"

using namespace fse;

namespace {

bool same_params(const fse_params &a, const fse_params &b) {
    return a.block == b.block && a.border == b.border && a.dft == b.dft && a.iters == b.iters &&
           a.rho == b.rho && a.delta == b.delta && a.gamma == b.gamma && a.order == b.order &&
           a.precision == b.precision && a.executor == b.executor;
}

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// Device rows are padded to 16 bytes (TMA row pitch).
int device_pitch(const fse_frame &f) { return (f.width + 15) & ~15; }

size_t frame_bytes(const fse_frame &f) {
    return ((size_t)device_pitch(f) * f.height + 255) & ~(size_t)255;
}


// Page-locked host memory (allocated or registered by CUDA): copies to and
// from it run asynchronously without staging.
bool page_locked(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

void finish(fse_ctx *ctx, Slot &s, int status) {
    const auto now = Clock::now();
    const int nb = (int)s.reqs.size();
    for (Request *r : s.reqs) {
        if (status == FSE_OK && !r->direct_out) {
            const uint8_t *src = static_cast<const uint8_t *>(s.ws.io.ptr) + r->io_off;
            for (int y = 0; y < r->frame.height; ++y)
                std::memcpy(r->frame.out + (size_t)y * r->frame.stride,
                            src + (size_t)y * r->frame.width, r->frame.width);
        }
        r->stats.status = status;
        r->stats.batch_requests = nb;
        r->stats.latency_ms = ms_between(r->t_submit, now);
        r->done = true;
    }
    s.reqs.clear();
    s.busy = false;
    ctx->outstanding -= nb;
}

// Enqueue one batch on slot `s`.  Called without ctx->mu held.
int launch_batch(fse_ctx *ctx, Slot &s) {
    const int n = (int)s.reqs.size();
    Workspace &ws = s.ws;
    size_t total = 0;
    for (Request *r : s.reqs) {
        r->io_off = total;
        total += frame_bytes(r->frame);
    }
    int rc = ctx->dev_reserve(ws.d_luma, total);
    if (!rc) rc = ctx->dev_reserve(ws.d_mask, total);
    if (!rc) rc = ctx->dev_reserve(ws.d_out, total);
    if (!rc) rc = ctx->host_reserve(ws.io, 2 * total);
    if (rc) return rc;
    // The previous batch of this slot is complete (done_ev was observed), so
    // the pinned `io` buffer is free.
    uint8_t *io = static_cast<uint8_t *>(ws.io.ptr);
    std::vector<fse_frame> dev(n);
    std::vector<std::vector<uint8_t>> lost(n);
    for (Request *r : s.reqs) {
        r->direct_in = page_locked(r->frame.luma) && page_locked(r->frame.loss_mask);
        r->direct_out = page_locked(r->frame.out);
    }
    // staging copies of pageable frames and the block-loss maps, requests in
    // parallel on the context's worker threads
    ctx->pool.run(n, [&](int i) {
        Request *r = s.reqs[i];
        const fse_frame &h = r->frame;
        if (!r->direct_in) {
            uint8_t *pl = io + r->io_off;          // luma, later the result
            uint8_t *pm = io + total + r->io_off;  // mask
            for (int y = 0; y < h.height; ++y) {
                std::memcpy(pl + (size_t)y * h.width, h.luma + (size_t)y * h.stride, h.width);
                std::memcpy(pm + (size_t)y * h.width, h.loss_mask + (size_t)y * h.stride, h.width);
            }
        }
        lost[i] = host_block_loss(h, r->params.block);
        int cnt = 0;
        for (uint8_t v : lost[i]) cnt += v != 0;
        r->stats.lost_blocks = cnt;
    });
    for (int i = 0; i < n; ++i) {
        Request *r = s.reqs[i];
        const fse_frame &h = r->frame;
        const uint8_t *sl = r->direct_in ? h.luma : io + r->io_off;
        const uint8_t *sm = r->direct_in ? h.loss_mask : io + total + r->io_off;
        const size_t sp = r->direct_in ? (size_t)h.stride : (size_t)h.width;
        uint8_t *dl = static_cast<uint8_t *>(ws.d_luma.ptr) + r->io_off;
        uint8_t *dm = static_cast<uint8_t *>(ws.d_mask.ptr) + r->io_off;
        uint8_t *dout = static_cast<uint8_t *>(ws.d_out.ptr) + r->io_off;
        const int dp = device_pitch(h);
        if (cudaMemcpy2DAsync(dl, dp, sl, sp, h.width, h.height, cudaMemcpyHostToDevice,
                              s.stream) != cudaSuccess ||
            cudaMemcpy2DAsync(dm, dp, sm, sp, h.width, h.height, cudaMemcpyHostToDevice,
                              s.stream) != cudaSuccess) {
            cudaGetLastError();
            return FSE_ECUDA;
        }
        dev[i] = fse_frame{dl, dout, dm, h.width, h.height, dp};
    }
    const fse_params p = s.reqs[0]->params;
    rc = run_batch(ctx, ws, dev.data(), n, &p, s.stream, &lost);
    if (rc) return rc;
    for (int i = 0; i < n; ++i) {
        Request *r = s.reqs[i];
        s.reqs[i]->stats.groups = ws.groups;  // max over the batch
        uint8_t *dst = r->direct_out ? r->frame.out : io + r->io_off;
        const size_t dpitch = r->direct_out ? (size_t)r->frame.stride : (size_t)r->frame.width;
        if (cudaMemcpy2DAsync(dst, dpitch, dev[i].out, dev[i].stride, r->frame.width,
                              r->frame.height, cudaMemcpyDeviceToHost, s.stream) != cudaSuccess) {
            cudaGetLastError();
            return FSE_ECUDA;
        }
    }
    if (cudaEventRecord(s.done_ev, s.stream) != cudaSuccess) {
        cudaGetLastError();
        return FSE_ECUDA;
    }
    return FSE_OK;
}

void server_main(fse_ctx *ctx) {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(ctx->mu);
    while (true) {
        // 1. completions
        for (Slot &s : ctx->slots) {
            if (!s.busy) continue;
            const cudaError_t q = cudaEventQuery(s.done_ev);
            if (q == cudaErrorNotReady) continue;
            int st = FSE_OK;
            if (q != cudaSuccess) {
                cudaGetLastError();
                st = FSE_ECUDA;
            } else {
                st = read_status(ctx, s.ws, s.stream);
            }
            finish(ctx, s, st);
            ctx->done_cv.notify_all();
        }
        if (ctx->stop && ctx->outstanding == 0) break;

        // 2. admission: the head request opens a batch on a free slot; later
        // requests with the same parameters join while the batch fits.
        Slot *free_slot = nullptr;
        for (Slot &s : ctx->slots)
            if (!s.busy) {
                free_slot = &s;
                break;
            }
        bool any_busy = false;
        for (Slot &s : ctx->slots) any_busy |= s.busy;
        if (free_slot && !ctx->pending.empty() && !ctx->stop) {
            Slot &s = *free_slot;
            const fse_params head = ctx->pending.front()->params;
            for (auto it = ctx->pending.begin();
                 it != ctx->pending.end() && (int)s.reqs.size() < ctx->max_batch;) {
                if (same_params((*it)->params, head)) {
                    s.reqs.push_back(*it);
                    it = ctx->pending.erase(it);
                } else {
                    ++it;
                }
            }
            int others = 0;
            for (Slot &o : ctx->slots) others += (&o != &s) && o.busy;
            s.busy = true;
            const auto t0 = Clock::now();
            for (Request *r : s.reqs) {
                r->t_start = t0;
                r->stats.queue_ms = ms_between(r->t_submit, t0);
                r->stats.inflight = others;
            }
            lk.unlock();
            int rc = launch_batch(ctx, s);
            lk.lock();
            if (rc == FSE_ENOMEM) {
                bool others_busy = false;
                for (Slot &o : ctx->slots) others_busy |= (&o != &s) && o.busy;
                if (others_busy) {
                    // Memory is held by running batches: requeue at the front
                    // and retry after a completion.
                    for (auto it = s.reqs.rbegin(); it != s.reqs.rend(); ++it)
                        ctx->pending.push_front(*it);
                    s.reqs.clear();
                    s.busy = false;
                    release_workspace(ctx, s.ws);
                    ctx->cv.wait_for(lk, std::chrono::microseconds(200));
                    continue;
                }
                // Nothing runs: idle slots only cache buffers.  Free them and
                // retry the head request alone; if it still does not fit it
                // never will.
                for (Slot &o : ctx->slots) release_workspace(ctx, o.ws);
                for (size_t i = s.reqs.size(); i-- > 1;) ctx->pending.push_front(s.reqs[i]);
                s.reqs.resize(1);
                lk.unlock();
                rc = launch_batch(ctx, s);
                lk.lock();
            }
            if (rc) {
                cudaStreamSynchronize(s.stream);
                finish(ctx, s, rc);
                ctx->done_cv.notify_all();
            }
            continue;
        }
        if (any_busy)
            ctx->cv.wait_for(lk, std::chrono::microseconds(50));
        else
            ctx->cv.wait(lk, [&] { return ctx->stop || !ctx->pending.empty(); });
    }
}

int start_server(fse_ctx *ctx) {
    if (ctx->server_started) return FSE_OK;
    cudaSetDevice(ctx->device);
    ctx->slots.resize(ctx->n_slots);
    for (Slot &s : ctx->slots) {
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done_ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return FSE_ECUDA;
        }
    }
    ctx->stop = false;
    ctx->server = std::thread(server_main, ctx);
    ctx->server_started = true;
    return FSE_OK;
}

}  // namespace

void fse::stop_server(fse_ctx *ctx) {
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (!ctx->server_started) return;
        ctx->stop = true;
        // requests never admitted are failed
        for (Request *r : ctx->pending) {
            r->stats.status = FSE_EAGAIN;
            r->done = true;
            ctx->outstanding -= 1;
        }
        ctx->pending.clear();
    }
    ctx->cv.notify_all();
    ctx->server.join();
    for (Slot &s : ctx->slots) {
        cudaStreamSynchronize(s.stream);
        release_workspace(ctx, s.ws);
        ctx->host_release(s.ws.io);
        cudaStreamDestroy(s.stream);
        cudaEventDestroy(s.done_ev);
    }
    ctx->slots.clear();
    for (auto &kv : ctx->tickets) delete kv.second;
    ctx->tickets.clear();
    ctx->server_started = false;
}

extern "C" int fse_submit(fse_ctx *ctx, const fse_frame *frame, const fse_params *params,
                          uint64_t *ticket) {
    if (!ctx || !frame || !ticket) return FSE_EINVAL;
    int rc = check_params(params);
    if (rc) return rc;
    if (!frame->luma || !frame->out || !frame->loss_mask || frame->width <= 0 ||
        frame->height <= 0 || frame->stride < frame->width ||
        (long long)frame->height * frame->stride >= (1LL << 31))
        return FSE_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->stop) return FSE_EINVAL;
    if ((rc = start_server(ctx))) return rc;
    if (ctx->pending.size() >= ctx->max_pending) return FSE_EAGAIN;
    const auto now = Clock::now();
    // Latency-aware admission: the head of the queue is the oldest request
    // not yet on the GPU; its wait is the queueing delay a new request would
    // at least see.
    if (ctx->serve_latency_ms > 0.0 && !ctx->pending.empty() &&
        ms_between(ctx->pending.front()->t_submit, now) > ctx->serve_latency_ms)
        return FSE_EAGAIN;
    Request *r = new (std::nothrow) Request();
    if (!r) return FSE_ENOMEM;
    r->ticket = ctx->next_ticket++;
    r->frame = *frame;
    r->params = *params;
    r->t_submit = now;
    ctx->pending.push_back(r);
    ctx->tickets[r->ticket] = r;
    ctx->outstanding += 1;
    *ticket = r->ticket;
    ctx->cv.notify_all();
    return FSE_OK;
}

extern "C" int fse_poll(fse_ctx *ctx, uint64_t ticket, int *done, fse_stats *out) {
    if (!ctx || !done) return FSE_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return FSE_ENOTFOUND;
    Request *r = it->second;
    *done = r->done ? 1 : 0;
    if (r->done) {
        if (out) *out = r->stats;
        ctx->tickets.erase(it);
        delete r;
    }
    return FSE_OK;
}

extern "C" int fse_drain(fse_ctx *ctx, int timeout_ms) {
    if (!ctx) return FSE_EINVAL;
    std::unique_lock<std::mutex> lk(ctx->mu);
    auto pred = [&] { return ctx->outstanding == 0; };
    if (timeout_ms < 0) {
        ctx->done_cv.wait(lk, pred);
        return FSE_OK;
    }
    return ctx->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)
               ? FSE_OK
               : FSE_ETIMEDOUT;
}
