// Host runtime of the FSE library: context, device workspace, the batch
// executors (one launch per dependency level, or one persistent launch whose
// CTAs claim blocks in a list-schedule order and wait on completion flags),
// and the inspection entry point.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "../../include/fse.h"
#include "fse_ctx.h"
#include "fse_internal.h"

using namespace fse;

// ---------------------------------------------------------------------------
// TMA descriptors of a frame
// ---------------------------------------------------------------------------

// cuTensorMapEncodeTiled from the driver, through the runtime (no link
// dependency on libcuda); null when the driver does not provide it.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

// One 2-D map with a kStageCols x kStageRows box; samples outside the frame
// read as zero.
static bool encode_map(CUtensorMap *map, CUtensorMapDataType type, const void *base,
                       int width, int height, size_t row_bytes) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || !base || (reinterpret_cast<uintptr_t>(base) & 15) || (row_bytes & 15))
        return false;
    const cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)height};
    const cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)kStageCols, (cuuint32_t)kStageRows};
    const cuuint32_t elem[2] = {1, 1};
    return enc(map, type, 2, const_cast<void *>(base), dims, strides, box, elem,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The luma and loss-mask maps of a frame.  False when a buffer or the row
// pitch is not 16-byte aligned (the frame is then gathered with plain loads).
static bool encode_frame_maps(const FrameDesc &d, CUtensorMap *maps) {
    static_assert(sizeof(CUtensorMap) == kTensorMapBytes, "tensor map size");
    return encode_map(&maps[0], CU_TENSOR_MAP_DATA_TYPE_UINT8, d.luma, d.W, d.H,
                      (size_t)d.stride) &&
           encode_map(&maps[1], CU_TENSOR_MAP_DATA_TYPE_UINT8, d.mask, d.W, d.H,
                      (size_t)d.stride);
}

// ---------------------------------------------------------------------------
// Tables
// ---------------------------------------------------------------------------

// cos / sin of 2 pi t / 64.  Built from the first octant with the exact
// symmetries of the circle, so that entries for t and 64 - t are exact
// mirrors (a real input then has an exactly conjugate-symmetric spectrum)
// and the axis values are exact.
static void build_twiddles(float2 *tw) {
    double c[kDft], s[kDft];
    const double step = 2.0 * 3.14159265358979323846 / kDft;
    for (int t = 0; t <= kDft / 8; ++t) {
        c[t] = std::cos(step * t);
        s[t] = std::sin(step * t);
    }
    for (int t = kDft / 8 + 1; t <= kDft / 4; ++t) {  // reflect about 45 degrees
        c[t] = s[kDft / 4 - t];
        s[t] = c[kDft / 4 - t];
    }
    c[kDft / 4] = 0.0;
    s[kDft / 4] = 1.0;
    for (int t = kDft / 4 + 1; t <= kDft / 2; ++t) {  // second quadrant
        c[t] = -c[kDft / 2 - t];
        s[t] = s[kDft / 2 - t];
    }
    s[0] = 0.0;
    s[kDft / 2] = 0.0;
    for (int t = kDft / 2 + 1; t < kDft; ++t) {  // lower half: conjugates
        c[t] = c[kDft - t];
        s[t] = -s[kDft - t];
    }
    for (int t = 0; t < kDft; ++t) tw[t] = make_float2((float)c[t], (float)s[t]);
}

// Eq. (2) distance decay rho^dist over an M x M area, centre ((M-1)/2,
// (M-1)/2), stored in the top-left of a 48x48 table.
static void build_rho_table(float rho, int M, float *tab) {
    const double cm = 0.5 * (M - 1);
    for (int i = 0; i < kArea * kArea; ++i) tab[i] = 0.f;
    for (int m = 0; m < M; ++m)
        for (int n = 0; n < M; ++n) {
            const double dm = m - cm, dn = n - cm;
            tab[m * kArea + n] = (float)std::pow((double)rho, std::sqrt(dm * dm + dn * dn));
        }
}

// ---------------------------------------------------------------------------
// Device buffers with budget accounting
// ---------------------------------------------------------------------------

int fse_ctx::dev_reserve(DevBuf &b, size_t bytes) {
    if (bytes <= b.cap) return FSE_OK;
    std::lock_guard<std::mutex> lk(mem_mu);
    size_t want = std::max(bytes, b.cap + b.cap / 2);
    want = (want + 255) & ~(size_t)255;
    if (budget && used + want - b.cap > budget) {
        want = (bytes + 255) & ~(size_t)255;
        if (used + want - b.cap > budget) return FSE_ENOMEM;
    }
    void *p = nullptr;
    if (cudaMalloc(&p, want) != cudaSuccess) {
        cudaGetLastError();
        return FSE_ENOMEM;
    }
    if (b.ptr) {
        cudaFree(b.ptr);
        used -= b.cap;
    }
    b.ptr = p;
    b.cap = want;
    used += want;
    return FSE_OK;
}

void fse_ctx::dev_release(DevBuf &b) {
    std::lock_guard<std::mutex> lk(mem_mu);
    if (b.ptr) {
        cudaFree(b.ptr);
        used -= b.cap;
    }
    b.ptr = nullptr;
    b.cap = 0;
}

int fse_ctx::host_reserve(HostBuf &b, size_t bytes) {
    if (bytes <= b.cap) return FSE_OK;
    size_t want = std::max(bytes, b.cap + b.cap / 2);
    void *p = nullptr;
    if (cudaHostAlloc(&p, want, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return FSE_ENOMEM;
    }
    if (b.ptr) cudaFreeHost(b.ptr);
    b.ptr = p;
    b.cap = want;
    return FSE_OK;
}

void fse_ctx::host_release(HostBuf &b) {
    if (b.ptr) cudaFreeHost(b.ptr);
    b.ptr = nullptr;
    b.cap = 0;
}

const float *fse_ctx::rho_table(float rho, int block, int *rc) {
    // cache key: rho and the area size (block + 32)
    const float key = rho + 16.f * (float)block;
    {
        std::lock_guard<std::mutex> lk(mem_mu);
        for (auto &e : rho_tabs)
            if (e.first == key) return static_cast<const float *>(e.second.ptr);
    }
    DevBuf b;
    *rc = dev_reserve(b, kArea * kArea * sizeof(float));
    if (*rc) return nullptr;
    std::vector<float> tab(kArea * kArea);
    build_rho_table(rho, block + 2 * kBorder, tab.data());
    if (cudaMemcpy(b.ptr, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
        cudaGetLastError();
        dev_release(b);
        *rc = FSE_ECUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mem_mu);
    rho_tabs.emplace_back(key, b);
    return static_cast<const float *>(b.ptr);
}

const uint4 *fse_ctx::frag_table(int precision, int *rc) {
    *rc = FSE_OK;
    if (precision == FSE_PREC_FP32) return nullptr;
    if (precision < 0 || precision > 5) {
        *rc = FSE_EINVAL;
        return nullptr;
    }
    {
        std::lock_guard<std::mutex> lk(mem_mu);
        if (frags[precision].ptr) return static_cast<const uint4 *>(frags[precision].ptr);
    }
    DevBuf b;
    *rc = dev_reserve(b, frag_bytes(precision));
    if (*rc) return nullptr;
    if (launch_build_frags(precision, static_cast<const float2 *>(tw_dev.ptr),
                           static_cast<uint4 *>(b.ptr), nullptr) != cudaSuccess ||
        cudaStreamSynchronize(nullptr) != cudaSuccess) {
        cudaGetLastError();
        dev_release(b);
        *rc = FSE_ECUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mem_mu);
    if (frags[precision].ptr) {  // built concurrently by another thread
        DevBuf extra = b;
        used -= extra.cap;
        cudaFree(extra.ptr);
        return static_cast<const uint4 *>(frags[precision].ptr);
    }
    frags[precision] = b;
    return static_cast<const uint4 *>(b.ptr);
}

// ---------------------------------------------------------------------------
// Validation
// ---------------------------------------------------------------------------

int fse::check_params(const fse_params *p) {
    if (!p) return FSE_EINVAL;
    if (block_log2(p->block) < 0 || p->border != kBorder || p->dft != kDft) return FSE_EINVAL;
    if (p->iters < 0 || p->iters > FSE_MAX_ITERS) return FSE_EINVAL;
    if (!(p->rho > 0.f && p->rho < 1.f)) return FSE_EINVAL;
    if (!(p->delta >= 0.f && p->delta <= 1.f)) return FSE_EINVAL;
    if (!(p->gamma > 0.f && p->gamma < 2.f)) return FSE_EINVAL;
    if (p->order != FSE_ORDER_LINESCAN && p->order != FSE_ORDER_OPTIMIZED) return FSE_EINVAL;
    if (p->executor != FSE_EXEC_GROUPS && p->executor != FSE_EXEC_PERSISTENT) return FSE_EINVAL;
    if (!precision_supported(p->precision)) return FSE_EINVAL;
    return FSE_OK;
}

int fse::check_frame(const fse_frame &f) {
    if (!f.luma || !f.out || !f.loss_mask) return FSE_EINVAL;
    if (f.width <= 0 || f.height <= 0 || f.stride < f.width) return FSE_EINVAL;
    if ((long long)f.width * f.height > (1LL << 30)) return FSE_EINVAL;
    if ((long long)f.height * f.stride >= (1LL << 31)) return FSE_EINVAL;  // 32-bit offsets
    // the FP32 working frame's rows are padded to 32 samples; its offsets are 32-bit too
    if ((long long)f.height * ((f.width + 31) & ~31) >= (1LL << 31)) return FSE_EINVAL;
    return FSE_OK;
}

// ---------------------------------------------------------------------------
// Batch execution on device-resident frames
// ---------------------------------------------------------------------------


// Block-loss map of a host frame: a block is lost when any of its in-image
// samples is lost (as k_block_loss computes it on the device).
std::vector<uint8_t> fse::host_block_loss(const fse_frame &f, int B) {
    const int bh = (f.height + B - 1) / B, bw = (f.width + B - 1) / B;
    std::vector<uint8_t> lost((size_t)bh * bw, 0);
    // OR (any lost) and AND of "lost" (all lost) of the B rows of a block
    // row, 8 bytes at a time; then each block's B bytes of the results.
    const size_t words = ((size_t)f.width + 7) / 8;
    std::vector<uint64_t> acc(words), all(words);
    for (int by = 0; by < bh; ++by) {
        std::fill(acc.begin(), acc.end(), 0ull);
        std::fill(all.begin(), all.end(), ~0ull);
        const int y1 = std::min(f.height, (by + 1) * B);
        for (int y = by * B; y < y1; ++y) {
            const uint8_t *row = f.loss_mask + (size_t)y * f.stride;
            const size_t full = (size_t)f.width / 8;
            for (size_t k = 0; k < full; ++k) {
                uint64_t v;
                std::memcpy(&v, row + 8 * k, 8);
                acc[k] |= v;
                // bytes of v that are non-zero, as 0x01 per byte
                uint64_t nz = v | (v >> 4);
                nz |= nz >> 2;
                nz |= nz >> 1;
                all[k] &= nz & 0x0101010101010101ull;
            }
            uint8_t *a = reinterpret_cast<uint8_t *>(acc.data());
            uint8_t *l = reinterpret_cast<uint8_t *>(all.data());
            for (int x = (int)(full * 8); x < f.width; ++x) {
                a[x] |= row[x];
                l[x] &= row[x] != 0 ? 1 : 0;
            }
        }
        const uint8_t *a = reinterpret_cast<const uint8_t *>(acc.data());
        const uint8_t *l = reinterpret_cast<const uint8_t *>(all.data());
        for (int bx = 0; bx < bw; ++bx) {
            const int x0 = bx * B, x1 = std::min(f.width, x0 + B);
            uint8_t any = 0, every = 1;
            for (int x = x0; x < x1; ++x) {
                any |= a[x];
                every &= l[x] & 1;
            }
            lost[(size_t)by * bw + bx] = any ? (every ? kLostWhole : kLostPart) : 0;
        }
    }
    return lost;
}

// ---------------------------------------------------------------------------
// Host worker pool
// ---------------------------------------------------------------------------

fse::WorkerPool::~WorkerPool() {
    {
        std::lock_guard<std::mutex> lk(mu_);
        stop_ = true;
    }
    cv_.notify_all();
    for (auto &t : threads_) t.join();
}

void fse::WorkerPool::worker() {
    unsigned seen = 0;
    std::unique_lock<std::mutex> lk(mu_);
    for (;;) {
        cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
        if (!open_) continue;  // woke after the job was finished
        ++in_job_;
        const std::function<void(int)> *fn = fn_;
        const int n = n_;
        lk.unlock();
        for (int i = next_.fetch_add(1); i < n; i = next_.fetch_add(1)) {
            (*fn)(i);
            if (done_.fetch_add(1) + 1 == n) {
                std::lock_guard<std::mutex> g(mu_);
                done_cv_.notify_all();
            }
        }
        lk.lock();
        if (--in_job_ == 0) done_cv_.notify_all();
    }
}

void fse::WorkerPool::run(int n, const std::function<void(int)> &fn) {
    std::unique_lock<std::mutex> run_lk(run_mu_, std::try_to_lock);
    if (n <= 1 || !run_lk.owns_lock()) {
        for (int i = 0; i < n; ++i) fn(i);
        return;
    }
    if (!started_) {
        started_ = true;
        // a few threads: the jobs are short, and a thread that the OS is
        // slow to wake only loses its share
        const int hw = (int)std::thread::hardware_concurrency();
        const int nt = std::min(std::max(hw - 2, 0), 14);
        try {
            for (int t = 0; t < nt; ++t) threads_.emplace_back([this] { worker(); });
        } catch (...) {  // no threads: the calling thread does the work
        }
    }
    if (threads_.empty()) {
        for (int i = 0; i < n; ++i) fn(i);
        return;
    }
    {
        std::lock_guard<std::mutex> lk(mu_);
        fn_ = &fn;
        n_ = n;
        next_.store(0);
        done_.store(0);
        open_ = true;
        ++gen_;
    }
    cv_.notify_all();
    for (int i = next_.fetch_add(1); i < n; i = next_.fetch_add(1)) {
        fn(i);
        done_.fetch_add(1);
    }
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return done_.load() == n; });
    open_ = false;  // late workers skip this job
    done_cv_.wait(lk, [&] { return in_job_ == 0; });
    fn_ = nullptr;
}

// FSE_OPT_INPUTS_READY: statuses of earlier batches whose read-back has
// completed; FSE_ETIMEDOUT if one of them reported a failed device wait.
// `wait_slot` >= 0 also waits for that slot (before it is reused).
static int poll_status_ring(Workspace &ws, int wait_slot) {
    int rc = FSE_OK;
    for (int k = 0; k < 2; ++k) {
        if (!ws.st_pending[k]) continue;
        cudaError_t e = k == wait_slot ? cudaEventSynchronize(ws.st_ev[k])
                                       : cudaEventQuery(ws.st_ev[k]);
        if (e == cudaErrorNotReady) continue;
        ws.st_pending[k] = false;
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = FSE_ECUDA;
        } else if (static_cast<int *>(ws.st_host.ptr)[k] != 0 && rc == FSE_OK) {
            rc = FSE_ETIMEDOUT;
        }
    }
    return rc;
}

namespace {

// Host-side state of one batch, from the frames to the work items.
struct Batch {
    std::vector<FrameDesc> fd;
    std::vector<int> lost_off;  // first block of each frame in the flat maps
    int nblocks = 0;
    std::vector<uint8_t> lost;  // block-loss maps
    std::vector<int32_t> gob;   // group of each block (-1: nothing to do)
    std::vector<std::vector<int32_t>> gptr, ids;  // groups of each frame
    std::vector<FrameDepths> depths;
    int max_groups = 0, lost_blocks = 0;
    std::vector<int2> items;       // claim or launch order
    std::vector<int> level_start;  // launch boundaries (groups executor)
    bool map_kernel = false;       // the loss maps were built on the device
    std::vector<int32_t> wkey;     // W-table key of each block, -1: none
    std::vector<uint64_t> wptr;    // address of each block's W table, 0: none
    bool tables = false;           // some block uses a table
};

// Whether the blocks of a batch with these parameters can use W tables:
// 16x16 blocks, FP32 projection, tables on.
bool wtables_apply(const fse_ctx *ctx, const fse_params *p) {
    return ctx->w_tables != 0 && p->block == kBlock && p->precision == FSE_PREC_FP32;
}

// The W-table key of every lost block of frame i (see fse_internal.h):
// the block lost as a whole and inside the image, each of its 8 neighbours
// inside the image and not lost, or lost as a whole, or wholly outside.
void frame_wkeys(const FrameDesc &d, const uint8_t *lost, const int32_t *gob, int32_t *key) {
    static const int kDy[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
    static const int kDx[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
    auto inside = [&](int by, int bx) {
        return (by + 1) * kBlock <= d.H && (bx + 1) * kBlock <= d.W;
    };
    for (int by = 0; by < d.bh; ++by)
        for (int bx = 0; bx < d.bw; ++bx) {
            const int b = by * d.bw + bx;
            key[b] = -1;
            if (lost[b] != kLostWhole || !inside(by, bx)) continue;
            int k = 0;
            bool ok = true;
            for (int j = 0; j < 8 && ok; ++j) {
                const int ny = by + kDy[j], nx = bx + kDx[j];
                int st;
                if (ny < 0 || ny >= d.bh || nx < 0 || nx >= d.bw) {
                    st = 3;  // no sample of the cell is in the image
                } else if (!inside(ny, nx)) {
                    ok = false;  // a cell cut by the image border
                    break;
                } else {
                    const int c = ny * d.bw + nx;
                    if (lost[c] == 0) st = 0;
                    else if (lost[c] == kLostWhole) st = gob[c] < gob[b] ? 1 : 2;
                    else {
                        ok = false;  // partly lost: classes vary inside the cell
                        break;
                    }
                }
                k |= st << (2 * j);
            }
            if (ok) key[b] = k;
        }
}

// Frame descriptors and the workspace buffers they point into.
int setup_frames(fse_ctx *ctx, Workspace &ws, const fse_frame *frames, int n,
                 const fse_params *p, Batch &b) {
    b.fd.assign(n, FrameDesc{});
    b.lost_off.assign(n + 1, 0);
    size_t work_floats = 0;
    for (int i = 0; i < n; ++i) {
        FrameDesc &d = b.fd[i];
        d.luma = frames[i].luma;
        d.mask = frames[i].loss_mask;
        d.out = frames[i].out;
        d.H = frames[i].height;
        d.W = frames[i].width;
        d.stride = frames[i].stride;
        d.wstride = (d.W + 31) & ~31;
        d.lb = block_log2(p->block);
        d.pad0 = 0;
        d.tmaps = nullptr;
        d.bh = (d.H + p->block - 1) / p->block;
        d.bw = (d.W + p->block - 1) / p->block;
        b.lost_off[i + 1] = b.lost_off[i] + d.bh * d.bw;
        work_floats += (size_t)d.H * d.wstride;
    }
    b.nblocks = b.lost_off[n];
    int rc = ctx->dev_reserve(ws.frames, sizeof(FrameDesc) * n);
    if (!rc && ctx->keep_trace)
        rc = ctx->dev_reserve(ws.trace, sizeof(int16_t) * std::max<size_t>(
                                            (size_t)b.nblocks * std::max(p->iters, 1), 1));
    if (!rc) rc = ctx->dev_reserve(ws.work, sizeof(float) * work_floats);
    if (!rc) rc = ctx->dev_reserve(ws.lost, 2 * (size_t)b.nblocks);  // any lost, part intact
    if (!rc) rc = ctx->dev_reserve(ws.lost_off, sizeof(int) * (n + 1));
    if (!rc) rc = ctx->dev_reserve(ws.gob, sizeof(int32_t) * b.nblocks);
    if (!rc) rc = ctx->dev_reserve(ws.status, sizeof(int) * 4);
    if (rc) return rc;
    float *wp = static_cast<float *>(ws.work.ptr);
    for (int i = 0; i < n; ++i) {
        b.fd[i].work = wp;
        b.fd[i].gob = static_cast<int32_t *>(ws.gob.ptr) + b.lost_off[i];
        b.fd[i].trace = ctx->keep_trace ? static_cast<int16_t *>(ws.trace.ptr) +
                                              (size_t)b.lost_off[i] * p->iters
                                        : nullptr;
        wp += (size_t)b.fd[i].H * b.fd[i].wstride;
    }
    return FSE_OK;
}

// Block-loss maps: given by the caller (host frames), built on the host from
// a side-stream copy of the masks (FSE_OPT_INPUTS_READY), or built on the
// device in stream order and read back (which also reports a failed wait of
// the previous batch).
int block_loss_maps(fse_ctx *ctx, Workspace &ws, int n, const fse_params *p, cudaStream_t stream,
                    const std::vector<std::vector<uint8_t>> *host_lost, Batch &b) {
    const std::vector<FrameDesc> &fd = b.fd;
    b.lost.assign(b.nblocks, 0);
    int rc = FSE_OK;
    if (host_lost) {
        for (int i = 0; i < n; ++i)
            std::memcpy(b.lost.data() + b.lost_off[i], (*host_lost)[i].data(),
                        (size_t)fd[i].bh * fd[i].bw);
        return FSE_OK;
    }
    if (ctx->inputs_ready) {
        // The masks are complete now: copy them to the host on a side stream,
        // not behind the work queued on `stream` (typically the previous
        // batch, still running), and build the maps there, so that planning
        // overlaps that work.
        if ((rc = poll_status_ring(ws, -1))) return rc;
        if (!ws.side) CK(cudaStreamCreateWithFlags(&ws.side, cudaStreamNonBlocking));
        std::vector<size_t> moff(n + 1, 0);
        for (int i = 0; i < n; ++i) moff[i + 1] = moff[i] + (size_t)fd[i].W * fd[i].H;
        if ((rc = ctx->host_reserve(ws.mstage, std::max<size_t>(moff[n], 1)))) return rc;
        uint8_t *ms = static_cast<uint8_t *>(ws.mstage.ptr);
        for (int i = 0; i < n; ++i)
            CK(cudaMemcpy2DAsync(ms + moff[i], fd[i].W, fd[i].mask, fd[i].stride, fd[i].W,
                                 fd[i].H, cudaMemcpyDeviceToHost, ws.side));
        CK(cudaStreamSynchronize(ws.side));
        ctx->pool.run(n, [&](int i) {
            const fse_frame h{nullptr, nullptr, ms + moff[i], fd[i].W, fd[i].H, fd[i].W};
            const std::vector<uint8_t> m = host_block_loss(h, p->block);
            std::memcpy(b.lost.data() + b.lost_off[i], m.data(), m.size());
        });
        return FSE_OK;
    }
    int max_rows_x_bw = 0;
    for (int i = 0; i < n; ++i) max_rows_x_bw = std::max(max_rows_x_bw, fd[i].H * fd[i].bw);
    rc = ctx->host_reserve(ws.stage, sizeof(FrameDesc) * n + sizeof(int) * (n + 1) +
                                         2 * (size_t)b.nblocks + 64);
    if (rc) return rc;
    char *st = static_cast<char *>(ws.stage.ptr);
    std::memcpy(st, fd.data(), sizeof(FrameDesc) * n);
    std::memcpy(st + sizeof(FrameDesc) * n, b.lost_off.data(), sizeof(int) * (n + 1));
    CK(cudaMemcpyAsync(ws.frames.ptr, st, sizeof(FrameDesc) * n, cudaMemcpyHostToDevice,
                       stream));
    CK(cudaMemcpyAsync(ws.lost_off.ptr, st + sizeof(FrameDesc) * n, sizeof(int) * (n + 1),
                       cudaMemcpyHostToDevice, stream));
    CK(cudaMemsetAsync(ws.lost.ptr, 0, 2 * (size_t)b.nblocks, stream));
    uint8_t *d_lost = static_cast<uint8_t *>(ws.lost.ptr);
    CK(launch_block_loss(static_cast<FrameDesc *>(ws.frames.ptr), n, max_rows_x_bw, d_lost,
                         d_lost + b.nblocks, static_cast<int *>(ws.lost_off.ptr), stream));
    b.map_kernel = true;
    uint8_t *lost_stage =
        reinterpret_cast<uint8_t *>(st + sizeof(FrameDesc) * n + sizeof(int) * (n + 1));
    int *err_stage = reinterpret_cast<int *>(
        (reinterpret_cast<uintptr_t>(lost_stage + 2 * (size_t)b.nblocks) + 15) & ~(uintptr_t)15);
    CK(cudaMemcpyAsync(lost_stage, d_lost, 2 * (size_t)b.nblocks, cudaMemcpyDeviceToHost,
                       stream));
    if (ws.status_live)
        CK(cudaMemcpyAsync(err_stage, static_cast<int *>(ws.status.ptr) + 1, sizeof(int),
                           cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    for (int k = 0; k < b.nblocks; ++k)
        b.lost[k] = lost_stage[k] ? (lost_stage[b.nblocks + k] ? kLostPart : kLostWhole) : 0;
    if (ws.status_live && *err_stage) {
        ws.status_live = false;
        return FSE_ETIMEDOUT;
    }
    return FSE_OK;
}

// Processing order of every frame (Algorithm 1 or line scan) and the
// dependency depths of its lost blocks, frames on the worker pool.
int plan_frames(fse_ctx *ctx, int n, const fse_params *p, Batch &b) {
    b.gob.assign(b.nblocks, -1);
    b.gptr.assign(n, {});
    b.ids.assign(n, {});
    b.depths.assign(n, FrameDepths{});
    std::vector<int> plan_rc(n, FSE_OK);
    const int rad = kBorder >> block_log2(p->block);
    const bool keys = wtables_apply(ctx, p);
    b.wkey.assign(keys ? b.nblocks : 0, -1);
    ctx->pool.run(n, [&](int i) {
        const FrameDesc &d = b.fd[i];
        const int nb = d.bh * d.bw;
        std::vector<int32_t> gptr(nb + 1, 0), ids(nb, 0);
        int32_t ng = 0;
        plan_rc[i] = fse_plan_order(d.bw, d.bh, b.lost.data() + b.lost_off[i], p->order,
                                    b.gob.data() + b.lost_off[i], gptr.data(), ids.data(), &ng);
        if (plan_rc[i]) return;
        b.gptr[i].assign(gptr.begin(), gptr.begin() + ng + 1);
        b.ids[i].assign(ids.begin(), ids.begin() + gptr[ng]);
        FrameDepths &f = b.depths[i];
        f.bw = d.bw;
        f.bh = d.bh;
        f.gob = b.gob.data() + b.lost_off[i];
        f.ids = b.ids[i].data();
        f.n = (int)b.ids[i].size();
        frame_depths(f, rad);
        if (keys)
            frame_wkeys(d, b.lost.data() + b.lost_off[i], b.gob.data() + b.lost_off[i],
                        b.wkey.data() + b.lost_off[i]);
    });
    b.max_groups = b.lost_blocks = 0;
    for (int i = 0; i < n; ++i) {
        if (plan_rc[i]) return plan_rc[i];
        const int ng = (int)b.gptr[i].size() - 1;
        b.max_groups = std::max(b.max_groups, ng);
        b.lost_blocks += b.gptr[i][ng];
    }
    return FSE_OK;
}

// Work items: the persistent CTAs' claim order (delayed height order), one
// launch per dependency level, or one launch per plan group.
void claim_order(fse_ctx *ctx, int n, bool persistent, int grid, int claim, Batch &b) {
    b.items.clear();
    b.level_start.clear();
    if (persistent && claim == FSE_CLAIM_HEIGHT) {
        height_claims(b.depths, b.items);
    } else if (persistent && claim == FSE_CLAIM_LIST) {
        schedule_claims(b.depths, std::max(grid, 1), b.items);
    } else if (persistent) {
        delay_claims(b.depths, std::max(grid, 1), b.items,
                     [&](int m, const std::function<void(int)> &fn) { ctx->pool.run(m, fn); });
    } else if (ctx->group_launches) {
        // group g of every frame, frame by frame
        b.items.reserve(b.lost_blocks);
        b.level_start.assign(1, 0);
        for (int g = 0; g < b.max_groups; ++g) {
            for (int i = 0; i < n; ++i) {
                const auto &gp = b.gptr[i];
                if (g + 1 >= (int)gp.size()) continue;
                for (int j = gp[g]; j < gp[g + 1]; ++j) b.items.push_back(make_int2(i, b.ids[i][j]));
            }
            b.level_start.push_back((int)b.items.size());
        }
    } else {
        level_claims(b.depths, b.items, b.level_start);
    }
}

// W tables of the batch's blocks: keys not yet in the context's set for
// (rho, delta) get a table slot and are filled on `stream` (before the
// extrapolation); a key that finds no room within the memory budget stays
// without a table (its block computes W).  b.wptr gets each block's table.
int wtables_for_batch(fse_ctx *ctx, Workspace &ws, const fse_params *p, const float *rho_tab,
                      cudaStream_t stream, Batch &b) {
    b.wptr.assign(b.wkey.empty() ? 0 : b.nblocks, 0);
    b.tables = false;
    if (b.wkey.empty()) return FSE_OK;
    std::lock_guard<std::mutex> lk(ctx->wt_mu);
    fse_ctx::WTableSet *set = nullptr;
    for (auto &t : ctx->wsets)
        if (t.rho == p->rho && t.delta == p->delta && t.builder == ctx->w_tables) set = &t;
    if (!set) {
        ctx->wsets.emplace_back();
        set = &ctx->wsets.back();
        set->rho = p->rho;
        set->delta = p->delta;
        set->builder = ctx->w_tables;
        set->slot.assign(kWKeys, -1);
    }
    constexpr int kChunk = 32;  // tables per chunk
    std::vector<int32_t> new_keys;
    std::vector<uint64_t> new_dst;
    for (int k = 0; k < b.nblocks; ++k) {
        const int key = b.wkey[k];
        if (key < 0) continue;
        int s = set->slot[key];
        if (s < 0) {
            if (ctx->wchunks.empty() || ctx->wchunk_used == kChunk) {
                fse::DevBuf c;
                if (ctx->dev_reserve(c, (size_t)kChunk * kW4Bytes) != FSE_OK) {
                    b.wkey[k] = -1;  // over budget: this block computes W
                    continue;
                }
                ctx->wchunks.push_back(c);
                ctx->wchunk_used = 0;
            }
            s = (int)set->addr.size();
            set->addr.push_back(reinterpret_cast<uint64_t>(ctx->wchunks.back().ptr) +
                                (uint64_t)ctx->wchunk_used * kW4Bytes);
            ctx->wchunk_used += 1;
            set->slot[key] = s;
            new_keys.push_back(key);
            new_dst.push_back(set->addr[s]);
        }
        b.wptr[k] = set->addr[s];
        b.tables = true;
    }
    if (!b.tables) return FSE_OK;
    // tables filled by batches on other streams are complete before use
    if (ctx->wt_fill) CK(cudaStreamWaitEvent(stream, ctx->wt_fill, 0));
    if (!new_keys.empty()) {
        const size_t nk = new_keys.size();
        const size_t kbytes = (sizeof(int32_t) * nk + 15) & ~(size_t)15;
        int rc = ctx->host_reserve(ws.wstage, kbytes + sizeof(uint64_t) * nk);
        if (!rc) rc = ctx->dev_reserve(ws.wfill, kbytes + sizeof(uint64_t) * nk);
        if (rc) return rc;
        char *hs = static_cast<char *>(ws.wstage.ptr);
        std::memcpy(hs, new_keys.data(), sizeof(int32_t) * nk);
        std::memcpy(hs + kbytes, new_dst.data(), sizeof(uint64_t) * nk);
        CK(cudaMemcpyAsync(ws.wfill.ptr, hs, kbytes + sizeof(uint64_t) * nk,
                           cudaMemcpyHostToDevice, stream));
        const char *df = static_cast<const char *>(ws.wfill.ptr);
        const int32_t *dkeys = reinterpret_cast<const int32_t *>(df);
        const uint64_t *ddst = reinterpret_cast<const uint64_t *>(df + kbytes);
        if (ctx->w_tables == 2) {
            if (!ctx->wt_image.ptr) {
                std::vector<float> img;
                wtable_tc_image(img);
                if ((rc = ctx->dev_reserve(ctx->wt_image, sizeof(float) * img.size()))) return rc;
                CK(cudaMemcpy(ctx->wt_image.ptr, img.data(), sizeof(float) * img.size(),
                              cudaMemcpyHostToDevice));
            }
            int *status = static_cast<int *>(ws.status.ptr);
            CK(launch_wtables_tc(dkeys, ddst, (int)nk, p->delta, rho_tab,
                                 static_cast<const float4 *>(ctx->wt_image.ptr), status + 1,
                                 stream));
        } else {
            CK(launch_wtables(dkeys, ddst, (int)nk, p->delta, rho_tab,
                              static_cast<const float2 *>(ctx->tw_dev.ptr), stream));
        }
        if (!ctx->wt_fill) CK(cudaEventCreateWithFlags(&ctx->wt_fill, cudaEventDisableTiming));
        CK(cudaEventRecord(ctx->wt_fill, stream));
        // the staging is reused by the next fill of this workspace
        CK(cudaStreamSynchronize(stream));
    }
    return FSE_OK;
}

// Descriptors, group maps, items and TMA descriptors to the device through
// the pinned staging buffer; completion flags cleared.
int upload_batch(fse_ctx *ctx, Workspace &ws, int n, bool persistent, cudaStream_t stream,
                 Batch &b) {
    const size_t n_items = b.items.size();
    int rc = ctx->dev_reserve(ws.items, sizeof(int2) * std::max<size_t>(n_items, 1));
    if (!rc && persistent) rc = ctx->dev_reserve(ws.done, sizeof(uint32_t) * b.nblocks);
    if (!rc && b.tables) rc = ctx->dev_reserve(ws.wptr, sizeof(uint64_t) * b.nblocks);
    if (rc) return rc;
    for (int i = 0; i < n; ++i)
        b.fd[i].wtab = b.tables ? static_cast<const uint64_t *>(ws.wptr.ptr) + b.lost_off[i]
                                : nullptr;
    uint32_t *dp = static_cast<uint32_t *>(ws.done.ptr);
    for (int i = 0; i < n; ++i) b.fd[i].done = persistent ? dp + b.lost_off[i] : nullptr;
    // TMA descriptors (frames whose buffers allow it)
    std::vector<CUtensorMap> maps((size_t)kMapsPerFrame * n);
    if (n_items > 0) {
        if ((rc = ctx->dev_reserve(ws.tmaps, sizeof(CUtensorMap) * kMapsPerFrame * n))) return rc;
        const char *mp = static_cast<const char *>(ws.tmaps.ptr);
        for (int i = 0; i < n; ++i)
            if (encode_frame_maps(b.fd[i], &maps[(size_t)kMapsPerFrame * i]))
                b.fd[i].tmaps = mp + sizeof(CUtensorMap) * kMapsPerFrame * i;
    }
    const size_t stage_bytes = sizeof(FrameDesc) * n + sizeof(int32_t) * b.nblocks +
                               sizeof(int2) * n_items + sizeof(CUtensorMap) * maps.size() +
                               (b.tables ? sizeof(uint64_t) * b.nblocks : 0) + 256;
    if ((rc = ctx->host_reserve(ws.stage, stage_bytes))) return rc;
    char *st = static_cast<char *>(ws.stage.ptr);
    size_t off = 0;
    auto put = [&](void *dev, const void *src, size_t bytes) -> int {
        if (!bytes) return FSE_OK;
        std::memcpy(st + off, src, bytes);
        if (cudaMemcpyAsync(dev, st + off, bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess) {
            cudaGetLastError();
            return FSE_ECUDA;
        }
        off = (off + bytes + 15) & ~(size_t)15;
        return FSE_OK;
    };
    rc = put(ws.frames.ptr, b.fd.data(), sizeof(FrameDesc) * n);
    if (!rc) rc = put(ws.gob.ptr, b.gob.data(), sizeof(int32_t) * b.nblocks);
    if (!rc) rc = put(ws.items.ptr, b.items.data(), sizeof(int2) * n_items);
    if (!rc && n_items > 0) rc = put(ws.tmaps.ptr, maps.data(), sizeof(CUtensorMap) * maps.size());
    if (!rc && b.tables) rc = put(ws.wptr.ptr, b.wptr.data(), sizeof(uint64_t) * b.nblocks);
    if (rc) return rc;
    if (persistent && b.nblocks > 0)
        CK(cudaMemsetAsync(ws.done.ptr, 0, sizeof(uint32_t) * b.nblocks, stream));
    if (!ws.staged) CK(cudaEventCreateWithFlags(&ws.staged, cudaEventDisableTiming));
    CK(cudaEventRecord(ws.staged, stream));
    return FSE_OK;
}

}  // namespace

int fse::run_batch(fse_ctx *ctx, Workspace &ws, const fse_frame *frames, int n,
                   const fse_params *p, cudaStream_t stream,
                   const std::vector<std::vector<uint8_t>> *host_lost, int ctas_per_sm,
                   int claim) {
    int rc = FSE_OK;
    const float *rho_tab = ctx->rho_table(p->rho, p->block, &rc);
    if (!rho_tab) return rc;
    const uint4 *frags = ctx->frag_table(p->precision, &rc);
    if (rc) return rc;
    // The staging buffers of the previous batch on this workspace must have
    // been consumed before they are overwritten.
    if (ws.staged) CK(cudaEventSynchronize(ws.staged));
    // The previous batch's launches read the device workspace; it may have
    // been queued on another stream.
    if (ws.released) CK(cudaStreamWaitEvent(stream, ws.released, 0));

    Batch b;
    if ((rc = setup_frames(ctx, ws, frames, n, p, b))) return rc;
    if ((rc = block_loss_maps(ctx, ws, n, p, stream, host_lost, b))) return rc;
    if ((rc = plan_frames(ctx, n, p, b))) return rc;

    const bool persistent = p->executor == FSE_EXEC_PERSISTENT;
    int grid = 0, per_sm = 0;
    if (persistent) {
        per_sm = max_resident_ctas(p->iters);
        const int cap = ctas_per_sm >= 0 ? ctas_per_sm : ctx->persistent_ctas;
        if (cap > 0) per_sm = std::min(per_sm, cap);
        grid = std::min<int>(b.lost_blocks, ctx->num_sms * per_sm);
    }
    ws.executor = p->executor;
    ws.ctas_per_sm = per_sm;
    if (claim < 0) claim = ctx->claim_order;
    ws.claim = persistent ? claim : 0;
    claim_order(ctx, n, persistent, grid, claim, b);
    const size_t n_items = b.items.size();
    int stuck_item = -1;
    if (persistent && ctx->test_stuck_dep && n_items > 0) {
        stuck_item = (int)n_items - 1;  // waits on a flag nothing sets
        ctx->test_stuck_dep = false;
    }
    // status words of this batch (work counter, error) start at zero before
    // its first launch, the table fill included
    if (n_items > 0) CK(cudaMemsetAsync(ws.status.ptr, 0, sizeof(int) * 2, stream));
    if ((rc = wtables_for_batch(ctx, ws, p, rho_tab, stream, b))) return rc;
    if ((rc = upload_batch(ctx, ws, n, persistent, stream, b))) return rc;

    // ---- outputs start as copies of the inputs ----
    for (int i = 0; i < n; ++i) {
        if (frames[i].out != frames[i].luma)
            CK(cudaMemcpy2DAsync(frames[i].out, frames[i].stride, frames[i].luma,
                                 frames[i].stride, frames[i].width, frames[i].height,
                                 cudaMemcpyDeviceToDevice, stream));
    }

    // ---- extrapolation ----
    int *status = static_cast<int *>(ws.status.ptr);
    uint32_t *clocks = nullptr;
    ws.clock_items = 0;
    if (persistent && ctx->phase_clocks && n_items > 0 && p->precision == FSE_PREC_FP32) {
        if ((rc = ctx->dev_reserve(ws.clocks, sizeof(uint32_t) * kPhaseStamps * n_items)))
            return rc;
        clocks = static_cast<uint32_t *>(ws.clocks.ptr);
        ws.clock_items = (int)n_items;
    }
    const KParams kp{p->rho, p->delta, p->gamma, p->iters, frags, block_log2(p->block),
                     status + 1, clocks};
    const FrameDesc *fdev = static_cast<const FrameDesc *>(ws.frames.ptr);
    const float2 *tw_tab = static_cast<const float2 *>(ctx->tw_dev.ptr);
    int launches = b.map_kernel ? 1 : 0;
    ws.k_timed = false;
    if (n_items > 0) {
        const int kslot = ws.k_pos;
        if (!ws.k_begin[kslot]) {
            CK(cudaEventCreate(&ws.k_begin[kslot]));
            CK(cudaEventCreate(&ws.k_end[kslot]));
        }
        CK(cudaEventRecord(ws.k_begin[kslot], stream));
        if (persistent) {
            WorkQueue wq;
            wq.items = static_cast<const int2 *>(ws.items.ptr);
            wq.head = status;
            wq.error = status + 1;
            wq.n = (int)n_items;
            wq.stuck_item = stuck_item;
            wq.spin_limit = ctx->spin_limit;
            CK(launch_persistent(fdev, wq, kp, rho_tab, tw_tab, p->precision, grid, stream));
            launches += 1;
        } else {
            const int2 *idev = static_cast<const int2 *>(ws.items.ptr);
            for (size_t l = 0; l + 1 < b.level_start.size(); ++l) {
                const int cnt = b.level_start[l + 1] - b.level_start[l];
                CK(launch_group(fdev, idev + b.level_start[l], cnt, kp, rho_tab, tw_tab,
                                p->precision, stream));
                launches += 1;
            }
        }
        CK(cudaEventRecord(ws.k_end[kslot], stream));
        ws.k_timed = true;
        ws.k_pos = (kslot + 1) % Workspace::kKernelRing;
        ws.k_count = std::min(ws.k_count + 1, Workspace::kKernelRing);
        ws.status_live = true;
        if (ctx->inputs_ready && !host_lost) {
            // read the status back in stream order; a later call reports it
            if (!ws.st_host.ptr && (rc = ctx->host_reserve(ws.st_host, 2 * sizeof(int))))
                return rc;
            const int slot = ws.st_slot;
            if ((rc = poll_status_ring(ws, slot))) return rc;
            if (!ws.st_ev[slot])
                CK(cudaEventCreateWithFlags(&ws.st_ev[slot], cudaEventDisableTiming));
            CK(cudaMemcpyAsync(static_cast<int *>(ws.st_host.ptr) + slot, status + 1, sizeof(int),
                               cudaMemcpyDeviceToHost, stream));
            CK(cudaEventRecord(ws.st_ev[slot], stream));
            ws.st_pending[slot] = true;
            ws.st_slot = slot ^ 1;
            ws.status_live = false;
        }
    }

    if (!ws.released) CK(cudaEventCreateWithFlags(&ws.released, cudaEventDisableTiming));
    CK(cudaEventRecord(ws.released, stream));

    // ---- what the inspection entry points read back ----
    ws.lost_blocks = b.lost_blocks;
    ws.groups = b.max_groups;
    ws.launches = launches;
    ws.trace_ptr.assign(n, nullptr);
    ws.trace_len.assign(n, 0);
    ws.work_ptr.resize(n);
    ws.work_w.resize(n);
    ws.work_h.resize(n);
    ws.work_stride.resize(n);
    for (int i = 0; i < n; ++i) {
        const FrameDesc &d = b.fd[i];
        ws.trace_ptr[i] = d.trace;
        ws.trace_len[i] = d.trace ? (size_t)d.bh * d.bw * p->iters : 0;
        ws.work_ptr[i] = d.work;
        ws.work_w[i] = d.W;
        ws.work_h[i] = d.H;
        ws.work_stride[i] = d.wstride;
    }
    return FSE_OK;
}

// Reads the status word of the last launch (after a sync).
int fse::read_status(fse_ctx *, Workspace &ws, cudaStream_t stream) {
    if (!ws.status_live) return FSE_OK;
    int err = 0;
    if (cudaMemcpyAsync(&err, static_cast<int *>(ws.status.ptr) + 1, sizeof(int),
                        cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
        cudaGetLastError();
        return FSE_ECUDA;
    }
    ws.status_live = false;
    return err ? FSE_ETIMEDOUT : FSE_OK;
}

void fse::release_workspace(fse_ctx *ctx, Workspace &ws) {
    ctx->dev_release(ws.frames);
    ctx->dev_release(ws.work);
    ctx->dev_release(ws.lost);
    ctx->dev_release(ws.lost_off);
    ctx->dev_release(ws.gob);
    ctx->dev_release(ws.items);
    ctx->dev_release(ws.done);
    ctx->dev_release(ws.status);
    ctx->dev_release(ws.tmaps);
    ctx->dev_release(ws.trace);
    ctx->dev_release(ws.wptr);
    ctx->dev_release(ws.clocks);
    ws.clock_items = 0;
    ctx->dev_release(ws.wfill);
    ctx->host_release(ws.wstage);
    ctx->dev_release(ws.d_luma);
    ctx->dev_release(ws.d_mask);
    ctx->dev_release(ws.d_out);
    ctx->host_release(ws.stage);
    ctx->host_release(ws.mstage);
    ctx->host_release(ws.st_host);
    for (int k = 0; k < 2; ++k) {
        if (ws.st_ev[k]) cudaEventDestroy(ws.st_ev[k]);
        ws.st_ev[k] = nullptr;
        ws.st_pending[k] = false;
    }
    if (ws.side) cudaStreamDestroy(ws.side);
    ws.side = nullptr;
    if (ws.staged) cudaEventDestroy(ws.staged);
    if (ws.released) cudaEventDestroy(ws.released);
    ws.released = nullptr;
    for (int k = 0; k < Workspace::kKernelRing; ++k) {
        if (ws.k_begin[k]) cudaEventDestroy(ws.k_begin[k]);
        if (ws.k_end[k]) cudaEventDestroy(ws.k_end[k]);
        ws.k_begin[k] = ws.k_end[k] = nullptr;
    }
    ws.staged = nullptr;
    ws.k_pos = ws.k_count = 0;
    ws.k_timed = false;
}

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------

extern "C" int fse_ctx_create(fse_ctx **out, int device, size_t mem_budget) {
    if (!out) return FSE_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return FSE_ECUDA;
    }
    if (device < 0 || device >= ndev) return FSE_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return FSE_ECUDA;
    }
    fse_ctx *c = new (std::nothrow) fse_ctx();
    if (!c) return FSE_ENOMEM;
    c->device = device;
    c->budget = mem_budget;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return FSE_ECUDA;
    }
    c->num_sms = prop.multiProcessorCount;
    float2 tw[kDft];
    build_twiddles(tw);
    int rc = c->dev_reserve(c->tw_dev, sizeof(tw));
    if (rc || cudaMemcpy(c->tw_dev.ptr, tw, sizeof(tw), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        c->dev_release(c->tw_dev);
        delete c;
        return rc ? rc : FSE_ECUDA;
    }
    *out = c;
    return FSE_OK;
}

extern "C" void fse_ctx_destroy(fse_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    stop_server(ctx);
    cudaDeviceSynchronize();
    release_host_batches(ctx);
    release_workspace(ctx, ctx->ws);
    ctx->dev_release(ctx->tw_dev);
    for (auto &e : ctx->rho_tabs) ctx->dev_release(e.second);
    for (auto &f : ctx->frags) ctx->dev_release(f);
    for (auto &c : ctx->wchunks) ctx->dev_release(c);
    ctx->dev_release(ctx->wt_image);
    if (ctx->wt_fill) cudaEventDestroy(ctx->wt_fill);
    delete ctx;
}

// FSE_OPT_AUTOTUNE: the first batch of a shape runs every launch
// configuration with identical results and keeps the fastest (device time
// from the call's start to its last launch, planning included): one
// untimed pass first (first-use costs), then each candidate twice, the
// faster run counting.
static int autotuned_batch(fse_ctx *ctx, const fse_frame *frames, int n,
                           const fse_params *params, cudaStream_t stream) {
    long long samples = 0;
    for (int i = 0; i < n; ++i) samples += (long long)frames[i].width * frames[i].height;
    const std::vector<long long> key = {n, samples, params->iters, params->block, params->order,
                                        params->precision};
    fse_params p = *params;
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) {
        p.executor = it->second[0];
        return run_batch(ctx, ctx->ws, frames, n, &p, stream, nullptr, it->second[1],
                         it->second[2]);
    }
    // candidates (executor, CTAs per SM, claim order): the persistent launch
    // with every residency and claim order, and one launch per dependency
    // level
    std::vector<std::vector<int>> cand;
    const int max_per_sm = max_resident_ctas(params->iters);
    for (int c = max_per_sm; c >= 1; --c)
        for (int o : {FSE_CLAIM_DELAYED, FSE_CLAIM_HEIGHT, FSE_CLAIM_LIST})
            cand.push_back({FSE_EXEC_PERSISTENT, c, o});
    cand.push_back({FSE_EXEC_GROUPS, 0, 0});
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return FSE_ECUDA;
    }
    float best = -1.f;
    std::vector<int> choice = cand.front();
    int rc = FSE_OK;
    p.executor = cand.front()[0];  // untimed pass
    rc = run_batch(ctx, ctx->ws, frames, n, &p, stream, nullptr, cand.front()[1],
                   cand.front()[2]);
    if (!rc) rc = read_status(ctx, ctx->ws, stream);
    for (size_t k = 0; k < 2 * cand.size() && !rc; ++k) {
        const auto &c = cand[k % cand.size()];
        p.executor = c[0];
        if (cudaEventRecord(e0, stream) != cudaSuccess) {
            rc = FSE_ECUDA;
            break;
        }
        rc = run_batch(ctx, ctx->ws, frames, n, &p, stream, nullptr, c[1], c[2]);
        if (!rc) rc = read_status(ctx, ctx->ws, stream);
        if (rc) break;
        float ms = 0.f;
        if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = FSE_ECUDA;
            break;
        }
        if (best < 0.f || ms < best) {
            best = ms;
            choice = c;
        }
    }
    if (rc) cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    ctx->tuned[key] = choice;
    // the last candidate's output stands (every candidate gives the same
    // bytes); report the chosen configuration
    ctx->ws.executor = choice[0];
    ctx->ws.ctas_per_sm = choice[1];
    ctx->ws.claim = choice[2];
    return FSE_OK;
}

extern "C" int fse_conceal_batch(fse_ctx *ctx, const fse_frame *frames, int n,
                                 const fse_params *params, void *cuda_stream) {
    if (!ctx || !frames || n <= 0) return FSE_EINVAL;
    int rc = check_params(params);
    if (rc) return rc;
    for (int i = 0; i < n; ++i)
        if ((rc = check_frame(frames[i]))) return rc;
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    cudaSetDevice(ctx->device);
    if (ctx->autotune && params->executor == FSE_EXEC_PERSISTENT)
        rc = autotuned_batch(ctx, frames, n, params, static_cast<cudaStream_t>(cuda_stream));
    else
        rc = run_batch(ctx, ctx->ws, frames, n, params, static_cast<cudaStream_t>(cuda_stream),
                       nullptr);
    ctx->last_lost_blocks = ctx->ws.lost_blocks;
    ctx->last_groups = ctx->ws.groups;
    ctx->last_launches = ctx->ws.launches;
    ctx->last_executor = ctx->ws.executor;
    ctx->last_ctas = ctx->ws.ctas_per_sm;
    ctx->last_claim = ctx->ws.claim;
    return rc;
}

extern "C" int fse_extrapolate_areas(fse_ctx *ctx, const float *area_f,
                                     const uint8_t *area_cls, int n, const fse_params *params,
                                     float *g_out, int32_t *u_out, float *dc_out, float *r_out,
                                     void *cuda_stream) {
    if (!ctx || !area_f || !area_cls || !g_out || n < 0) return FSE_EINVAL;
    int rc = check_params(params);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    cudaSetDevice(ctx->device);
    const float *rho_tab = ctx->rho_table(params->rho, params->block, &rc);
    if (!rho_tab) return rc;
    const uint4 *frags = ctx->frag_table(params->precision, &rc);
    if (rc) return rc;
    const KParams kp{params->rho, params->delta, params->gamma, params->iters, frags,
                     block_log2(params->block), nullptr};  // areas are not staged
    CK(launch_areas(area_f, area_cls, n, kp, rho_tab,
                    static_cast<const float2 *>(ctx->tw_dev.ptr), params->precision, g_out,
                    u_out, dc_out, r_out, static_cast<cudaStream_t>(cuda_stream)));
    return FSE_OK;
}

extern "C" int fse_last_batch_info(fse_ctx *ctx, int *lost_blocks, int *groups, int *launches) {
    if (!ctx) return FSE_EINVAL;
    if (lost_blocks) *lost_blocks = ctx->last_lost_blocks;
    if (groups) *groups = ctx->last_groups;
    if (launches) *launches = ctx->last_launches;
    return FSE_OK;
}

extern "C" int fse_last_batch_config(fse_ctx *ctx, int *executor, int *ctas_per_sm) {
    if (!ctx) return FSE_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    if (executor) *executor = ctx->last_executor;
    if (ctas_per_sm) *ctas_per_sm = ctx->last_ctas;
    return FSE_OK;
}

extern "C" int fse_last_batch_shape(fse_ctx *ctx, int *executor, int *ctas_per_sm,
                                    int *claim_order, int *threads_per_cta,
                                    int *blocks_per_cta) {
    if (!ctx) return FSE_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    if (executor) *executor = ctx->last_executor;
    if (ctas_per_sm) *ctas_per_sm = ctx->last_ctas;
    if (claim_order) *claim_order = ctx->last_claim;
    if (threads_per_cta) *threads_per_cta = kThreads;
    if (blocks_per_cta) *blocks_per_cta = 1;
    return FSE_OK;
}

extern "C" int fse_last_phase_clocks(fse_ctx *ctx, void *cuda_stream, double *clk, int n,
                                     int *blocks) {
    if (!ctx || !clk || n <= 0) return FSE_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    Workspace &ws = ctx->ws;
    if (blocks) *blocks = ws.clock_items;
    for (int k = 0; k < n; ++k) clk[k] = 0.0;
    if (ws.clock_items <= 0) return FSE_OK;
    cudaSetDevice(ctx->device);
    std::vector<uint32_t> st((size_t)ws.clock_items * kPhaseStamps);
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    CK(cudaMemcpyAsync(st.data(), ws.clocks.ptr, sizeof(uint32_t) * st.size(),
                       cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    const int phases = std::min(n, kPhaseStamps - 1);
    for (int i = 0; i < ws.clock_items; ++i)
        for (int k = 0; k < phases; ++k)  // 32-bit SM clock: differences modulo 2^32
            clk[k] += (double)(uint32_t)(st[(size_t)i * kPhaseStamps + k + 1] -
                                         st[(size_t)i * kPhaseStamps + k]);
    for (int k = 0; k < phases; ++k) clk[k] /= ws.clock_items;
    return FSE_OK;
}

extern "C" int fse_last_kernel_ms(fse_ctx *ctx, float *ms) {
    if (!ctx || !ms) return FSE_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    *ms = 0.f;
    if (!ctx->ws.k_timed) return FSE_OK;
    cudaSetDevice(ctx->device);
    const Workspace &ws = ctx->ws;
    const int k = (ws.k_pos + Workspace::kKernelRing - 1) % Workspace::kKernelRing;
    CK(cudaEventSynchronize(ws.k_end[k]));
    CK(cudaEventElapsedTime(ms, ws.k_begin[k], ws.k_end[k]));
    return FSE_OK;
}

extern "C" int fse_recent_kernel_ms(fse_ctx *ctx, int n, float *ms, int *count) {
    if (!ctx || !ms || !count || n < 0) return FSE_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    cudaSetDevice(ctx->device);
    const Workspace &ws = ctx->ws;
    const int m = std::min(n, ws.k_count);
    for (int j = 0; j < m; ++j) {  // j = 0: the most recent batch
        const int k = (ws.k_pos + Workspace::kKernelRing - 1 - j) % Workspace::kKernelRing;
        CK(cudaEventSynchronize(ws.k_end[k]));
        CK(cudaEventElapsedTime(&ms[j], ws.k_begin[k], ws.k_end[k]));
    }
    *count = m;
    return FSE_OK;
}

extern "C" int fse_copy_work(fse_ctx *ctx, int frame, float *dst, int dst_stride,
                             void *cuda_stream) {
    if (!ctx || !dst) return FSE_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    const Workspace &ws = ctx->ws;
    if (frame < 0 || frame >= (int)ws.work_ptr.size()) return FSE_EINVAL;
    if (dst_stride < ws.work_w[frame]) return FSE_EINVAL;
    cudaSetDevice(ctx->device);
    CK(cudaMemcpy2DAsync(dst, sizeof(float) * dst_stride, ws.work_ptr[frame],
                         sizeof(float) * ws.work_stride[frame], sizeof(float) * ws.work_w[frame],
                         ws.work_h[frame], cudaMemcpyDeviceToDevice,
                         static_cast<cudaStream_t>(cuda_stream)));
    return FSE_OK;
}

extern "C" int fse_copy_trace(fse_ctx *ctx, int frame, int16_t *dst, void *cuda_stream) {
    if (!ctx || !dst) return FSE_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    const Workspace &ws = ctx->ws;
    if (frame < 0 || frame >= (int)ws.trace_ptr.size() || !ws.trace_ptr[frame])
        return FSE_EINVAL;
    cudaSetDevice(ctx->device);
    CK(cudaMemcpyAsync(dst, ws.trace_ptr[frame], sizeof(int16_t) * ws.trace_len[frame],
                       cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(cuda_stream)));
    return FSE_OK;
}

extern "C" int fse_weight_table(fse_ctx *ctx, int key, float rho, float delta, int builder,
                                void *dst, void *cuda_stream) {
    if (!ctx || !dst || key < 0 || key >= kWKeys || !(rho > 0.f && rho < 1.f) ||
        !(delta >= 0.f && delta <= 1.f) || (builder != 1 && builder != 2) ||
        (reinterpret_cast<uintptr_t>(dst) & 15))
        return FSE_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    cudaSetDevice(ctx->device);
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    int rc = FSE_OK;
    const float *rho_tab = ctx->rho_table(rho, kBlock, &rc);
    if (!rho_tab) return rc;
    Workspace &ws = ctx->ws;
    if ((rc = ctx->dev_reserve(ws.wfill, 32)) || (rc = ctx->dev_reserve(ws.status, sizeof(int) * 4)))
        return rc;
    const uint64_t d = reinterpret_cast<uint64_t>(dst);
    int32_t hk[4] = {key, 0, 0, 0};
    char *df = static_cast<char *>(ws.wfill.ptr);
    CK(cudaMemcpyAsync(df, hk, 16, cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(df + 16, &d, 8, cudaMemcpyHostToDevice, stream));
    int *status = static_cast<int *>(ws.status.ptr);
    CK(cudaMemsetAsync(status, 0, sizeof(int) * 2, stream));
    if (builder == 2) {
        if (!ctx->wt_image.ptr) {
            std::vector<float> img;
            wtable_tc_image(img);
            if ((rc = ctx->dev_reserve(ctx->wt_image, sizeof(float) * img.size()))) return rc;
            CK(cudaMemcpy(ctx->wt_image.ptr, img.data(), sizeof(float) * img.size(),
                          cudaMemcpyHostToDevice));
        }
        CK(launch_wtables_tc(reinterpret_cast<const int32_t *>(df),
                             reinterpret_cast<const uint64_t *>(df + 16), 1, delta, rho_tab,
                             static_cast<const float4 *>(ctx->wt_image.ptr), status + 1, stream));
    } else {
        CK(launch_wtables(reinterpret_cast<const int32_t *>(df),
                          reinterpret_cast<const uint64_t *>(df + 16), 1, delta, rho_tab,
                          static_cast<const float2 *>(ctx->tw_dev.ptr), stream));
    }
    int err = 0;
    CK(cudaMemcpyAsync(&err, status + 1, sizeof(int), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    return err ? FSE_ETIMEDOUT : FSE_OK;
}

extern "C" int fse_ctx_set_option(fse_ctx *ctx, int option, long long value) {
    if (!ctx) return FSE_EINVAL;
    switch (option) {
    case FSE_OPT_KEEP_TRACE:
        if (value != 0 && value != 1) return FSE_EINVAL;
        ctx->keep_trace = value != 0;
        return FSE_OK;
    case FSE_OPT_SPIN_LIMIT:
        if (value < 1) return FSE_EINVAL;
        ctx->spin_limit = value;
        return FSE_OK;
    case FSE_OPT_PERSISTENT_CTAS:
        if (value < 0 || value > 32) return FSE_EINVAL;
        ctx->persistent_ctas = (int)value;
        return FSE_OK;
    case FSE_OPT_SERVE_SLOTS: {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (value < 1 || value > 16 || ctx->server_started) return FSE_EINVAL;
        ctx->n_slots = (int)value;
        return FSE_OK;
    }
    case FSE_OPT_SERVE_MAX_BATCH: {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (value < 1 || value > 4096) return FSE_EINVAL;
        ctx->max_batch = (int)value;
        return FSE_OK;
    }
    case FSE_OPT_PHASE_CLOCKS: {
        if (value != 0 && value != 1) return FSE_EINVAL;
        std::lock_guard<std::mutex> lk(ctx->api_mu);
        ctx->phase_clocks = value != 0;
        return FSE_OK;
    }
    case FSE_OPT_CLAIM_ORDER: {
        if (value < FSE_CLAIM_DELAYED || value > FSE_CLAIM_LIST) return FSE_EINVAL;
        std::lock_guard<std::mutex> lk(ctx->api_mu);
        ctx->claim_order = (int)value;
        return FSE_OK;
    }
    case FSE_OPT_W_TABLES: {
        if (value < 0 || value > 2) return FSE_EINVAL;
        std::lock_guard<std::mutex> lk(ctx->wt_mu);
        ctx->w_tables = (int)value;
        return FSE_OK;
    }
    case FSE_OPT_SERVE_LATENCY_MS: {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (value < 0 || value > 3600000) return FSE_EINVAL;
        ctx->serve_latency_ms = (double)value;
        return FSE_OK;
    }
    case FSE_OPT_TEST_STUCK_DEP:
        if (value != 0 && value != 1) return FSE_EINVAL;
        ctx->test_stuck_dep = value != 0;
        return FSE_OK;
    case FSE_OPT_GROUP_LAUNCHES:
        if (value != 0 && value != 1) return FSE_EINVAL;
        ctx->group_launches = value != 0;
        return FSE_OK;
    case FSE_OPT_INPUTS_READY: {
        if (value != 0 && value != 1) return FSE_EINVAL;
        std::lock_guard<std::mutex> lk(ctx->api_mu);
        ctx->inputs_ready = value != 0;
        return FSE_OK;
    }
    case FSE_OPT_AUTOTUNE: {
        if (value != 0 && value != 1) return FSE_EINVAL;
        std::lock_guard<std::mutex> lk(ctx->api_mu);
        ctx->autotune = value != 0;
        return FSE_OK;
    }
    default:
        return FSE_EINVAL;
    }
}

extern "C" const char *fse_strerror(int status) {
    switch (status) {
    case FSE_OK: return "ok";
    case FSE_EINVAL: return "invalid argument";
    case FSE_ENOMEM: return "out of memory or over the context's memory budget";
    case FSE_EAGAIN: return "admission refused; retry later";
    case FSE_ETIMEDOUT: return "a bounded device wait timed out";
    case FSE_ECUDA: return "CUDA runtime error";
    case FSE_ENOTFOUND: return "unknown ticket";
    case FSE_ETOOBIG: return "frame larger than the fixed scratch of fse_conceal_frame_noalloc (1920 x 1088)";
    default: return "unknown status";
    }
}
