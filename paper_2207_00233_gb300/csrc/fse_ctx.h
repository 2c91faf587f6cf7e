// Context, workspace and serving state of the FSE library (host side).
#pragma once

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <map>
#include <cstdint>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fse.h"

// Returns FSE_ECUDA from the calling function when a CUDA call fails (and
// clears the error).
#define CK(call)                     \
    do {                             \
        if ((call) != cudaSuccess) { \
            cudaGetLastError();      \
            return FSE_ECUDA;        \
        }                            \
    } while (0)

namespace fse {

struct DevBuf {
    void *ptr = nullptr;
    size_t cap = 0;
};
struct HostBuf {
    void *ptr = nullptr;
    size_t cap = 0;
};

// Everything one in-flight batch needs on the device.
struct Workspace {
    DevBuf frames, work, lost, lost_off, gob, items, done, status, trace;
    DevBuf wptr;                   // per block: address of its W table, or 0
    DevBuf clocks;                 // phase stamps of the last persistent batch
    int clock_items = 0;           // items stamped (0: none)
    DevBuf wfill;                  // keys and destinations of new W tables
    HostBuf wstage;                // pinned staging of wfill
    DevBuf tmaps;                  // TMA descriptors of the frames (2 per frame)
    DevBuf d_luma, d_mask, d_out;  // device copies of host frames
    HostBuf stage;                 // pinned staging for uploads / readback
    HostBuf io;                    // pinned staging of serving frames
    cudaEvent_t staged = nullptr;  // uploads from `stage` are complete
    cudaEvent_t released = nullptr;  // the last batch's launches are complete
    // events around the extrapolation launches of the last kKernelRing
    // batches (ring; k_pos is the next slot, k_count the recorded batches)
    static constexpr int kKernelRing = 64;
    cudaEvent_t k_begin[kKernelRing] = {}, k_end[kKernelRing] = {};
    int k_pos = 0, k_count = 0;
    bool k_timed = false;  // the last batch recorded a pair
    bool status_live = false;      // status word of the last launch pending
    int lost_blocks = 0, groups = 0, launches = 0;  // of the last batch
    int executor = 0, ctas_per_sm = 0, claim = 0;   // its launch configuration
    std::vector<int16_t *> trace_ptr;               // per frame of the last batch
    std::vector<size_t> trace_len;
    std::vector<float *> work_ptr;
    std::vector<int> work_w, work_h, work_stride;
    // FSE_OPT_INPUTS_READY: masks copied to the host on a side stream, and the
    // status words of batches still in flight read back in a ring of two
    cudaStream_t side = nullptr;
    HostBuf mstage;                 // pinned copies of the device masks
    HostBuf st_host;                // pinned status words (2)
    cudaEvent_t st_ev[2] = {nullptr, nullptr};
    bool st_pending[2] = {false, false};
    int st_slot = 0;
};

// One batch of host frames in flight (fse_conceal_batch_host_async): device
// copies of its frames, the events that order the copy streams around its
// launch, and its status word.
struct HostBatch {
    DevBuf d_luma, d_mask, d_out;
    cudaEvent_t loaded = nullptr;    // inputs on the device (copy-in stream)
    cudaEvent_t launched = nullptr;  // extrapolation complete (caller's stream)
    cudaEvent_t done = nullptr;      // outputs in host memory (copy-out stream)
    uint64_t ticket = 0;             // 0: free
};

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    fse_frame frame{};
    fse_params params{};
    Clock::time_point t_submit, t_start;
    fse_stats stats{};
    bool done = false;
    size_t io_off = 0;
    // page-locked caller buffers are copied directly, without staging
    bool direct_in = false, direct_out = false;
};

struct Slot {
    Workspace ws;
    cudaStream_t stream = nullptr;
    cudaEvent_t done_ev = nullptr;
    std::vector<Request *> reqs;
    bool busy = false;
};

int check_params(const fse_params *p);
int check_frame(const fse_frame &f);

// Host worker threads of a context, started on first use and kept until the
// context is destroyed (planning the frames of a batch in parallel without
// starting threads on every call).
class WorkerPool {
public:
    WorkerPool() = default;
    WorkerPool(const WorkerPool &) = delete;
    WorkerPool &operator=(const WorkerPool &) = delete;
    ~WorkerPool();
    // fn(i) for i in [0, n) on the workers and the calling thread; returns
    // when all are done.  Workers that have not woken up by then do not
    // join in (no wait on a descheduled thread).  A call that finds the pool
    // busy (another thread's batch) runs its jobs on the calling thread.
    void run(int n, const std::function<void(int)> &fn);

private:
    void worker();
    std::vector<std::thread> threads_;
    std::mutex run_mu_;  // one run at a time
    std::mutex mu_;      // guards the job description below
    std::condition_variable cv_, done_cv_;
    const std::function<void(int)> *fn_ = nullptr;
    int n_ = 0, in_job_ = 0;  // workers inside the current job
    unsigned gen_ = 0;
    bool open_ = false, stop_ = false, started_ = false;
    std::atomic<int> next_{0}, done_{0};
};

}  // namespace fse

struct fse_ctx {
    int device = 0;
    size_t budget = 0;  // 0 = unlimited
    size_t used = 0;    // bytes of device memory held
    int num_sms = 1;
    long long spin_limit = 1LL << 23;
    int persistent_ctas = 0;   // per SM; 0 = occupancy limit
    bool test_stuck_dep = false;
    bool keep_trace = false;
    bool group_launches = false;  // groups executor: one launch per plan group
    bool autotune = false;        // choose the launch configuration per shape
    bool inputs_ready = false;    // masks complete at the call (plan ahead)
    int claim_order = 0;          // FSE_OPT_CLAIM_ORDER of the persistent executor
    bool phase_clocks = false;    // FSE_OPT_PHASE_CLOCKS
    // autotuned (executor, CTAs per SM, claim order) per batch shape
    std::map<std::vector<long long>, std::vector<int>> tuned;
    int last_executor = 0, last_ctas = 0, last_claim = 0;  // configuration of the last batch

    // Weight-spectrum tables per (rho, delta, builder): slot[key] indexes addr, the
    // device address of the key's table (-1: none yet).  Tables live in
    // chunks that are never moved or freed before the context is destroyed,
    // so batches in flight on other streams keep valid addresses.  wt_fill
    // is recorded after every fill; a batch that uses tables waits for it.
    struct WTableSet {
        float rho = 0.f, delta = 0.f;
        int builder = 0;  // FSE_OPT_W_TABLES value that filled them
        std::vector<int32_t> slot;
        std::vector<uint64_t> addr;
    };
    std::vector<WTableSet> wsets;
    std::vector<fse::DevBuf> wchunks;
    int wchunk_used = 0;            // tables in the last chunk
    cudaEvent_t wt_fill = nullptr;
    std::mutex wt_mu;
    int w_tables = 2;               // FSE_OPT_W_TABLES: 0 off, 1 FP32, 2 tensor cores
    fse::DevBuf wt_image;           // constant operands of the tensor-core tables

    fse::DevBuf tw_dev;                                   // 64 twiddles
    std::vector<std::pair<float, fse::DevBuf>> rho_tabs;  // Eq. (2) decay per (rho, block)
    fse::DevBuf frags[6];                                 // per precision (tensor cores)
    fse::Workspace ws;  // synchronous API
    fse::WorkerPool pool;  // host planning threads
    std::mutex api_mu;  // one synchronous API call at a time
    std::mutex mem_mu;  // budget accounting and table cache

    int last_lost_blocks = 0, last_groups = 0, last_launches = 0;

    // batches of host frames (synchronous and asynchronous forms): two in
    // flight at most, copies on their own streams
    fse::HostBatch hb[2];
    int hb_next = 0;                   // slot of the next batch
    uint64_t hb_ticket = 1;            // next ticket
    cudaStream_t h2d = nullptr, d2h = nullptr;
    fse::HostBuf hb_status;            // pinned status words, one per slot
    std::map<uint64_t, int> hb_results;  // finished, not yet waited for

    // serving
    std::mutex mu;  // guards everything below and the budget accounting
    std::condition_variable cv, done_cv;
    std::thread server;
    bool server_started = false, stop = false;
    std::deque<fse::Request *> pending;
    std::unordered_map<uint64_t, fse::Request *> tickets;
    uint64_t next_ticket = 1;
    size_t max_pending = 1 << 16;
    double serve_latency_ms = 0.0;  // FSE_OPT_SERVE_LATENCY_MS (0: off)
    int n_slots = 4;
    int max_batch = 32;
    std::vector<fse::Slot> slots;
    int outstanding = 0;

    int dev_reserve(fse::DevBuf &b, size_t bytes);
    void dev_release(fse::DevBuf &b);
    int host_reserve(fse::HostBuf &b, size_t bytes);
    void host_release(fse::HostBuf &b);
    // Device table of rho^dist for this rho (created once, kept until
    // destroy); nullptr on failure.
    const float *rho_table(float rho, int block, int *rc);
    // Packed DFT operand fragments of the tensor-core projection for this
    // precision (built once); nullptr for FSE_PREC_FP32 or on failure.
    const uint4 *frag_table(int precision, int *rc);
};

namespace fse {
// Block-loss states: 0 = no lost sample, kLostPart = some in-image samples
// lost, kLostWhole = every in-image sample lost.
constexpr uint8_t kLostPart = 1, kLostWhole = 2;
// Block-loss map [bh][bw] of a frame in host memory (states above).
std::vector<uint8_t> host_block_loss(const fse_frame &f, int B);
// ctas_per_sm: persistent CTAs per SM for this batch (< 0: the context's
// FSE_OPT_PERSISTENT_CTAS setting).
// claim: the persistent executor's claim order (< 0: FSE_OPT_CLAIM_ORDER).
int run_batch(fse_ctx *ctx, Workspace &ws, const fse_frame *frames, int n,
              const fse_params *p, cudaStream_t stream,
              const std::vector<std::vector<uint8_t>> *host_lost, int ctas_per_sm = -1,
              int claim = -1);
int read_status(fse_ctx *ctx, Workspace &ws, cudaStream_t stream);
void release_workspace(fse_ctx *ctx, Workspace &ws);
void release_host_batches(fse_ctx *ctx);
void stop_server(fse_ctx *ctx);
}  // namespace fse
