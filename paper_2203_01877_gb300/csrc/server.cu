// tqp_server: continuous batching of submitted plans (serving).
//
// The paper executes one query at a time (Section 4.3).  Here a host
// dispatcher thread keeps up to max_inflight batches on the device: whenever
// a slot is free it takes the pending plans in arrival order (at most
// max_batch) and launches them as one batch on the slot's stream, with the
// slot's sub-arena as scratch.  A batch whose scratch does not fit the slot
// (the admission budget) is split; a plan that alone does not fit completes
// with TQP_ERR_OUT_OF_MEMORY.  Completion is seen by polling each slot's
// event, so new plans are admitted while earlier batches still run.  Each
// slot latches device errors in a word of its own, so a failing batch marks
// only its own requests.
//
// Admission by free HBM: a single plan whose scratch exceeds the slot's share
// of the budget is not refused while the device has room for it.  The
// dispatcher reads the free device memory (cudaMemGetInfo) and, if the plan's
// scratch fits with kHbmReserve to spare, gives the plan a scratch region of
// its own from the stream-ordered allocator (cudaMallocAsync on the slot's
// stream; freed on that stream when the batch retires), growing it while the
// plan still reports a shortfall and the device still has room.  Only then
// does the plan complete with TQP_ERR_OUT_OF_MEMORY.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "host.h"

namespace {

using Clock = std::chrono::steady_clock;

double since(Clock::time_point t0, Clock::time_point t) { return std::chrono::duration<double>(t - t0).count(); }

struct Req {
    tqp_plan plan;
    tqp_result res;
    uint64_t tag;
    Clock::time_point t_submit;
    Clock::time_point t_launch;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    tqp_ctx sub{};             // the context restricted to this slot's region
    std::vector<Req> reqs;     // the batch in flight
    bool busy = false;
    tqp_status launch_status = TQP_OK;
    void* overflow = nullptr;  // scratch of a plan larger than the share (freed at retire)
};

// Device memory kept free when a plan's scratch is taken from free HBM.
constexpr size_t kHbmReserve = size_t(1) << 30;

}  // namespace

struct tqp_server {
    tqp_ctx* ctx = nullptr;
    tqp_server_config cfg{};
    size_t top_before = 0, top_after = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work;  // submissions / stop
    std::condition_variable cv_done;  // completions
    std::deque<Req> pending;
    std::deque<tqp_completion> done;
    uint64_t submitted = 0, finished = 0;
    bool stop = false;
    std::thread th;
};

namespace tqp {

static void complete(tqp_server* s, std::vector<Req>& reqs, tqp_status st, Clock::time_point t) {
    std::lock_guard<std::mutex> lk(s->mu);
    for (const Req& r : reqs) {
        tqp_completion c;
        c.tag = r.tag;
        c.status = st;
        c.batch_size = static_cast<int32_t>(reqs.size());
        c.queue_s = since(r.t_submit, r.t_launch);
        c.latency_s = since(r.t_submit, t);
        s->done.push_back(c);
    }
    s->finished += reqs.size();
    reqs.clear();
    s->cv_done.notify_all();
}

// A finished batch: its status is the launch status or the slot's latched device error.
static void retire(tqp_server* s, Slot& sl) {
    const Clock::time_point t = Clock::now();
    tqp_status st = sl.launch_status;
    int err = 0;
    if (cudaMemcpy(&err, sl.sub.d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) st = TQP_ERR_CUDA;
    if (err != 0) {
        st = static_cast<tqp_status>(err);
        cudaMemset(sl.sub.d_err, 0, sizeof(int));
    }
    complete(s, sl.reqs, st, t);
    if (sl.overflow) {
        cudaFreeAsync(sl.overflow, sl.st);
        sl.overflow = nullptr;
    }
    sl.busy = false;
}

// One plan that does not fit the slot's share: run it in scratch taken from
// free HBM when the device has room (see the file comment).  Returns the
// plan's status (TQP_ERR_OUT_OF_MEMORY when the device has no room either).
static tqp_status launch_overflow(Slot& sl, const tqp_plan* plan, const tqp_result* res) {
    size_t need = std::max<size_t>(2 * sl.sub.used, size_t(16) << 20);
    for (int attempt = 0; attempt < 6; ++attempt) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return TQP_ERR_CUDA;
        if (need + kHbmReserve > free_b) break;
        void* buf = nullptr;
        if (cudaMallocAsync(&buf, need, sl.st) != cudaSuccess) {
            cudaGetLastError();
            break;
        }
        tqp_ctx ov = sl.sub;  // the slot's context over the new region, reporting into the slot's error word
        ov.arena = static_cast<unsigned char*>(buf);
        ov.arena_bytes = need;
        ov.owns_arena = false;
        ov.used = kPersistentBytes;
        ov.top = need;
        ov.live_regions = 0;
        const tqp_status st = run_plans_on(&ov, plan, res, 1, sl.st);
        if (st != TQP_ERR_OUT_OF_MEMORY) {
            sl.overflow = buf;
            return st;
        }
        cudaFreeAsync(buf, sl.st);
        need = std::max(2 * need, 2 * ov.used);
    }
    return fail(TQP_ERR_OUT_OF_MEMORY, "plan scratch exceeds the slot's share and the device's free memory");
}

// Launch the first plans of `take` that fit the slot; the rest go back to the
// front of the queue in order.
static void launch(tqp_server* s, Slot& sl, std::vector<Req>& take) {
    size_t n = take.size();
    std::vector<tqp_plan> plans;
    std::vector<tqp_result> res;
    tqp_status st = TQP_OK;
    while (true) {
        plans.clear();
        res.clear();
        for (size_t i = 0; i < n; ++i) {
            plans.push_back(take[i].plan);
            res.push_back(take[i].res);
        }
        st = run_plans_on(&sl.sub, plans.data(), res.data(), static_cast<int32_t>(n), sl.st);
        if (st == TQP_ERR_OUT_OF_MEMORY && n > 1) {
            n = (n + 1) / 2;  // nothing was launched yet: admit fewer plans
            continue;
        }
        if (st == TQP_ERR_OUT_OF_MEMORY) st = launch_overflow(sl, plans.data(), res.data());
        break;
    }
    if (n < take.size()) {
        std::lock_guard<std::mutex> lk(s->mu);
        for (size_t i = take.size(); i-- > n;) s->pending.push_front(take[i]);
    }
    take.resize(n);
    const Clock::time_point t = Clock::now();
    for (Req& r : take) r.t_launch = t;
    sl.reqs = take;
    sl.launch_status = st;
    cudaEventRecord(sl.ev, sl.st);
    sl.busy = true;
}

static void dispatch(tqp_server* s) {
    cudaSetDevice(s->ctx->device);
    while (true) {
        bool progress = false;
        for (Slot& sl : s->slots)
            if (sl.busy && cudaEventQuery(sl.ev) != cudaErrorNotReady) {
                retire(s, sl);
                progress = true;
            }
        for (Slot& sl : s->slots) {
            if (sl.busy) continue;
            std::vector<Req> take;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                while (!s->pending.empty() && static_cast<int32_t>(take.size()) < s->cfg.max_batch) {
                    take.push_back(s->pending.front());
                    s->pending.pop_front();
                }
            }
            if (take.empty()) break;
            launch(s, sl, take);
            progress = true;
        }
        bool any_busy = false;
        for (Slot& sl : s->slots) any_busy |= sl.busy;
        if (progress) continue;
        if (any_busy) {
            std::this_thread::yield();  // batches in flight: poll their events
            continue;
        }
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->stop && s->pending.empty()) break;
        s->cv_work.wait_for(lk, std::chrono::milliseconds(1), [s] { return s->stop || !s->pending.empty(); });
    }
}

}  // namespace tqp

using namespace tqp;

extern "C" {

tqp_status tqp_server_create(tqp_ctx* ctx, const tqp_server_config* cfg, tqp_server** out) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    if (!cfg || !out) return fail(TQP_ERR_INVALID_ARG, "cfg or out is NULL");
    *out = nullptr;
    if (cfg->max_batch < 1 || cfg->max_inflight < 1 || cfg->max_inflight > 8)
        return fail(TQP_ERR_INVALID_ARG, "max_batch >= 1 and 1 <= max_inflight <= 8 required");
    const size_t share = cfg->budget_bytes > 0 ? static_cast<size_t>(cfg->budget_bytes) / cfg->max_inflight : 0;
    if (share < (1u << 20)) return fail(TQP_ERR_INVALID_ARG, "budget_bytes leaves under 1 MiB per in-flight slot");
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(TQP_ERR_CUDA, "cannot select device %d", ctx->device);
    tqp_server* s = new (std::nothrow) tqp_server();
    if (!s) return fail(TQP_ERR_OUT_OF_MEMORY, "host allocation failed");
    s->ctx = ctx;
    s->cfg = *cfg;
    top_open(ctx);
    s->top_before = ctx->top;
    tqp_status st = TQP_OK;
    s->slots.resize(cfg->max_inflight);
    for (Slot& sl : s->slots) {
        unsigned char* base = static_cast<unsigned char*>(arena_alloc_top(ctx, share));
        if (!base) {
            st = arena_oom(ctx, static_cast<size_t>(cfg->budget_bytes));
            break;
        }
        sl.sub = *ctx;
        sl.sub.arena = base;
        sl.sub.arena_bytes = share;
        sl.sub.owns_arena = false;
        sl.sub.used = kPersistentBytes;
        sl.sub.top = share;
        sl.sub.live_regions = 0;
        sl.sub.d_err = reinterpret_cast<int*>(base);  // the slot's own error word
        if (cudaMemset(base, 0, kPersistentBytes) != cudaSuccess ||
            cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
            st = fail(TQP_ERR_CUDA, "cannot create the server's streams");
            break;
        }
    }
    s->top_after = ctx->top;
    if (st == TQP_OK && cudaDeviceSynchronize() != cudaSuccess) st = fail(TQP_ERR_CUDA, "device synchronize failed");
    if (st != TQP_OK) {
        for (Slot& sl : s->slots) {
            if (sl.ev) cudaEventDestroy(sl.ev);
            if (sl.st) cudaStreamDestroy(sl.st);
        }
        top_close(ctx, s->top_before, s->top_after);
        delete s;
        return st;
    }
    s->th = std::thread(dispatch, s);
    *out = s;
    return TQP_OK;
}

tqp_status tqp_server_submit(tqp_server* s, const tqp_plan* plan, const tqp_result* res, uint64_t tag) {
    if (!s || !plan || !res) return fail(TQP_ERR_INVALID_ARG, "server, plan or result is NULL");
    Req r;
    r.plan = *plan;
    r.res = *res;
    r.tag = tag;
    r.t_submit = Clock::now();
    r.t_launch = r.t_submit;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return fail(TQP_ERR_INVALID_ARG, "server is stopping");
        s->pending.push_back(r);
        ++s->submitted;
    }
    s->cv_work.notify_one();
    return TQP_OK;
}

int32_t tqp_server_poll(tqp_server* s, tqp_completion* out, int32_t max) {
    if (!s || !out) return -1;
    std::lock_guard<std::mutex> lk(s->mu);
    int32_t k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    return k;
}

tqp_status tqp_server_drain(tqp_server* s, double timeout_s) {
    clear_error();
    if (!s) return fail(TQP_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                        [s] { return s->finished == s->submitted; });
    return ok ? TQP_OK : fail(TQP_ERR_TIMEOUT, "requests still pending after %.3f s", timeout_s);
}

tqp_status tqp_server_destroy(tqp_server* s) {
    clear_error();
    if (!s) return TQP_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    {
        DeviceGuard g(s->ctx->device);
        for (Slot& sl : s->slots) {
            if (sl.st) cudaStreamSynchronize(sl.st);
            if (sl.ev) cudaEventDestroy(sl.ev);
            if (sl.st) cudaStreamDestroy(sl.st);
        }
        top_close(s->ctx, s->top_before, s->top_after);
    }
    delete s;
    return TQP_OK;
}

}  // extern "C"
