// server.cu — the repair server: continuous batching of single-program repair
// requests over a fixed device-memory budget.
//
// A dispatcher thread owns `n_slots` launch slots.  Each slot has its own
// stream, its own device buffers (packed arena, scratch, results) and pinned
// host staging buffers, all sized at creation so that the slots together stay
// within the memory budget; nothing is allocated while serving.  Whenever a
// slot is idle and requests are queued, the dispatcher admits queued requests
// in arrival order while their packed size fits the slot (and the in-flight
// cap allows), packs them, and enqueues copy-in, trace expansion, the
// persistent repair launch and copy-out on the slot's stream.  Requests that
// arrive while other launches run are admitted by the next free slot, so
// their work overlaps on the device with the launches already running.  A
// request's traces, clauses and masks stay in device memory for its whole
// repair loop, which runs inside one launch.  Completion is detected by an
// event query; latency is measured on the host from submit to harvest.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.cuh"

using namespace gr;

namespace {

using Clock = std::chrono::steady_clock;

// A request's program, deep-copied so the caller may free its buffers.
struct ProgramCopy {
    std::vector<gr_stmt> stmts;
    std::vector<uint8_t> level, pos;
    std::vector<uint16_t> guard;
    std::vector<uint32_t> weight, perm, coef, neg;
    std::vector<gr_loop> loops;
    gr_program p;
    void take(const gr_program &src) {
        const uint32_t n = slots_of(src);
        stmts.assign(src.stmts, src.stmts + src.n_stmts);
        if (src.slot_pos) pos.assign(src.slot_pos, src.slot_pos + n);
        level.assign(src.slot_level, src.slot_level + n);
        if (src.slot_guard) guard.assign(src.slot_guard, src.slot_guard + 2 * n);
        if (src.slot_weight) weight.assign(src.slot_weight, src.slot_weight + n);
        if (src.perm) perm.assign(src.perm, src.perm + src.perm_len);
        if (src.n_loops) loops.assign(src.loops, src.loops + src.n_loops);
        if (src.iter_coef) coef.assign(src.iter_coef, src.iter_coef + src.n_stmts);
        if (src.n_neg) neg.assign(src.neg, src.neg + src.n_neg);
        p = src;
        rebind();
    }
    void rebind() {
        p.stmts = stmts.data();
        p.slot_level = level.empty() ? nullptr : level.data();
        p.slot_guard = guard.empty() ? nullptr : guard.data();
        p.slot_weight = weight.empty() ? nullptr : weight.data();
        p.perm = perm.empty() ? nullptr : perm.data();
        p.loops = loops.empty() ? nullptr : loops.data();
        p.iter_coef = coef.empty() ? nullptr : coef.data();
        p.neg = neg.empty() ? nullptr : neg.data();
        p.slot_pos = pos.empty() ? nullptr : pos.data();
    }
};

// Programs with at least this many blocks whose blocks differ (see
// blocks_alike) take the wide lane (one CTA per block per check, the loop as
// a device-side graph); the rest share the persistent launch, one CTA per
// program, which checks a single block when all blocks are alike.
constexpr uint32_t kWideMinBlocks = 32;

struct Request {
    uint64_t ticket;
    ProgramCopy prog;
    gr_launch launch;
    int32_t mode;
    size_t arena_bytes, scratch_bytes;
    Clock::time_point t_submit;
    bool spread = false;  // set at submit: many blocks that differ
    bool wide() const { return spread; }
};

struct Done {
    gr_repair_result r;
    uint64_t latency_ns;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t event = nullptr;
    void *d_arena = nullptr, *d_scratch = nullptr;
    gr_repair_result *d_out = nullptr;
    uint8_t *h_arena = nullptr;
    gr_repair_result *h_out = nullptr;
    size_t arena_cap = 0, scratch_cap = 0;
    uint32_t out_cap = 0;
    bool busy = false;
    std::vector<uint64_t> tickets;
    std::vector<Clock::time_point> t_submit;
};

}  // namespace

struct gr_server {
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    gr_status error = GR_OK;
    char error_text[256] = {0};
    int device = 0;
    uint32_t expand_grid = 1216;  // CTAs of the trace expansion: 8 per SM
    gr_options opts;
    uint32_t max_inflight = 0, inflight = 0, max_batch = 0;
    uint64_t next_ticket = 1;
    std::deque<Request> pending;
    std::unordered_map<uint64_t, Done> done;
    std::vector<Slot> slots;
    uint64_t launches = 0;
};

namespace {

// Room a single program takes in a packed batch (arena, scratch), with the
// per-item alignment the packer uses.
void footprint(const gr_program &p, gr_launch l, size_t *arena, size_t *scratch) {
    const uint64_t segs = (uint64_t)exec_count(p) * l.blocks;
    const uint64_t tpad = (l.threads + 7u) & ~7u;
    *arena = sizeof(DevProg) + 4 + 8 + 64 + 16 * ((segs + kItemSegs - 1) / kItemSegs + exec_count(p) + 1) +
             16 * (size_t)check_items_of(p, l) + (size_t)perm_window_elems(p, l) * 2 + 32;
    *scratch = segs * 12 + 512 + align_to(segs * tpad, 128) * 2 + wide_bytes(1);
}

void set_error(gr_server *s, gr_status code, const char *what, cudaError_t e) {
    s->error = code;
    snprintf(s->error_text, sizeof(s->error_text), "%s: %s", what, cudaGetErrorString(e));
}

// Dispatch one batch on an idle slot.  Called with the lock held; releases it
// while packing and enqueueing.
bool dispatch(gr_server *s, Slot &sl, std::unique_lock<std::mutex> &lk) {
    std::vector<Request> batch;
    size_t a_sum = sizeof(ArenaHeader) + 256, s_sum = 1024;
    // one lane per launch: the queue's head decides, and the batch stops at
    // the first request of the other lane (arrival order is kept)
    const bool wide = !s->pending.empty() && s->pending.front().wide();
    while (!s->pending.empty() && s->inflight + batch.size() < s->max_inflight && batch.size() < s->max_batch) {
        const Request &r = s->pending.front();
        if (r.wide() != wide || (wide && batch.size() >= 65535u)) break;
        if (!batch.empty() && (a_sum + r.arena_bytes > sl.arena_cap || s_sum + r.scratch_bytes > sl.scratch_cap)) break;
        a_sum += r.arena_bytes;
        s_sum += r.scratch_bytes;
        batch.push_back(std::move(s->pending.front()));
        s->pending.pop_front();
    }
    if (batch.empty()) return false;
    const uint32_t n = (uint32_t)batch.size();
    s->inflight += n;
    sl.busy = true;
    lk.unlock();
    std::vector<gr_program> progs(n);
    std::vector<gr_launch> ls(n);
    std::vector<int32_t> modes(n);
    sl.tickets.resize(n);
    sl.t_submit.resize(n);
    for (uint32_t i = 0; i < n; ++i) {
        batch[i].prog.rebind();
        progs[i] = batch[i].prog.p;
        ls[i] = batch[i].launch;
        modes[i] = batch[i].mode;
        sl.tickets[i] = batch[i].ticket;
        sl.t_submit[i] = batch[i].t_submit;
    }
    const Layout L = layout_of(progs.data(), ls.data(), n);
    cudaError_t e = cudaSuccess;
    if (L.arena_bytes > sl.arena_cap || L.scratch_bytes > sl.scratch_cap || n > sl.out_cap) {
        // cannot happen for requests admitted by footprint(); fail loudly
        lk.lock();
        s->inflight -= n;
        sl.busy = false;
        s->error = GR_ECAPACITY;
        snprintf(s->error_text, sizeof(s->error_text), "internal: batch of %u does not fit its slot", n);
        return false;
    }
    pack_into(progs.data(), ls.data(), modes.data(), n, L, sl.h_arena);
    gr_status cs = GR_OK;
    uint32_t s_max = 1, b_max = 1;
    for (uint32_t i = 0; i < n; ++i) {
        s_max = std::max(s_max, exec_count(progs[i]));
        b_max = std::max(b_max, ls[i].blocks);
    }
    const ArenaHeader &hd = *reinterpret_cast<const ArenaHeader *>(sl.h_arena);
    const uint32_t skip = skip_bits(hd);
    const LaunchCfg cfg = wide ? wide_launch_cfg(n, s_max, &cs) : packed_launch_cfg(sl.d_arena, n, skip, (hd.flags & kArenaSimple) != 0, hd.scratch_rel_off, &cs);
    e = cudaMemcpyAsync(sl.d_arena, sl.h_arena, L.arena_bytes, cudaMemcpyHostToDevice, sl.stream);
    if (e == cudaSuccess) {
        if (wide) {
            e = cudaMemsetAsync(sl.d_scratch, 0, 256, sl.stream);
            if (e == cudaSuccess)
                e = launch_expand(sl.d_arena, sl.d_scratch, L.scratch_bytes, false, s->expand_grid, sl.stream);
            if (e == cudaSuccess)
                e = launch_wide(sl.d_arena, n, b_max, s->opts, sl.d_scratch, L.wide_off, sl.d_out, cfg.table_bytes,
                                sl.stream);
        } else {
            e = enqueue_repair(sl.d_arena, n, s->opts, sl.d_scratch, L.scratch_bytes, sl.d_out, cfg, s->expand_grid,
                               true, true, sl.stream);
        }
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sl.h_out, sl.d_out, (size_t)n * sizeof(gr_repair_result), cudaMemcpyDeviceToHost,
                            sl.stream);
    if (e == cudaSuccess) e = cudaEventRecord(sl.event, sl.stream);
    lk.lock();
    if (cs != GR_OK) e = cudaErrorUnknown;
    if (e != cudaSuccess) {
        set_error(s, GR_ECUDA, "server launch", e);
        return false;
    }
    ++s->launches;
    return true;
}

// Move the results of a finished slot into the done map.  Lock held.
void harvest(gr_server *s, Slot &sl) {
    const auto now = Clock::now();
    for (size_t i = 0; i < sl.tickets.size(); ++i) {
        Done d;
        d.r = sl.h_out[i];
        d.latency_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(now - sl.t_submit[i]).count();
        s->done.emplace(sl.tickets[i], d);
    }
    s->inflight -= (uint32_t)sl.tickets.size();
    sl.tickets.clear();
    sl.busy = false;
}

void worker_main(gr_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        bool progress = false;
        for (Slot &sl : s->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.event);
            if (q == cudaSuccess) {
                harvest(s, sl);
                progress = true;
            } else if (q != cudaErrorNotReady) {
                set_error(s, GR_ECUDA, "server completion", q);
                sl.busy = false;
            }
        }
        if (s->error == GR_OK) {
            for (Slot &sl : s->slots)
                if (!sl.busy && !s->pending.empty() && dispatch(s, sl, lk)) progress = true;
        }
        if (!progress) {
            const bool any_busy = std::any_of(s->slots.begin(), s->slots.end(), [](const Slot &x) { return x.busy; });
            // poll completions every 20 us while work runs; otherwise sleep until a submit
            s->cv.wait_for(lk, any_busy ? std::chrono::microseconds(20) : std::chrono::milliseconds(50));
        }
    }
}

void free_slot(Slot &sl) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.d_arena) cudaFree(sl.d_arena);
    if (sl.d_scratch) cudaFree(sl.d_scratch);
    if (sl.d_out) cudaFree(sl.d_out);
    if (sl.h_arena) cudaFreeHost(sl.h_arena);
    if (sl.h_out) cudaFreeHost(sl.h_out);
    if (sl.event) cudaEventDestroy(sl.event);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    sl = Slot();
}

}  // namespace

extern "C" {

gr_status gr_server_create(uint64_t mem_budget_bytes, uint32_t n_slots, uint32_t max_inflight,
                           const gr_options *opts, gr_server **out) {
    if (!out) return fail(GR_EINVAL, "out is NULL");
    if (n_slots < 1 || n_slots > 16) return fail(GR_EINVAL, "n_slots %u outside 1..16", n_slots);
    if (max_inflight < 1) return fail(GR_EINVAL, "max_inflight must be >= 1");
    gr_status vs = validate_opts(opts);
    if (vs != GR_OK) return vs;
    const uint64_t per_slot = mem_budget_bytes / n_slots;
    if (per_slot < (8ull << 20)) return fail(GR_EINVAL, "budget below 8 MiB per slot");
    gr_status cs = GR_OK;
    packed_launch_cfg(nullptr, 1, 0, false, 0, &cs);  // configures the kernels on this device
    if (cs != GR_OK) return cs;
    gr_server *s = new gr_server();
    cudaGetDevice(&s->device);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device) == cudaSuccess && sms > 0)
        s->expand_grid = 8u * (uint32_t)sms;
    s->opts = opts_or_default(opts);
    s->max_inflight = max_inflight;
    s->slots.resize(n_slots);
    // each slot: 1/16 of its share for the arena, 1/64 for results, the rest scratch
    const size_t arena_cap = align_to(per_slot / 16, 256);
    const uint32_t out_cap = (uint32_t)std::min<uint64_t>(per_slot / 64 / sizeof(gr_repair_result), 1u << 20);
    const size_t scratch_cap = align_to(per_slot - arena_cap - (size_t)out_cap * sizeof(gr_repair_result) - 4096, 256) - 256;
    s->max_batch = out_cap;
    for (Slot &sl : s->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.event, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_arena, arena_cap);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_scratch, scratch_cap);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_out, (size_t)out_cap * sizeof(gr_repair_result));
        if (e == cudaSuccess) e = cudaHostAlloc(&sl.h_arena, arena_cap, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaHostAlloc(&sl.h_out, (size_t)out_cap * sizeof(gr_repair_result), cudaHostAllocDefault);
        if (e != cudaSuccess) {
            for (Slot &x : s->slots) free_slot(x);
            delete s;
            return fail(e == cudaErrorMemoryAllocation ? GR_ENOMEM : GR_ECUDA, "server slot: %s", cudaGetErrorString(e));
        }
        sl.arena_cap = arena_cap;
        sl.scratch_cap = scratch_cap;
        sl.out_cap = out_cap;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return GR_OK;
}

gr_status gr_server_submit(gr_server *s, const gr_program *prog, gr_launch launch, int32_t mode, uint64_t *ticket) {
    if (!s || !ticket) return fail(GR_EINVAL, "NULL server or ticket");
    gr_status st = validate_one(prog, launch, 0);
    if (st != GR_OK) return st;
    if (mode != GR_MODE_REPAIR && mode != GR_MODE_REMOVE) return fail(GR_EINVAL, "bad mode %d", mode);
    Request r;
    r.prog.take(*prog);
    r.launch = launch;
    r.mode = mode;
    footprint(*prog, launch, &r.arena_bytes, &r.scratch_bytes);
    r.spread = launch.blocks >= kWideMinBlocks && !blocks_alike(*prog);
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->error != GR_OK) return fail(s->error, "server failed: %s", s->error_text);
        const Slot &sl = s->slots[0];
        if (r.arena_bytes + sizeof(ArenaHeader) + 256 > sl.arena_cap || r.scratch_bytes + 1024 > sl.scratch_cap)
            return fail(GR_ECAPACITY, "request needs more device memory than one slot of the budget");
        r.ticket = s->next_ticket++;
        r.t_submit = Clock::now();
        *ticket = r.ticket;
        s->pending.push_back(std::move(r));
    }
    s->cv.notify_one();
    return GR_OK;
}

gr_status gr_server_poll(gr_server *s, uint64_t ticket, gr_repair_result *out, uint64_t *latency_ns) {
    if (!s || !out) return fail(GR_EINVAL, "NULL server or out");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->done.find(ticket);
    if (it == s->done.end()) {
        if (s->error != GR_OK) return fail(s->error, "server failed: %s", s->error_text);
        if (ticket == 0 || ticket >= s->next_ticket) return fail(GR_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
        return GR_EBUSY;
    }
    *out = it->second.r;
    if (latency_ns) *latency_ns = it->second.latency_ns;
    s->done.erase(it);
    return GR_OK;
}

gr_status gr_server_drain(gr_server *s, uint32_t timeout_ms) {
    if (!s) return fail(GR_EINVAL, "NULL server");
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        {
            std::lock_guard<std::mutex> g(s->mu);
            if (s->error != GR_OK) return fail(s->error, "server failed: %s", s->error_text);
            if (s->pending.empty() && s->inflight == 0) return GR_OK;
        }
        if (Clock::now() >= deadline) return GR_EBUSY;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

gr_status gr_server_stats(gr_server *s, uint64_t *pending, uint64_t *inflight, uint64_t *launches) {
    if (!s) return fail(GR_EINVAL, "NULL server");
    std::lock_guard<std::mutex> g(s->mu);
    if (pending) *pending = s->pending.size();
    if (inflight) *inflight = s->inflight;
    if (launches) *launches = s->launches;
    return GR_OK;
}

gr_status gr_server_destroy(gr_server *s) {
    if (!s) return fail(GR_EINVAL, "NULL server");
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (Slot &sl : s->slots) free_slot(sl);
    delete s;
    return GR_OK;
}

}  // extern "C"
