// capi.cu — host side of the C ABI (include/gpurepair.h): validation, packing
// of programs into the device arena, the per-device workspace, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <atomic>
#include <condition_variable>
#include <functional>
#include <thread>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <numeric>
#include <string>
#include <vector>

#include "engine.cuh"

using namespace gr;

namespace gr {

thread_local std::string g_last_error;

gr_status fail(gr_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

gr_status cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? GR_ENOMEM : GR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define GR_CUDA(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

uint32_t slot_weight_of(const gr_program &p, uint32_t k) {
    if (p.slot_weight) return p.slot_weight[k];
    return p.slot_level[k] == GR_GRID ? 13u : 1u;  // (gw*gb) + lw^0 with gw = 12
}

// Control runs through the statements; after the last statement of a loop
// body it jumps back to the body's first statement while iterations remain
// (the innermost loop ending there first, then its parents).
uint32_t exec_order(const gr_program &p, uint8_t *st, uint8_t *ctr, uint32_t cap) {
    uint32_t count[GR_MAX_LOOPS] = {0, 0, 0, 0};
    const uint32_t nl = std::min<uint32_t>(p.n_loops, GR_MAX_LOOPS);
    uint32_t n = 0, pc = 0;
    while (pc < p.n_stmts) {
        int inner = -1;
        for (uint32_t q = 0; q < nl; ++q)
            if (p.loops[q].lo <= pc && pc <= p.loops[q].hi && (inner < 0 || p.loops[q].lo > p.loops[inner].lo))
                inner = (int)q;
        if (n < cap) {
            st[n] = (uint8_t)pc;
            ctr[n] = (uint8_t)(inner < 0 ? 0u : count[inner]);
        }
        if (++n > cap) return n;
        uint32_t next = pc + 1;
        for (;;) {  // loops ending at pc, innermost (latest start) first
            int q = -1;
            for (uint32_t r = 0; r < nl; ++r)
                if (p.loops[r].hi == pc && (count[r] != 0xFFFFFFFFu) && (q < 0 || p.loops[r].lo > p.loops[q].lo))
                    q = (int)r;
            if (q < 0) break;
            if (count[q] + 1 < p.loops[q].trips) {
                ++count[q];
                next = p.loops[q].lo;
                break;
            }
            count[q] = 0xFFFFFFFFu;  // finished: skip it while looking for a parent
        }
        for (uint32_t r = 0; r < nl; ++r)
            if (count[r] == 0xFFFFFFFFu) count[r] = 0;
        pc = next;
    }
    return n;
}

// Blocks see one access pattern when, in each array, either no statement's
// address depends on the block (c = 0 mod M) or every statement is affine /
// strided with the same c mod M: block b then shifts all addresses of the
// array by the same c*b mod M, a bijection that keeps every equality between
// two addresses.  Guards depend on tid only, so block b's same-block
// witnesses are block 0's.
bool blocks_alike(const gr_program &p) {
    for (uint32_t sp = 0; sp < 2; ++sp) {
        const uint32_t M = sp == GR_SHARED ? p.m_shared : p.m_global;
        bool any = false, perm_any = false, all_zero = true, same = true;
        uint32_t c0 = 0;
        for (uint32_t s = 0; s < p.n_stmts; ++s) {
            const gr_stmt &st = p.stmts[s];
            if (st.space != sp) continue;
            const uint32_t cm = st.c % M;
            if (!any) c0 = cm;
            any = true;
            perm_any |= st.kind == GR_PERM;
            all_zero &= cm == 0;
            same &= cm == c0;
        }
        if (any && !all_zero && (perm_any || !same)) return false;
    }
    return true;
}

gr_status validate_loops(const gr_program *p, uint32_t idx) {
    if (p->n_loops == 0) return GR_OK;
    if (p->n_loops > GR_MAX_LOOPS) return fail(GR_EINVAL, "program %u: more than %d loops", idx, GR_MAX_LOOPS);
    if (!p->loops) return fail(GR_EINVAL, "program %u: loops is NULL", idx);
    for (uint32_t q = 0; q < p->n_loops; ++q) {
        const gr_loop &a = p->loops[q];
        if (a.lo < 1 || a.lo > a.hi || a.hi >= p->n_stmts || a.trips < 1)
            return fail(GR_EINVAL, "program %u loop %u: needs 1 <= lo <= hi < n_stmts and trips >= 1", idx, q);
        if (a.trips > GR_MAX_STMTS)
            return fail(GR_EINVAL, "program %u loop %u: more than %d trips", idx, q, GR_MAX_STMTS);
        for (uint32_t r = 0; r < q; ++r) {
            const gr_loop &b = p->loops[r];
            const bool disjoint = a.hi < b.lo || b.hi < a.lo;
            const bool nested = (a.lo < b.lo && b.hi <= a.hi) || (b.lo < a.lo && a.hi <= b.hi);
            if (!disjoint && !nested)
                return fail(GR_EINVAL, "program %u loops %u, %u: neither disjoint nor nested inside the first "
                                       "statement", idx, r, q);
        }
    }
    const uint32_t x = exec_count(*p);
    if (x > GR_MAX_STMTS)
        return fail(GR_EINVAL, "program %u: more than %d statement instances executed", idx, GR_MAX_STMTS);
    return GR_OK;
}

// The entries of its table a permutation statement reads, rotated to start
// at its offset b: when its address does not depend on the block (c = 0 mod
// M, or one block) the threads of a block read entries (b + t) mod M,
// t < T, else every entry.  The packed window holds `len` entries (the
// padded thread count, for the expansion kernel's padding lanes, or M) of
// which the first `need` (min(T, M), or M) must be distinct indices below M.
struct PermWindow {
    uint32_t len, need;
};

uint32_t t_pad_of(uint32_t T) { return (T + 7u) & ~7u; }

PermWindow perm_window(const gr_stmt &st, uint32_t M, const gr_launch &l) {
    if (l.blocks > 1 && st.c % M != 0) return {M, M};
    return {std::min(M, t_pad_of(l.threads)), std::min(M, l.threads)};
}

// The window of tbl from b (entries tbl[(b + k) mod M], k < w.len) into dst
// (may be NULL) as u16; true when its first w.need entries are below M and,
// unless range_only, distinct.
bool window_to_u16(const uint32_t *tbl, uint32_t M, uint32_t b, PermWindow w, uint16_t *dst, bool range_only) {
    const uint32_t n1 = std::min(w.len, M - b);  // [b, b + n1), then [0, len - n1)
    uint32_t mx = 0;
    // one streaming pass per run: the entries that must be in range, then the rest
    auto run = [&](const uint32_t *src, uint16_t *d, uint32_t cnt, uint32_t cnt_need) {
        if (d) {
            for (uint32_t k = 0; k < cnt_need; ++k) {
                const uint32_t v = src[k];
                mx = v > mx ? v : mx;
                d[k] = (uint16_t)v;
            }
            for (uint32_t k = cnt_need; k < cnt; ++k) d[k] = (uint16_t)src[k];
        } else {
            for (uint32_t k = 0; k < cnt_need; ++k) mx = src[k] > mx ? src[k] : mx;
        }
    };
    run(tbl + b, dst, n1, std::min(w.need, n1));
    run(tbl, dst ? dst + n1 : nullptr, w.len - n1, w.need > n1 ? w.need - n1 : 0u);
    if (mx >= M) return false;
    if (range_only) return true;
    uint64_t seen[GR_MAX_WORDS / 64];
    memset(seen, 0, ((M + 63u) / 64u) * 8u);
    for (uint32_t k = 0; k < w.need; ++k) {
        const uint32_t v = k < n1 ? tbl[b + k] : tbl[k - n1];
        const uint64_t bit = 1ull << (v & 63u);
        if (seen[v >> 6] & bit) return false;
        seen[v >> 6] |= bit;
    }
    return true;
}

// Visit each permutation instance of p in execution order: f(instance,
// statement, its gr_stmt, M, window start b, window).  Loop instances move b
// by their counter times the statement's loop coefficient.
template <typename F>
void for_each_perm_instance(const gr_program &P, const gr_launch &l, F f) {
    uint8_t st_of[GR_MAX_STMTS], ctr_of[GR_MAX_STMTS];
    uint32_t S = P.n_stmts;
    if (P.n_loops) {
        S = exec_order(P, st_of, ctr_of, GR_MAX_STMTS);
    } else {
        for (uint32_t s = 0; s < S; ++s) {
            st_of[s] = (uint8_t)s;
            ctr_of[s] = 0;
        }
    }
    for (uint32_t s = 0; s < S; ++s) {
        const gr_stmt &st = P.stmts[st_of[s]];
        if (st.kind != GR_PERM) continue;
        const uint32_t M = st.space == GR_SHARED ? P.m_shared : P.m_global;
        const uint64_t d = P.iter_coef ? (uint64_t)(P.iter_coef[st_of[s]] % M) * ctr_of[s] : 0u;
        const uint32_t b = (uint32_t)(((uint64_t)(st.b % M) + d) % M);
        f(s, (uint32_t)st_of[s], st, M, b, perm_window(st, M, l));
    }
}

uint64_t perm_window_elems(const gr_program &P, const gr_launch &l) {
    uint64_t e = 0;
    for_each_perm_instance(P, l, [&](uint32_t, uint32_t, const gr_stmt &, uint32_t, uint32_t, PermWindow w) {
        e += w.len;
    });
    return e;
}

// The lowest statement of p with a window that is not distinct indices
// below M, or ~0u.
uint32_t first_bad_window(const gr_program &P, const gr_launch &l) {
    uint32_t bad = 0xFFFFFFFFu;
    for_each_perm_instance(P, l, [&](uint32_t, uint32_t s, const gr_stmt &st, uint32_t M, uint32_t b, PermWindow w) {
        if (s < bad && !window_to_u16(P.perm + st.perm_off, M, b, w, nullptr, false)) bad = s;
    });
    return bad;
}

// tables == false leaves the permutation-window check to pack_into, which
// does it while converting the windows.
gr_status validate_one(const gr_program *p, gr_launch l, uint32_t idx, bool tables) {
    if (!p) return fail(GR_EINVAL, "program %u: NULL", idx);
    if (p->n_stmts < 1 || p->n_stmts > GR_MAX_STMTS)
        return fail(GR_EINVAL, "program %u: n_stmts %u outside 1..%d", idx, p->n_stmts, GR_MAX_STMTS);
    if (!p->stmts) return fail(GR_EINVAL, "program %u: stmts is NULL", idx);
    if (l.blocks < 1 || l.blocks > GR_MAX_BLOCKS)
        return fail(GR_EINVAL, "program %u: blocks %u outside 1..%d", idx, l.blocks, GR_MAX_BLOCKS);
    if (l.threads < 1 || l.threads > GR_MAX_THREADS)
        return fail(GR_EINVAL, "program %u: threads %u outside 1..%d", idx, l.threads, GR_MAX_THREADS);
    if (p->m_shared > GR_MAX_WORDS || p->m_global > GR_MAX_WORDS)
        return fail(GR_EINVAL, "program %u: array size above %d words", idx, GR_MAX_WORDS);
    if (p->n_slots > GR_MAX_SLOTS) return fail(GR_EINVAL, "program %u: more than %d slots", idx, GR_MAX_SLOTS);
    if (!p->slot_pos && p->n_slots && p->n_slots != p->n_stmts - 1)
        return fail(GR_EINVAL, "program %u: %u slots without slot_pos (one per place needs %u)", idx, p->n_slots,
                    p->n_stmts - 1);
    if (p->slot_pos && !p->n_slots) return fail(GR_EINVAL, "program %u: slot_pos needs n_slots", idx);
    const uint32_t n = slots_of(*p);
    for (uint32_t k = 0; p->slot_pos && k < n; ++k)
        if (p->slot_pos[k] + 1u >= p->n_stmts)
            return fail(GR_EINVAL, "program %u slot %u: place %u is not between two statements", idx, k, p->slot_pos[k]);
    for (uint32_t s = 0; s < p->n_stmts; ++s) {
        const gr_stmt &st = p->stmts[s];
        if (st.op > GR_W || st.space > GR_GLOBAL || st.kind > GR_PERM)
            return fail(GR_EINVAL, "program %u stmt %u: bad op/space/kind", idx, s);
        const uint32_t M = st.space == GR_SHARED ? p->m_shared : p->m_global;
        if (M == 0) return fail(GR_EINVAL, "program %u stmt %u: its array has 0 words", idx, s);
        if (st.guard_k == 0 ? st.guard_r != 0 : st.guard_r >= st.guard_k)
            return fail(GR_EINVAL, "program %u stmt %u: guard (%u, %u) needs r < k", idx, s, st.guard_k, st.guard_r);
        if (st.kind == GR_PERM) {
            if (!p->perm) return fail(GR_EINVAL, "program %u stmt %u: permutation map without perm", idx, s);
            if ((uint64_t)st.perm_off + M > p->perm_len)
                return fail(GR_EINVAL, "program %u stmt %u: perm_off + M beyond perm_len", idx, s);
        }
    }
    if (n > 0 && !p->slot_level) return fail(GR_EINVAL, "program %u: slot_level is NULL", idx);
    for (uint32_t k = 0; k < n; ++k) {
        if (p->slot_level[k] > GR_GRID) return fail(GR_EINVAL, "program %u slot %u: bad level", idx, k);
        if (p->slot_guard) {
            const uint32_t gk = p->slot_guard[2 * k], gr_ = p->slot_guard[2 * k + 1];
            if (gk == 0 ? gr_ != 0 : gr_ >= gk)
                return fail(GR_EINVAL, "program %u slot %u: guard (%u, %u) needs r < k", idx, k, gk, gr_);
        }
        if (p->slot_weight && (p->slot_weight[k] < 1 || p->slot_weight[k] > GR_MAX_WEIGHT))
            return fail(GR_EINVAL, "program %u slot %u: weight outside 1..2^24", idx, k);
    }
    if (n < 32 && (p->existing_mask >> n) != 0)
        return fail(GR_EINVAL, "program %u: existing_mask has bits beyond slot %u", idx, n);
    if (p->n_neg > GR_MAX_NEG) return fail(GR_EINVAL, "program %u: more than %d negative clauses", idx, GR_MAX_NEG);
    if (p->n_neg && !p->neg) return fail(GR_EINVAL, "program %u: neg is NULL", idx);
    for (uint32_t c = 0; c < p->n_neg; ++c)
        if (p->neg[c] == 0 || (n < 32 && (p->neg[c] >> n) != 0))
            return fail(GR_EINVAL, "program %u negative clause %u: empty or beyond slot %u", idx, c, n);
    gr_status ls = validate_loops(p, idx);
    if (ls != GR_OK || !tables) return ls;
    const uint32_t bad = first_bad_window(*p, l);
    if (bad != 0xFFFFFFFFu)
        return fail(GR_EINVAL, "program %u stmt %u: the permutation entries it reads are not distinct indices "
                               "below M", idx, bad);
    return GR_OK;
}

gr_status validate_opts(const gr_options *o) {
    if (o && o->max_iters > GR_MAX_ITERS) return fail(GR_EINVAL, "max_iters above %d", GR_MAX_ITERS);
    if (o && o->strategy > GR_STRATEGY_MHS) return fail(GR_EINVAL, "unknown strategy %u", o->strategy);
    if (o && o->deadline_us > GR_MAX_DEADLINE_US)
        return fail(GR_EINVAL, "deadline_us above %llu", (unsigned long long)GR_MAX_DEADLINE_US);
    return GR_OK;
}

gr_options opts_or_default(const gr_options *o) {
    gr_options d;
    memset(&d, 0, sizeof(d));
    d.grid_enabled = 1;
    d.max_iters = GR_MAX_ITERS;
    if (o) {
        d.grid_enabled = o->grid_enabled;
        d.strategy = o->strategy;
        d.max_iters = o->max_iters ? o->max_iters : GR_MAX_ITERS;
        d.deadline_us = o->deadline_us;
    }
    return d;
}

// ---------------------------------------------------------------------------
// Packing
// ---------------------------------------------------------------------------

size_t align_to(size_t x, size_t a) { return (x + a - 1) / a * a; }


// A program on the shared array alone whose blocks are alike (or that has
// one block) goes to the relation kernel; any other has one check item, or,
// when its blocks differ, one per range of blocks (up to kMaxCheckSplit), so
// that its same-block passes spread over several CTAs.
uint32_t check_items_of(const gr_program &p, const gr_launch &l) {
    bool global = false;
    for (uint32_t s = 0; s < p.n_stmts; ++s) global |= p.stmts[s].space == GR_GLOBAL;
    const bool alike = blocks_alike(p);
    if (!global && (alike || l.blocks == 1)) return 0;
    return alike ? 1u : std::min(l.blocks, kMaxCheckSplit);
}

template <typename F>
void parallel_over(uint32_t n, F body);

// One program's share of a packed batch (entries of each part).
struct ProgSizes {
    uint64_t items, citems, perm, segs, trace;
};
Layout layout_from(const ProgSizes *z, uint32_t n);

ProgSizes prog_sizes(const gr_program &p, const gr_launch &l) {
    ProgSizes z;
    const uint64_t x = exec_count(p), B = l.blocks;
    // room for either expansion item layout of the program (see pack_into)
    z.items = (x * B + kItemSegs - 1) / kItemSegs + x + 1;
    z.citems = check_items_of(p, l);
    z.perm = perm_window_elems(p, l);  // one window per instance (equal ones shared)
    z.segs = x * B;
    z.trace = align_to(x * B * t_pad_of(l.threads), 128);
    return z;
}

Layout layout_of(const gr_program *progs, const gr_launch *ls, uint32_t n) {
    std::vector<ProgSizes> z(n);
    parallel_over(n, [&](uint32_t lo, uint32_t hi) {
        for (uint32_t p = lo; p < hi; ++p) z[p] = prog_sizes(progs[p], ls[p]);
    });
    return layout_from(z.data(), n);
}

// The layout of n programs from their sizes: the prefix sums.
Layout layout_from(const ProgSizes *z, uint32_t n) {
    Layout L;
    L.progs_off = sizeof(ArenaHeader);
    L.order_off = align_to(L.progs_off + (size_t)n * sizeof(DevProg), 16);
    L.segbase_off = align_to(L.order_off + (size_t)n * 4, 16);
    L.items_off = align_to(L.segbase_off + (size_t)(n + 1) * 8, 16);
    L.n_items = 0;
    L.n_citems = 0;
    L.trace_elem.resize(n);
    L.segmask_elem.resize(n);
    L.perm_base.resize(n);
    uint64_t perm_total = 0, seg_total = 0, trace_total = 0;
    for (uint32_t p = 0; p < n; ++p) {
        L.n_items += z[p].items;
        L.n_citems += z[p].citems;
        L.perm_base[p] = perm_total;
        perm_total += z[p].perm;
        L.segmask_elem[p] = seg_total;
        seg_total += z[p].segs;
        L.trace_elem[p] = trace_total;
        trace_total += z[p].trace;
    }
    L.citems_off = align_to(L.items_off + (size_t)L.n_items * 16, 16);
    L.perm_off = align_to(L.citems_off + (size_t)L.n_citems * 16, 16);
    L.n_segments = seg_total;
    L.perm_elems = perm_total;
    L.arena_bytes = align_to(L.perm_off + perm_total * 2, 256);  // windows as u16 (M <= 65,536)
    L.segmask_off = 256;
    L.segrange_off = align_to(L.segmask_off + seg_total * 8, 256);
    L.trace_off = align_to(L.segrange_off + seg_total * 4, 256);
    L.wide_off = align_to(L.trace_off + trace_total * 2, 256);
    L.rel_off = align_to(L.wide_off + wide_bytes(n), 256);
    L.scratch_bytes = align_to(rel_flags_off(L.rel_off, n) + (size_t)n * 4u, 256);
    return L;
}

// A pool of host workers started once (up to 16, one per core) for the
// per-program host work of a batch: validation and packing.  Programs are
// independent, so each worker takes a contiguous range.  One batch uses the
// pool at a time; a call that finds it busy (another host thread) or that
// has few programs runs inline.
class HostPool {
  public:
    static HostPool &get() {
        static HostPool *pool = new HostPool();  // never destroyed: its workers never exit
        return *pool;
    }
    template <typename F>
    void run(uint32_t n, F &body) {
        // more parts than threads, taken in turn by the caller and the
        // workers, so that programs of uneven size balance
        const uint32_t threads = n_workers_ + 1;
        const uint32_t parts = n >= 32 ? std::min<uint32_t>(4u * threads, (n + 7) / 8) : 1u;
        std::unique_lock<std::mutex> busy(use_, std::try_to_lock);
        if (parts <= 1 || !busy.owns_lock()) {
            body(0u, n);
            return;
        }
        const uint32_t per = (n + parts - 1) / parts;
        {
            std::lock_guard<std::mutex> g(mu_);
            job_ = [&body](uint32_t lo, uint32_t hi) { body(lo, hi); };
            n_ = n;
            per_ = per;
            next_.store(0);
            parts_ = parts;
            pending_ = parts;
            gen_.fetch_add(1, std::memory_order_release);
        }
        cv_.notify_all();
        uint32_t mine = 0;
        for (;;) {
            const uint32_t k = next_.fetch_add(1);
            if (k >= parts) break;
            const uint32_t lo = k * per, hi = std::min(n, lo + per);
            if (lo < hi) body(lo, hi);
            ++mine;
        }
        std::unique_lock<std::mutex> g(mu_);
        pending_ -= mine;
        done_.wait(g, [&] { return pending_ == 0; });
    }

  private:
    HostPool() {
        const uint32_t hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        n_workers_ = hw - 1;
        for (uint32_t i = 0; i < n_workers_; ++i) threads_.emplace_back([this] { loop(); });
        for (auto &th : threads_) th.detach();  // live until the process exits
    }
    void loop() {
        uint64_t seen = 0;
        for (;;) {
            // spin a little before sleeping: the parallel steps of one batch
            // call follow each other within microseconds, and a woken thread
            // takes longer than that to start
            {
                const auto until = std::chrono::steady_clock::now() + std::chrono::microseconds(kSpinUs);
                for (uint32_t i = 1; gen_.load(std::memory_order_acquire) == seen; ++i)
                    if ((i & 255u) == 0 && std::chrono::steady_clock::now() > until) break;
            }
            std::unique_lock<std::mutex> g(mu_);
            cv_.wait(g, [&] { return gen_.load(std::memory_order_relaxed) != seen; });
            seen = gen_.load(std::memory_order_relaxed);
            for (;;) {
                const uint32_t k = next_.fetch_add(1);
                if (k >= parts_) break;
                const uint32_t lo = k * per_, hi = std::min(n_, lo + per_);
                g.unlock();
                if (lo < hi) job_(lo, hi);
                g.lock();
                if (--pending_ == 0) done_.notify_all();
            }
        }
    }
    std::mutex use_, mu_;
    std::condition_variable cv_, done_;
    std::vector<std::thread> threads_;
    std::function<void(uint32_t, uint32_t)> job_;
    std::atomic<uint32_t> next_{0};
    static constexpr int kSpinUs = 200;
    uint32_t n_workers_ = 0, n_ = 0, per_ = 0, parts_ = 0, pending_ = 0;
    std::atomic<uint64_t> gen_{0};  // written under mu_; read without it while spinning
};

// Run body(lo, hi) over [0, n) on the host pool (programs are independent).
template <typename F>
void parallel_over(uint32_t n, F body) {
    HostPool::get().run(n, body);
}

gr_status validate_all(const gr_program *progs, const gr_launch *ls, uint32_t n, bool tables = true,
                       ProgSizes *sizes = nullptr) {
    if (n == 0) return fail(GR_EINVAL, "no programs");
    if (!progs || !ls) return fail(GR_EINVAL, "progs or launches is NULL");
    // the first invalid program (lowest index) is reported, as in a serial scan
    std::atomic<uint32_t> first_bad{n};
    std::mutex mu;
    std::string msg;
    gr_status code = GR_OK;
    parallel_over(n, [&](uint32_t lo, uint32_t hi) {
        for (uint32_t p = lo; p < hi && p < first_bad.load(); ++p) {
            gr_status s = validate_one(&progs[p], ls[p], p, tables);
            if (s == GR_OK && sizes) sizes[p] = prog_sizes(progs[p], ls[p]);
            if (s != GR_OK) {
                std::lock_guard<std::mutex> g(mu);
                if (p < first_bad.load()) {
                    first_bad.store(p);
                    msg = g_last_error;
                    code = s;
                }
                return;
            }
        }
    });
    if (code != GR_OK) g_last_error = msg;
    return code;
}

// Whether no two threads of a block share the statement's address: an
// affine or strided map a*tid + (the block's offset) mod M is injective on
// tid in [0, T) iff T <= M / gcd(a, M); a permutation map is iff T <= M.
// (A guard only removes threads.)  A false "no" costs only speed: the
// relation kernel then installs that row with compare-and-swap.
bool injective_on_threads(const gr_stmt &st, uint32_t M, uint32_t T) {
    if (T <= 1) return true;
    if (st.kind == GR_PERM) return T <= M;
    uint32_t a = st.a % M, b = M;
    if (a == 0) return false;
    while (b) {
        const uint32_t t = a % b;
        a = b;
        b = t;
    }
    return T <= M / a;
}

void pack_into(const gr_program *progs, const gr_launch *ls, const int32_t *modes, uint32_t n, const Layout &L,
               uint8_t *arena, uint32_t *table_bad, bool range_only) {
    // zero everything but the permutation area, which is fully overwritten:
    // the program records by their workers below, the rest here
    const size_t progs_end = L.progs_off + (size_t)n * sizeof(DevProg);
    memset(arena, 0, L.progs_off);
    memset(arena + progs_end, 0, L.perm_off - progs_end);
    ArenaHeader *H = reinterpret_cast<ArenaHeader *>(arena);
    H->magic = kArenaMagic;
    H->n_progs = n;
    for (uint32_t p = 0; p < n; ++p) {
        H->s_max = std::max(H->s_max, exec_count(progs[p]));
        H->b_max = std::max(H->b_max, ls[p].blocks);
    }
    H->progs_off = L.progs_off;
    H->order_off = L.order_off;
    H->segbase_off = L.segbase_off;
    H->items_off = L.items_off;
    H->n_items = (uint32_t)L.n_items;
    H->citems_off = L.citems_off;
    H->perm_off = L.perm_off;
    H->n_segments = L.n_segments;
    H->scratch_segmask_off = L.segmask_off;
    H->scratch_trace_off = L.trace_off;
    H->scratch_segrange_off = L.segrange_off;
    H->scratch_wide_off = L.wide_off;
    H->scratch_rel_off = L.rel_off;
    H->scratch_bytes = L.scratch_bytes;
    DevProg *dp = reinterpret_cast<DevProg *>(arena + L.progs_off);
    uint32_t *order = reinterpret_cast<uint32_t *>(arena + L.order_off);
    uint64_t *segbase = reinterpret_cast<uint64_t *>(arena + L.segbase_off);
    uint16_t *perm = reinterpret_cast<uint16_t *>(arena + L.perm_off);
    std::vector<uint64_t> cost(n);
    parallel_over(n, [&](uint32_t lo, uint32_t hi) {
    for (uint32_t p = lo; p < hi; ++p) {
        const gr_program &P = progs[p];
        DevProg &D = dp[p];
        memset(&D, 0, sizeof(DevProg));
        const uint32_t nsl = slots_of(P);
        // executed statement instances: identity without loops
        uint8_t st_of[GR_MAX_STMTS], ctr_of[GR_MAX_STMTS];
        uint32_t S = P.n_stmts;
        D.general = (P.n_loops || P.slot_pos) ? 1u : 0u;
        if (P.n_loops) {
            S = exec_order(P, st_of, ctr_of, GR_MAX_STMTS);
        } else {
            for (uint32_t s = 0; s < S; ++s) {
                st_of[s] = (uint8_t)s;
                ctr_of[s] = 0;
            }
        }
        D.n_stmts = S;
        D.n_slots = nsl;
        D.blocks = ls[p].blocks;
        D.threads = ls[p].threads;
        D.t_pad = t_pad_of(ls[p].threads);
        D.m_shared = P.m_shared;
        D.m_global = P.m_global;
        D.mode = modes ? modes[p] : GR_MODE_REPAIR;
        D.existing = P.existing_mask;
        D.n_neg = P.n_neg;
        for (uint32_t c = 0; c < P.n_neg; ++c) D.neg[c] = P.neg[c];
        D.trace_off = L.trace_elem[p];
        D.segmask_off = L.segmask_elem[p];
        for (uint32_t k = 0; k < nsl; ++k) {
            if (P.slot_level[k] == GR_GRID) D.grid_mask |= 1u << k;
            D.weights[k] = slot_weight_of(P, k);
            D.slot_gk[k] = P.slot_guard ? P.slot_guard[2 * k] : 0;
            D.slot_gr[k] = P.slot_guard ? P.slot_guard[2 * k + 1] : 0;
            if (D.slot_gk[k]) D.guarded_slots |= 1u << k;
        }
        // the slots whose barriers run before the next instance: those placed
        // after the statement preceding it
        for (uint32_t s = 0; s + 1 < S; ++s) {
            const uint32_t place = st_of[s + 1] - 1u;
            uint32_t m = 0;
            if (!P.slot_pos) {
                m = place < nsl ? 1u << place : 0u;  // slot k sits after statement k
            } else {
                for (uint32_t k = 0; k < nsl; ++k)
                    if (P.slot_pos[k] == place) m |= 1u << k;
            }
            D.gapslots[s] = m;
        }
        for (uint32_t s = 0; s < S; ++s) {
            const gr_stmt &st = P.stmts[st_of[s]];
            DevStmt &ds = D.stmts[s];
            const uint32_t M = st.space == GR_SHARED ? P.m_shared : P.m_global;
            const uint64_t d = P.iter_coef ? (uint64_t)(P.iter_coef[st_of[s]] % M) * ctr_of[s] : 0u;
            ds.op = st.op;
            ds.space = st.space;
            ds.kind = st.kind;
            ds.am = st.a % M;
            ds.bm = (uint32_t)(((uint64_t)(st.b % M) + d) % M);
            ds.cm = st.c % M;
            ds.perm_off = 0;
            ds.gk = st.guard_k;
            ds.gr = st.guard_r;
            ds.m = M;
            ds.flags = injective_on_threads(st, M, ls[p].threads) ? kStmtInjective : 0u;
            if (st.op == GR_W) D.write_mask |= 1u << s;
            if (st.space == GR_SHARED) D.shared_rows |= 1u << s;
            else D.global_rows |= 1u << s;
        }
        // permutation instances: each reads its window (rotated to start at
        // its b, which becomes 0); equal windows are shared, so that equal
        // instances stay one access pattern
        {
            uint16_t *dst = perm + L.perm_base[p];
            const uint64_t end = p + 1 < n ? L.perm_base[p + 1] : L.perm_elems;
            const uint32_t room = (uint32_t)(end - L.perm_base[p]);
            uint32_t used = 0, wst[GR_MAX_STMTS], wb[GR_MAX_STMTS], woff[GR_MAX_STMTS], nw = 0;
            for_each_perm_instance(P, ls[p], [&](uint32_t x, uint32_t s, const gr_stmt &st, uint32_t M, uint32_t b,
                                                 PermWindow w) {
                uint32_t off = 0xFFFFFFFFu;
                for (uint32_t k = 0; k < nw && off == 0xFFFFFFFFu; ++k)
                    if (wst[k] == s && wb[k] == b) off = woff[k];
                if (off == 0xFFFFFFFFu) {
                    off = used;
                    used += w.len;
                    wst[nw] = s;
                    wb[nw] = b;
                    woff[nw++] = off;
                    if (!window_to_u16(P.perm + st.perm_off, M, b, w, dst + off, range_only) && table_bad &&
                        s < table_bad[p])
                        table_bad[p] = s;
                }
                DevStmt &ds = D.stmts[x];
                ds.perm_off = (uint32_t)(L.perm_base[p] + off);
                ds.bm = 0;
                ds.pneed = w.need;
            });
            if (used < room) memset(dst + used, 0, (size_t)(room - used) * 2);
        }
        D.blk_invariant = blocks_alike(P) ? 1u : 0u;
        // the relation kernel takes programs on the shared array alone whose
        // blocks are alike (or that have one block): block 0's owner table
        // decides every pair
        D.fast = (D.global_rows == 0 && (D.blk_invariant || D.blocks == 1)) ? 1u : 0u;
        // access-pattern classes: statements with the same array, map and
        // guard touch the same words from the same threads
        for (uint32_t s = 0; s < 32; ++s) D.rep[s] = (uint8_t)s;
        {
            // a 64-bit key of each instance's pattern first, the fields on a match
            uint64_t key[GR_MAX_STMTS];
            for (uint32_t s = 0; s < S; ++s) {
                const DevStmt &a = D.stmts[s];
                uint64_t h = ((uint64_t)a.space << 8 | a.kind) * 0x9E3779B97F4A7C15ull;
                h = (h ^ a.am) * 0x9E3779B97F4A7C15ull;
                h = (h ^ a.bm) * 0x9E3779B97F4A7C15ull;
                h = (h ^ a.cm) * 0x9E3779B97F4A7C15ull;
                h = (h ^ a.perm_off) * 0x9E3779B97F4A7C15ull;
                h = (h ^ ((uint64_t)a.gk << 16 | a.gr)) * 0x9E3779B97F4A7C15ull;
                key[s] = h ^ a.m;
            }
            for (uint32_t s = 1; s < S; ++s) {
                const DevStmt &a = D.stmts[s];
                for (uint32_t q = 0; q < s; ++q) {
                    if (key[q] != key[s]) continue;
                    const DevStmt &b = D.stmts[q];
                    if (a.space == b.space && a.kind == b.kind && a.am == b.am && a.bm == b.bm && a.cm == b.cm &&
                        a.perm_off == b.perm_off && a.gk == b.gk && a.gr == b.gr && a.m == b.m) {
                        D.rep[s] = (uint8_t)q;
                        break;
                    }
                }
            }
        }
        segbase[p] = L.segmask_elem[p];
        // work estimate for the largest-first orders: block 0's accesses when
        // the blocks are alike (the same-block passes read no other block),
        // every block's otherwise, plus every block's global accesses (the
        // cross-block pass)
        {
            const uint64_t tp = t_pad_of(ls[p].threads), B = ls[p].blocks;
            const uint64_t G = (uint64_t)__builtin_popcount(D.global_rows);
            cost[p] = (uint64_t)S * tp * (D.blk_invariant ? 1u : B) + (B > 1 ? G * B * tp : 0u);
        }
    }
    });
    {
        const size_t tail = L.perm_off + L.perm_elems * 2;
        if (tail < L.arena_bytes) memset(arena + tail, 0, L.arena_bytes - tail);
    }
    segbase[n] = L.n_segments;
    // the relation kernel's programs first, then the general ones, each part
    // largest first
    std::iota(order, order + n, 0u);
    std::stable_sort(order, order + n, [&](uint32_t a, uint32_t b) {
        if (dp[a].fast != dp[b].fast) return dp[a].fast > dp[b].fast;
        return cost[a] > cost[b];
    });
    uint32_t n_fast = 0;
    while (n_fast < n && dp[order[n_fast]].fast) ++n_fast;
    H->n_fast = n_fast;
    bool simple = true;
    for (uint32_t p = 0; p < n && simple; ++p) simple = !dp[p].general && dp[p].global_rows == 0;
    H->flags = simple ? kArenaSimple : 0u;
    // expansion items, largest programs first: runs of up to kItemSegs
    // segments (kind 0); for a program whose blocks are alike the same-block
    // passes read block 0 only and only global statements have a cross-block
    // pass, so one item (kind 1) expands block 0 of its shared-array
    // statements and kind-0 items cover the global statements' segments
    uint32_t *items = reinterpret_cast<uint32_t *>(arena + L.items_off);
    uint64_t k = 0;
    auto emit = [&](uint32_t p, uint32_t lo, uint32_t hi, uint32_t kind) {
        items[4 * k] = p;
        items[4 * k + 1] = lo;
        items[4 * k + 2] = hi;
        items[4 * k + 3] = kind;
        ++k;
    };
    // the general programs' items first (the repair path expands only those)
    for (uint32_t ii = 0; ii < n; ++ii) {
        const uint32_t i = ii < n - n_fast ? n_fast + ii : ii - (n - n_fast);
        if (ii == n - n_fast) H->n_items_gen = (uint32_t)k;
        const uint32_t p = order[i];
        const DevProg &D = dp[p];
        const uint32_t segs = (uint32_t)(segbase[p + 1] - segbase[p]);
        if (D.blk_invariant && D.blocks > 1) {
            if (D.shared_rows) emit(p, 0, D.n_stmts, 1u);
            for (uint32_t s = 0; s < D.n_stmts; ++s) {
                if (!((D.global_rows >> s) & 1u)) continue;
                for (uint32_t lo = s * D.blocks; lo < (s + 1) * D.blocks; lo += kItemSegs)
                    emit(p, lo, std::min((s + 1) * D.blocks, lo + kItemSegs), 0u);
            }
        } else {
            for (uint32_t lo = 0; lo < segs; lo += kItemSegs) emit(p, lo, std::min(segs, lo + kItemSegs), 0u);
        }
    }
    if (n_fast == 0) H->n_items_gen = (uint32_t)k;
    H->n_items = (uint32_t)k;
    // check items of the general programs in their order (largest first); a
    // program split by blocks lists its first range (which also does the
    // cross-block pass) first
    uint32_t *citems = reinterpret_cast<uint32_t *>(arena + L.citems_off);
    uint32_t nc = 0, n_split = 0;
    for (uint32_t i = n_fast; i < n; ++i) {
        const uint32_t p = order[i];
        const uint32_t K = check_items_of(progs[p], ls[p]), B = ls[p].blocks;
        n_split += K > 1 ? 1u : 0u;
        for (uint32_t c = 0; c < K; ++c) {
            citems[4 * nc] = p;
            citems[4 * nc + 1] = (uint32_t)((uint64_t)B * c / K);
            citems[4 * nc + 2] = (uint32_t)((uint64_t)B * (c + 1) / K);
            citems[4 * nc + 3] = (c == 0 ? kItemPrimary : 0u) | (K > 1 ? kItemSplit : 0u);
            ++nc;
        }
    }
    H->n_citems = nc;
    H->n_split = n_split;
}

}  // namespace gr

namespace {

// ---------------------------------------------------------------------------
// Per-device workspace
// ---------------------------------------------------------------------------

struct SizeClass {
    uint32_t s_max, bt_log2, m_chunks, global, n_log2;
    bool operator<(const SizeClass &o) const {
        return std::tie(s_max, bt_log2, m_chunks, global, n_log2) <
               std::tie(o.s_max, o.bt_log2, o.m_chunks, o.global, o.n_log2);
    }
};

uint32_t ceil_log2(uint64_t x) {
    uint32_t l = 0;
    while ((1ull << l) < x) ++l;
    return l;
}


// The CTA shapes picked for a batch: the relation kernel's (kRelShapes), the
// general check kernel's (kShapes, plus kShapeBalanced), the largest
// program's statement instances (sizes the general check's table) and the
// kSkip* bits of the batch.
struct Tuned {
    uint32_t rel_shape = 0, gen_shape = 0, s_max = GR_MAX_STMTS, skip = 0, simple = 0;
    uint64_t rel_off = 0;  // the arena's scratch relation offset when known (0: no fused loop)
    uint32_t fuse = 0;     // the relation kernel runs the loop too (one launch), when timed faster
};

// The relation kernel's CTA shape that also runs the loop (kRelShapes[2]: 512
// threads, two per SM: 16 loop warps whose records fit its table).
constexpr uint32_t kRelFusedShape = 2;

struct DeviceBuf {
    void *p = nullptr;
    size_t cap = 0;
    gr_status ensure(size_t bytes) {
        if (bytes <= cap) return GR_OK;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t want = std::max(bytes, (size_t)1 << 20);
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(workspace)");
        cap = want;
        return GR_OK;
    }
};

struct Workspace {
    std::mutex mu;
    bool configured = false;
    int sms = 0;
    int smem_per_sm = 0;
    uint32_t max_dyn = 0;
    DeviceBuf arena, scratch, out, aux;
    std::map<SizeClass, Tuned> class_shape;                             // tuned host batches
    std::map<std::pair<const void *, uint32_t>, Tuned> arena_shape;     // gr_tune_packed
    uint8_t *host_arena = nullptr;  // pinned staging for the packed arena
    size_t host_arena_cap = 0;
    uint8_t *host_out = nullptr;    // pinned staging for a batch's results
    size_t host_out_cap = 0;
};

// A pinned host buffer of at least `bytes` in *buf (grown, contents dropped).
gr_status ensure_pinned(uint8_t **buf, size_t *cap, size_t bytes) {
    if (*cap >= bytes) return GR_OK;
    if (*buf) cudaFreeHost(*buf);
    *buf = nullptr;
    *cap = 0;
    const size_t want = std::max<size_t>(bytes, (size_t)1 << 20);
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void **>(buf), want, cudaHostAllocDefault);
    if (e != cudaSuccess) return cuda_fail(e, "cudaHostAlloc(staging)");
    *cap = want;
    return GR_OK;
}

constexpr int kMaxDevices = 64;
Workspace g_ws[kMaxDevices];

gr_status current_ws(Workspace **ws) {
    int dev = 0;
    GR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(GR_ECUDA, "device index %d unsupported", dev);
    *ws = &g_ws[dev];
    return GR_OK;
}


gr_status ensure_configured(Workspace &ws) {
    if (ws.configured) return GR_OK;
    int dev = 0;
    GR_CUDA(cudaGetDevice(&dev));
    GR_CUDA(cudaDeviceGetAttribute(&ws.sms, cudaDevAttrMultiProcessorCount, dev));
    GR_CUDA(cudaDeviceGetAttribute(&ws.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    int optin = 0;
    GR_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    ws.max_dyn = (uint32_t)optin;
    GR_CUDA(configure_kernels(ws.max_dyn));
    ws.configured = true;
    return GR_OK;
}

// Launch configuration of CTA shape `shape` for n programs whose largest has
// s_max statements: the owner table takes what is left of the SM's shared
// memory share after the fixed part (1 KB per CTA is reserved).  table_bytes
// is 0 when the shape cannot hold one address chunk of s_max rows.
LaunchCfg shape_cfg(const Workspace &ws, uint32_t n, uint32_t shape, uint32_t s_max) {
    const LaunchShape sh = kShapes[shape & kShapeMask];
    LaunchCfg c{0, 0, shape};
    const size_t per_cta = (size_t)ws.smem_per_sm / sh.ctas_per_sm;
    const size_t fixed = fixed_smem_bytes() + 1024;
    size_t table = per_cta > fixed ? (per_cta - fixed) / 2048 * 2048 : 0;
    const size_t room = ws.max_dyn > fixed_smem_bytes() ? (ws.max_dyn - fixed_smem_bytes()) / 2048 * 2048 : 0;
    table = std::min(table, room);
    if (shape == 0) table = std::min<size_t>(table, 96u * 1024u);
    const size_t need = std::max<size_t>((size_t)std::max(s_max, 1u) * 2u * kChunkWords, mhs_smem_bytes());
    static_assert(kMinTableBytes >= 25u * 2u * kChunkWords, "one chunk for 25 rows");
    if (table < need) return c;
    c.table_bytes = (uint32_t)table;
    const uint32_t resident = (uint32_t)ws.sms * sh.ctas_per_sm;
    // a program may take up to kMaxCheckSplit work items (blocks that differ)
    c.grid = std::max<uint32_t>(1u, (uint32_t)std::min<uint64_t>((uint64_t)n * kMaxCheckSplit, resident));
    if (shape & kShapeBalanced) {  // as many CTAs as give every CTA the same number of programs
        const uint32_t waves = (n + resident - 1) / resident;
        c.grid = std::max<uint32_t>(1u, (n + waves - 1) / waves);
    }
    return c;
}

// Launch of the relation kernel in CTA shape `shape` for n programs: the
// owner table takes what is left of the SM's shared-memory share after the
// fixed part (1 KB per CTA is reserved).  table_bytes is 0 when the shape
// cannot hold one 32-column window of 27 rows.
RelCfg rel_cfg(const Workspace &ws, uint32_t n, uint32_t shape) {
    const LaunchShape sh = kRelShapes[shape];
    RelCfg c{0, 0, shape};
    const size_t per_cta = (size_t)ws.smem_per_sm / sh.ctas_per_sm;
    const size_t fixed = rel_fixed_bytes() + 1024;
    size_t table = per_cta > fixed ? (per_cta - fixed) / 256 * 256 : 0;
    const size_t room = ws.max_dyn > rel_fixed_bytes() ? (ws.max_dyn - rel_fixed_bytes()) / 256 * 256 : 0;
    table = std::min(table, room);
    if (table < 2048) return c;
    c.table_bytes = (uint32_t)table;
    c.grid = std::max<uint32_t>(1u, std::min<uint32_t>(n, (uint32_t)ws.sms * sh.ctas_per_sm));
    return c;
}

// CTAs of the loop kernel: as many as the SMs hold at once, at most one warp
// per program.
uint32_t loop_grid(const Workspace &ws, uint32_t n, bool simple) {
    const size_t per = loop_smem_bytes(simple) + 1024;
    const uint32_t by_smem = (uint32_t)std::max<size_t>(1, (size_t)ws.smem_per_sm / per);
    const uint32_t by_threads = 2048u / loop_threads(simple);
    const uint32_t ctas = std::min(by_smem, by_threads);
    const uint32_t wpc = loop_threads(simple) / 32u;
    const uint32_t need = (n + wpc - 1) / wpc;
    return std::max<uint32_t>(1u, std::min<uint32_t>(need, (uint32_t)ws.sms * ctas));
}

// The whole launch configuration of a repair (or check) of n programs.
LaunchCfg full_cfg(const Workspace &ws, uint32_t n, const Tuned &t) {
    LaunchCfg c = shape_cfg(ws, n, t.gen_shape, t.s_max);
    if (!c.table_bytes) c = shape_cfg(ws, n, 0, t.s_max);
    if (!c.table_bytes) c = shape_cfg(ws, n, 3, t.s_max);
    c.rel = rel_cfg(ws, n, t.rel_shape);
    if (!c.rel.table_bytes) c.rel = rel_cfg(ws, n, 0);
    c.loop_grid = loop_grid(ws, n, t.simple != 0);
    c.skip = t.skip;
    c.simple = t.simple;
    // a batch of simple programs with no general one, where the autotuner
    // timed it faster: the relation kernel runs the loop too, overlapping it
    // with the relation tail
    c.fused = RelCfg{0, 0, 0};
    c.flags_off = 0;
    if (t.fuse && t.rel_off && t.simple && (t.skip & kSkipGeneral) && !(t.skip & kSkipFast)) {
        const RelCfg f = rel_cfg(ws, n, kRelFusedShape);
        if (f.table_bytes && relation_loop_fits(f.table_bytes)) {
            c.fused = f;
            c.flags_off = rel_flags_off(t.rel_off, n);
        }
    }
    return c;
}

// Default shapes (the relation kernel's first, the general check's 512 x 2,
// or 1024 x 1 when that cannot hold the rows).
LaunchCfg choose_cfg(const Workspace &ws, uint32_t n, uint32_t s_max = GR_MAX_STMTS) {
    Tuned t;
    t.s_max = s_max;
    return full_cfg(ws, n, t);
}

// The kSkip* bits of a packed batch from its header.

// ---- autotuner: the fastest CTA shapes per batch size class ---------------

SizeClass size_class(const gr_program *progs, const gr_launch *ls, uint32_t n) {
    SizeClass k{0, 0, 0, 0, ceil_log2(n)};
    for (uint32_t p = 0; p < n; ++p) {
        k.s_max = std::max(k.s_max, exec_count(progs[p]));
        k.bt_log2 = std::max(k.bt_log2, ceil_log2((uint64_t)ls[p].blocks * ls[p].threads));
        const uint32_t m = std::max(progs[p].m_shared, progs[p].m_global);
        k.m_chunks = std::max(k.m_chunks, (m + kChunkWords - 1) / kChunkWords);
        for (uint32_t s = 0; s < progs[p].n_stmts; ++s)
            if (progs[p].stmts[s].space == GR_GLOBAL) k.global = 1;
    }
    return k;
}

// Time every shape of the relation kernel on the batch's programs for it, and
// every shape of the general check kernel (plain and with the balanced grid)
// on the general programs' relations, and return the fastest of each.  The
// general traces must be expanded into d_scratch.  Synchronises the stream;
// leaves the scratch control words to be cleared by the next launch.
// The device time of launch(): the first run warms the shape, the fastest of
// the next three counts (single runs vary by several percent, enough to pick
// the wrong shape).  The scratch's control words are cleared before each run.
template <class F>
cudaError_t best_of_runs(F launch, void *d_scratch, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st, float *ms) {
    cudaError_t e = cudaSuccess;
    *ms = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        if ((e = cudaMemsetAsync(d_scratch, 0, 16, st)) != cudaSuccess) break;
        if ((e = cudaEventRecord(e0, st)) != cudaSuccess) break;
        if ((e = launch()) != cudaSuccess) break;
        if ((e = cudaEventRecord(e1, st)) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float t = 0;
        if ((e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) break;
        if (rep > 0 && t < *ms) *ms = t;
    }
    return e;
}

gr_status tune_cfg(const Workspace &ws, const void *d_arena, uint32_t n, void *d_scratch, uint64_t scratch_bytes,
                   cudaStream_t st, uint32_t s_max, uint32_t skip, Tuned *out) {
    Tuned t;
    t.s_max = s_max;
    t.skip = skip;
    cudaEvent_t e0, e1;
    GR_CUDA(cudaEventCreate(&e0));
    GR_CUDA(cudaEventCreate(&e1));
    auto timed = [&](auto launch, float *ms) { return best_of_runs(launch, d_scratch, e0, e1, st, ms); };
    cudaError_t e = cudaSuccess;
    if (!(skip & kSkipFast)) {
        float best = 1e30f;
        for (uint32_t sh = 0; sh < kNumRelShapes && e == cudaSuccess; ++sh) {
            const RelCfg rc = rel_cfg(ws, n, sh);
            if (!rc.table_bytes) continue;
            float ms = 0;
            e = timed([&] { return launch_relation(d_arena, n, nullptr, d_scratch, scratch_bytes, nullptr, rc, st); },
                      &ms);
            if (e == cudaSuccess && ms < best) {
                best = ms;
                t.rel_shape = sh;
            }
        }
    }
    if (!(skip & kSkipGeneral) && e == cudaSuccess) {
        float best = 1e30f;
        for (uint32_t v = 0; v < 2 * kNumShapes && e == cudaSuccess; ++v) {
            const uint32_t sh = v < kNumShapes ? v : ((v - kNumShapes) | kShapeBalanced);
            const LaunchCfg cfg = shape_cfg(ws, n, sh, s_max);
            if (!cfg.table_bytes) continue;
            if ((sh & kShapeBalanced) && cfg.grid == shape_cfg(ws, n, sh & kShapeMask, s_max).grid) continue;
            float ms = 0;
            e = timed([&] { return launch_check(d_arena, n, nullptr, d_scratch, scratch_bytes, nullptr, cfg, st); },
                      &ms);
            if (e == cudaSuccess && ms < best) {
                best = ms;
                t.gen_shape = sh;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "autotuner");
    *out = t;
    return GR_OK;
}

// Launch configuration for a device arena: its tuned shapes if gr_tune_packed
// ran on it, else the defaults.
LaunchCfg packed_cfg(const Workspace &ws, const void *d_arena, uint32_t n) {
    auto it = ws.arena_shape.find({d_arena, n});
    if (it != ws.arena_shape.end()) return full_cfg(ws, n, it->second);
    return choose_cfg(ws, n);
}

uint32_t expand_grid(const Workspace &ws) { return (uint32_t)ws.sms * 8u; }

gr_status upload_batch(Workspace &ws, const gr_program *progs, const gr_launch *ls, const int32_t *modes,
                       uint32_t n, cudaStream_t st, Layout *Lout) {
    Layout L = layout_of(progs, ls, n);
    // the previous call on this workspace may still be reading the staging buffer
    GR_CUDA(cudaStreamSynchronize(st));
    gr_status ps = ensure_pinned(&ws.host_arena, &ws.host_arena_cap, L.arena_bytes);
    if (ps != GR_OK) return ps;
    // the callers validated everything but the permutation tables, which are
    // checked while they are converted; the lowest bad program is reported
    // before any device work, as a full validation would
    std::vector<uint32_t> bad(n, 0xFFFFFFFFu);
    pack_into(progs, ls, modes, n, L, ws.host_arena, bad.data());
    for (uint32_t p = 0; p < n; ++p)
        if (bad[p] != 0xFFFFFFFFu) return fail(GR_EINVAL, "program %u stmt %u: the permutation entries it reads are not distinct indices below M", p, bad[p]);
    gr_status s;
    if ((s = ws.arena.ensure(L.arena_bytes)) != GR_OK) return s;
    if ((s = ws.scratch.ensure(L.scratch_bytes)) != GR_OK) return s;
    GR_CUDA(cudaMemcpyAsync(ws.arena.p, ws.host_arena, L.arena_bytes, cudaMemcpyHostToDevice, st));
    *Lout = L;
    return GR_OK;
}

// Wait for the stream, then report the kernels' device error word.
// The device error word's bits in words.
const char *device_error_text(uint32_t err) {
    if (err & kErrArgs) return "a launch's n or scratch size does not match the arena";
    if (err & kErrStall) return "a bounded wait for another CTA's result ran out";
    if (err & kErrTableTooSmall) return "owner table too small";
    return "unknown";
}

gr_status finish_sync(void *d_scratch, cudaStream_t st) {
    uint32_t err = 0;
    GR_CUDA(cudaMemcpyAsync(&err, static_cast<uint32_t *>(d_scratch) + 1, 4, cudaMemcpyDeviceToHost, st));
    GR_CUDA(cudaStreamSynchronize(st));
    if (err) return fail(GR_ECUDA, "device error word 0x%x (%s)", err, device_error_text(err));
    return GR_OK;
}

}  // namespace

namespace gr {
// Launch shape of the persistent repair for n packed programs on the current
// device (used by gr_repair_packed_noalloc in noalloc.cu).
LaunchCfg packed_launch_cfg(const void *d_arena, uint32_t n, uint32_t skip, bool simple, uint64_t rel_off,
                            gr_status *status) {
    Workspace *ws;
    LaunchCfg c{};
    if ((*status = current_ws(&ws)) != GR_OK) return c;
    std::lock_guard<std::mutex> g(ws->mu);
    if ((*status = ensure_configured(*ws)) != GR_OK) return c;
    auto it = ws->arena_shape.find({d_arena, n});
    Tuned t = it != ws->arena_shape.end() ? it->second : Tuned{};
    t.skip |= skip;
    t.simple = simple ? 1u : 0u;
    t.rel_off = rel_off;
    return full_cfg(*ws, n, t);
}

// Owner-table budget of the wide lane's check CTAs (512 threads, two per SM)
// for programs of up to s_max statement instances.
LaunchCfg wide_launch_cfg(uint32_t n, uint32_t s_max, gr_status *status) {
    Workspace *ws;
    LaunchCfg c{};
    if ((*status = current_ws(&ws)) != GR_OK) return c;
    std::lock_guard<std::mutex> g(ws->mu);
    if ((*status = ensure_configured(*ws)) != GR_OK) return c;
    return shape_cfg(*ws, n, 0, s_max);
}

void set_last_error(const char *msg) { g_last_error = msg; }
}  // namespace gr

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------

extern "C" {

const char *gr_version(void) { return "gpurepair-gb300 0.1 (sm_103a)"; }

const char *gr_last_error(void) { return g_last_error.c_str(); }

gr_status gr_validate(const gr_program *prog, gr_launch launch) { return validate_one(prog, launch, 0); }

gr_status gr_pack_size(const gr_program *progs, const gr_launch *launches, uint32_t n, uint64_t *arena_bytes,
                       uint64_t *scratch_bytes) {
    if (!arena_bytes || !scratch_bytes) return fail(GR_EINVAL, "NULL output");
    gr_status s = validate_all(progs, launches, n);
    if (s != GR_OK) return s;
    Layout L = layout_of(progs, launches, n);
    *arena_bytes = L.arena_bytes;
    *scratch_bytes = L.scratch_bytes;
    return GR_OK;
}

gr_status gr_pack(const gr_program *progs, const gr_launch *launches, const int32_t *modes, uint32_t n,
                  void *host_arena, uint64_t arena_bytes) {
    if (!host_arena) return fail(GR_EINVAL, "host_arena is NULL");
    if (reinterpret_cast<uintptr_t>(host_arena) % 16) return fail(GR_EINVAL, "host_arena not 16-byte aligned");
    gr_status s = validate_all(progs, launches, n);
    if (s != GR_OK) return s;
    if (modes)
        for (uint32_t p = 0; p < n; ++p)
            if (modes[p] != GR_MODE_REPAIR && modes[p] != GR_MODE_REMOVE)
                return fail(GR_EINVAL, "program %u: bad mode %d", p, modes[p]);
    Layout L = layout_of(progs, launches, n);
    if (arena_bytes < L.arena_bytes)
        return fail(GR_ECAPACITY, "arena needs %llu bytes", (unsigned long long)L.arena_bytes);
    pack_into(progs, launches, modes, n, L, static_cast<uint8_t *>(host_arena));
    return GR_OK;
}

gr_status gr_repair_packed(const void *d_arena, uint32_t n, const gr_options *opts, void *d_scratch,
                           uint64_t scratch_bytes, gr_repair_result *d_out, void *stream) {
    if (!d_arena || !d_scratch || !d_out || n == 0) return fail(GR_EINVAL, "NULL buffer or n == 0");
    if ((reinterpret_cast<uintptr_t>(d_arena) | reinterpret_cast<uintptr_t>(d_scratch)) % 256)
        return fail(GR_EINVAL, "d_arena and d_scratch must be 256-byte aligned");
    if (scratch_bytes < 256) return fail(GR_ECAPACITY, "scratch too small");
    gr_status s = validate_opts(opts);
    if (s != GR_OK) return s;
    Workspace *ws;
    if ((s = current_ws(&ws)) != GR_OK) return s;
    std::lock_guard<std::mutex> g(ws->mu);
    if ((s = ensure_configured(*ws)) != GR_OK) return s;
    GR_CUDA(enqueue_repair(d_arena, n, opts_or_default(opts), d_scratch, scratch_bytes, d_out,
                           packed_cfg(*ws, d_arena, n), expand_grid(*ws), true, true,
                           static_cast<cudaStream_t>(stream)));
    return GR_OK;
}

gr_status gr_repair_packed_wide(const void *d_arena, uint32_t n, const gr_options *opts, void *d_scratch,
                                uint64_t scratch_bytes, gr_repair_result *d_out, void *stream) {
    if (!d_arena || !d_scratch || !d_out || n == 0) return fail(GR_EINVAL, "NULL buffer or n == 0");
    if ((reinterpret_cast<uintptr_t>(d_arena) | reinterpret_cast<uintptr_t>(d_scratch)) % 256)
        return fail(GR_EINVAL, "d_arena and d_scratch must be 256-byte aligned");
    if (n > 65535) return fail(GR_EINVAL, "the wide lane takes at most 65,535 programs per call");
    gr_status s = validate_opts(opts);
    if (s != GR_OK) return s;
    Workspace *ws;
    if ((s = current_ws(&ws)) != GR_OK) return s;
    std::lock_guard<std::mutex> g(ws->mu);
    if ((s = ensure_configured(*ws)) != GR_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ArenaHeader h;
    GR_CUDA(cudaMemcpyAsync(&h, d_arena, sizeof(h), cudaMemcpyDeviceToHost, st));
    GR_CUDA(cudaStreamSynchronize(st));
    if (h.magic != kArenaMagic || h.n_progs < n) return fail(GR_EINVAL, "not a packed arena of %u programs", n);
    if (scratch_bytes < h.scratch_bytes)
        return fail(GR_ECAPACITY, "scratch needs %llu bytes", (unsigned long long)h.scratch_bytes);
    const LaunchCfg cfg = shape_cfg(*ws, n, 0, h.s_max);  // 512 threads, two CTAs per SM
    if (!cfg.table_bytes) return fail(GR_ECAPACITY, "no owner-table room for %u rows", h.s_max);
    GR_CUDA(cudaMemsetAsync(d_scratch, 0, 256, st));
    GR_CUDA(launch_expand(d_arena, d_scratch, scratch_bytes, false, expand_grid(*ws), st));
    GR_CUDA(launch_wide(d_arena, n, h.b_max, opts_or_default(opts), d_scratch, h.scratch_wide_off, d_out,
                        cfg.table_bytes, st));
    return GR_OK;
}

gr_status gr_expand_packed(const void *d_arena, void *d_scratch, uint64_t scratch_bytes, void *stream) {
    if (!d_arena || !d_scratch) return fail(GR_EINVAL, "NULL buffer");
    if ((reinterpret_cast<uintptr_t>(d_arena) | reinterpret_cast<uintptr_t>(d_scratch)) % 256)
        return fail(GR_EINVAL, "d_arena and d_scratch must be 256-byte aligned");
    if (scratch_bytes < 256) return fail(GR_ECAPACITY, "scratch too small");
    gr_status s;
    Workspace *ws;
    if ((s = current_ws(&ws)) != GR_OK) return s;
    std::lock_guard<std::mutex> g(ws->mu);
    if ((s = ensure_configured(*ws)) != GR_OK) return s;
    GR_CUDA(launch_expand(d_arena, d_scratch, scratch_bytes, true, expand_grid(*ws), static_cast<cudaStream_t>(stream)));
    return GR_OK;
}

gr_status gr_repair_expanded(const void *d_arena, uint32_t n, const gr_options *opts, void *d_scratch,
                             uint64_t scratch_bytes, gr_repair_result *d_out, void *stream) {
    if (!d_arena || !d_scratch || !d_out || n == 0) return fail(GR_EINVAL, "NULL buffer or n == 0");
    if ((reinterpret_cast<uintptr_t>(d_arena) | reinterpret_cast<uintptr_t>(d_scratch)) % 256)
        return fail(GR_EINVAL, "d_arena and d_scratch must be 256-byte aligned");
    if (scratch_bytes < 256) return fail(GR_ECAPACITY, "scratch too small");
    gr_status s = validate_opts(opts);
    if (s != GR_OK) return s;
    Workspace *ws;
    if ((s = current_ws(&ws)) != GR_OK) return s;
    std::lock_guard<std::mutex> g(ws->mu);
    if ((s = ensure_configured(*ws)) != GR_OK) return s;
    GR_CUDA(enqueue_repair(d_arena, n, opts_or_default(opts), d_scratch, scratch_bytes, d_out,
                           packed_cfg(*ws, d_arena, n), expand_grid(*ws), false, true,
                           static_cast<cudaStream_t>(stream)));
    return GR_OK;
}

gr_status gr_relation_packed(const void *d_arena, uint32_t n, void *d_scratch, uint64_t scratch_bytes,
                             void *stream) {
    if (!d_arena || !d_scratch || n == 0) return fail(GR_EINVAL, "NULL buffer or n == 0");
    if ((reinterpret_cast<uintptr_t>(d_arena) | reinterpret_cast<uintptr_t>(d_scratch)) % 256)
        return fail(GR_EINVAL, "d_arena and d_scratch must be 256-byte aligned");
    if (scratch_bytes < 256) return fail(GR_ECAPACITY, "scratch too small");
    gr_status s;
    Workspace *ws;
    if ((s = current_ws(&ws)) != GR_OK) return s;
    std::lock_guard<std::mutex> g(ws->mu);
    if ((s = ensure_configured(*ws)) != GR_OK) return s;
    GR_CUDA(enqueue_relation(d_arena, n, d_scratch, scratch_bytes, packed_cfg(*ws, d_arena, n), expand_grid(*ws),
                             false, true, static_cast<cudaStream_t>(stream)));
    return GR_OK;
}

gr_status gr_loop_packed(const void *d_arena, uint32_t n, const gr_options *opts, void *d_scratch,
                         uint64_t scratch_bytes, gr_repair_result *d_out, void *stream) {
    if (!d_arena || !d_scratch || !d_out || n == 0) return fail(GR_EINVAL, "NULL buffer or n == 0");
    if ((reinterpret_cast<uintptr_t>(d_arena) | reinterpret_cast<uintptr_t>(d_scratch)) % 256)
        return fail(GR_EINVAL, "d_arena and d_scratch must be 256-byte aligned");
    if (scratch_bytes < 256) return fail(GR_ECAPACITY, "scratch too small");
    gr_status s = validate_opts(opts);
    if (s != GR_OK) return s;
    Workspace *ws;
    if ((s = current_ws(&ws)) != GR_OK) return s;
    std::lock_guard<std::mutex> g(ws->mu);
    if ((s = ensure_configured(*ws)) != GR_OK) return s;
    GR_CUDA(enqueue_loop(d_arena, n, opts_or_default(opts), d_scratch, scratch_bytes, d_out,
                         packed_cfg(*ws, d_arena, n), static_cast<cudaStream_t>(stream)));
    return GR_OK;
}

gr_status gr_set_shape_packed(const void *d_arena, uint32_t n, uint32_t shape, void *stream) {
    if (!d_arena || n == 0) return fail(GR_EINVAL, "NULL arena or n == 0");
    if (reinterpret_cast<uintptr_t>(d_arena) % 256) return fail(GR_EINVAL, "d_arena must be 256-byte aligned");
    const uint32_t rel = shape & 0xFFu, gen = (shape >> 8) & 0xFFu;
    if (rel >= kNumRelShapes || (gen & ~(kShapeMask | kShapeBalanced)) || (gen & kShapeMask) >= kNumShapes ||
        (shape >> 17))
        return fail(GR_EINVAL, "shape word 0x%x names no built shape", shape);
    gr_status s;
    Workspace *ws;
    if ((s = current_ws(&ws)) != GR_OK) return s;
    std::lock_guard<std::mutex> g(ws->mu);
    if ((s = ensure_configured(*ws)) != GR_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ArenaHeader h;
    GR_CUDA(cudaMemcpyAsync(&h, d_arena, sizeof(h), cudaMemcpyDeviceToHost, st));
    GR_CUDA(cudaStreamSynchronize(st));
    if (h.magic != kArenaMagic || h.n_progs != n) return fail(GR_EINVAL, "d_arena is not a packed arena of %u programs", n);
    Tuned t;
    t.rel_shape = rel;
    t.gen_shape = gen;
    t.s_max = h.s_max;
    t.skip = skip_bits(h);
    t.simple = (h.flags & kArenaSimple) ? 1u : 0u;
    t.rel_off = h.scratch_rel_off;
    t.fuse = (shape >> 16) & 1u;
    if (t.fuse && !full_cfg(*ws, n, t).flags_off)
        return fail(GR_EINVAL, "bit 16 (one launch) is set, but the batch cannot run in one launch");
    ws->arena_shape[{d_arena, n}] = t;
    return GR_OK;
}

gr_status gr_relation_loop_packed(const void *d_arena, uint32_t n, const gr_options *opts, void *d_scratch,
                                  uint64_t scratch_bytes, gr_repair_result *d_out, void *stream) {
    if (!d_arena || !d_scratch || !d_out || n == 0) return fail(GR_EINVAL, "NULL buffer or n == 0");
    if ((reinterpret_cast<uintptr_t>(d_arena) | reinterpret_cast<uintptr_t>(d_scratch)) % 256)
        return fail(GR_EINVAL, "d_arena and d_scratch must be 256-byte aligned");
    gr_status s = validate_opts(opts);
    if (s != GR_OK) return s;
    Workspace *ws;
    if ((s = current_ws(&ws)) != GR_OK) return s;
    std::lock_guard<std::mutex> g(ws->mu);
    if ((s = ensure_configured(*ws)) != GR_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ArenaHeader h;
    GR_CUDA(cudaMemcpyAsync(&h, d_arena, sizeof(h), cudaMemcpyDeviceToHost, st));
    GR_CUDA(cudaStreamSynchronize(st));
    if (h.magic != kArenaMagic || h.n_progs != n) return fail(GR_EINVAL, "d_arena is not a packed arena of %u programs", n);
    if (scratch_bytes < h.scratch_bytes) return fail(GR_ECAPACITY, "scratch needs %llu bytes", (unsigned long long)h.scratch_bytes);
    // the tuned relation shape when gr_tune_packed ran on this arena; the
    // single launch itself always takes the 512 x 2 shape
    auto it = ws->arena_shape.find({d_arena, n});
    Tuned t = it != ws->arena_shape.end() ? it->second : Tuned{};
    t.skip = skip_bits(h);
    t.s_max = h.s_max;
    t.simple = (h.flags & kArenaSimple) ? 1u : 0u;
    t.rel_off = h.scratch_rel_off;
    t.fuse = 1;
    const LaunchCfg cfg = full_cfg(*ws, n, t);
    if (!cfg.flags_off)
        return fail(GR_EINVAL, "the batch cannot run in one launch: it needs straight-line programs on the "
                               "shared array only, with no general program");
    GR_CUDA(enqueue_repair(d_arena, n, opts_or_default(opts), d_scratch, scratch_bytes, d_out, cfg, expand_grid(*ws),
                           false, true, st));
    return GR_OK;
}

gr_status gr_tune_packed(const void *d_arena, uint32_t n, const gr_options *opts, void *d_scratch,
                         uint64_t scratch_bytes, gr_repair_result *d_out, void *stream, uint32_t *shape_out) {
    if (!d_arena || !d_scratch || !d_out || n == 0) return fail(GR_EINVAL, "NULL buffer or n == 0");
    if ((reinterpret_cast<uintptr_t>(d_arena) | reinterpret_cast<uintptr_t>(d_scratch)) % 256)
        return fail(GR_EINVAL, "d_arena and d_scratch must be 256-byte aligned");
    gr_status s = validate_opts(opts);
    if (s != GR_OK) return s;
    Workspace *ws;
    if ((s = current_ws(&ws)) != GR_OK) return s;
    std::lock_guard<std::mutex> g(ws->mu);
    if ((s = ensure_configured(*ws)) != GR_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ArenaHeader h;
    GR_CUDA(cudaMemcpyAsync(&h, d_arena, sizeof(h), cudaMemcpyDeviceToHost, st));
    GR_CUDA(cudaStreamSynchronize(st));
    if (h.magic != kArenaMagic || h.n_progs != n) return fail(GR_EINVAL, "d_arena is not a packed arena of %u programs", n);
    if (scratch_bytes < h.scratch_bytes) return fail(GR_ECAPACITY, "scratch needs %llu bytes", (unsigned long long)h.scratch_bytes);
    const uint32_t skip = skip_bits(h);
    GR_CUDA(cudaMemsetAsync(d_scratch, 0, 256, st));
    if (!(skip & kSkipGeneral)) GR_CUDA(launch_expand(d_arena, d_scratch, scratch_bytes, true, expand_grid(*ws), st));
    Tuned t;
    if ((s = tune_cfg(*ws, d_arena, n, d_scratch, scratch_bytes, st, h.s_max, skip, &t)) != GR_OK) return s;
    t.simple = (h.flags & kArenaSimple) ? 1u : 0u;
    t.rel_off = h.scratch_rel_off;
    // two launches (relation, loop): the single launch (bit 16) is only
    // taken when asked for (gr_set_shape_packed, gr_relation_loop_packed).
    // Timed here on a warm L2 it sometimes came out ahead, then lost in
    // steady runs that read their inputs from HBM.
    ws->arena_shape[{d_arena, n}] = t;
    // one repair with the picked shapes leaves d_out filled, as documented
    GR_CUDA(enqueue_repair(d_arena, n, opts_or_default(opts), d_scratch, scratch_bytes, d_out, full_cfg(*ws, n, t),
                           expand_grid(*ws), false, true, st));
    GR_CUDA(cudaStreamSynchronize(st));
    if (shape_out) *shape_out = t.rel_shape | (t.gen_shape << 8) | (t.fuse << 16);
    return GR_OK;
}

gr_status gr_check_packed(const void *d_arena, uint32_t n, const uint32_t *d_masks, void *d_scratch,
                          uint64_t scratch_bytes, gr_witnesses *d_out, void *stream) {
    if (!d_arena || !d_scratch || !d_out || !d_masks || n == 0) return fail(GR_EINVAL, "NULL buffer or n == 0");
    if ((reinterpret_cast<uintptr_t>(d_arena) | reinterpret_cast<uintptr_t>(d_scratch)) % 256)
        return fail(GR_EINVAL, "d_arena and d_scratch must be 256-byte aligned");
    if (scratch_bytes < 256) return fail(GR_ECAPACITY, "scratch too small");
    gr_status s;
    Workspace *ws;
    if ((s = current_ws(&ws)) != GR_OK) return s;
    std::lock_guard<std::mutex> g(ws->mu);
    if ((s = ensure_configured(*ws)) != GR_OK) return s;
    GR_CUDA(enqueue_check(d_arena, n, d_masks, d_scratch, scratch_bytes, d_out, packed_cfg(*ws, d_arena, n),
                          expand_grid(*ws), true, static_cast<cudaStream_t>(stream)));
    return GR_OK;
}

gr_status gr_check_expanded(const void *d_arena, uint32_t n, const uint32_t *d_masks, void *d_scratch,
                            uint64_t scratch_bytes, gr_witnesses *d_out, void *stream) {
    if (!d_arena || !d_scratch || !d_out || !d_masks || n == 0) return fail(GR_EINVAL, "NULL buffer or n == 0");
    if ((reinterpret_cast<uintptr_t>(d_arena) | reinterpret_cast<uintptr_t>(d_scratch)) % 256)
        return fail(GR_EINVAL, "d_arena and d_scratch must be 256-byte aligned");
    if (scratch_bytes < 256) return fail(GR_ECAPACITY, "scratch too small");
    gr_status s;
    Workspace *ws;
    if ((s = current_ws(&ws)) != GR_OK) return s;
    std::lock_guard<std::mutex> g(ws->mu);
    if ((s = ensure_configured(*ws)) != GR_OK) return s;
    GR_CUDA(enqueue_check(d_arena, n, d_masks, d_scratch, scratch_bytes, d_out, packed_cfg(*ws, d_arena, n),
                          expand_grid(*ws), false, static_cast<cudaStream_t>(stream)));
    return GR_OK;
}

gr_status gr_repair_batch(const gr_program *progs, const gr_launch *launches, const int32_t *modes, uint32_t n,
                          const gr_options *opts, gr_repair_result *out, void *stream) {
    if (!out) return fail(GR_EINVAL, "out is NULL");
    // validation and each program's share of the packed layout, in one pass
    std::vector<ProgSizes> sizes(n);
    gr_status s = validate_all(progs, launches, n, false, sizes.data());
    if (s != GR_OK) return s;
    if ((s = validate_opts(opts)) != GR_OK) return s;
    if (modes)
        for (uint32_t p = 0; p < n; ++p)
            if (modes[p] != GR_MODE_REPAIR && modes[p] != GR_MODE_REMOVE)
                return fail(GR_EINVAL, "program %u: bad mode %d", p, modes[p]);
    Workspace *ws;
    if ((s = current_ws(&ws)) != GR_OK) return s;
    std::lock_guard<std::mutex> g(ws->mu);
    if ((s = ensure_configured(*ws)) != GR_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Large batches go in chunks so that packing chunk c+1 on the host
    // overlaps the device work of chunk c (H2D, expansion, repair, all on one
    // stream: the device arena and scratch are reused in order).  Results
    // gather in the device result buffer and reach `out` in one copy at the
    // end, so `out` stays untouched when a later chunk holds a bad table.
    // Below 2,048 programs the batch goes in one chunk: a launch of a few
    // hundred programs takes about one program's latency (one per CTA), and
    // packing 1,024 programs takes about as long, so a second chunk adds a
    // latency to the device's chain without hiding more than it adds.
    // The last chunk is half the size of the others: only its device work is
    // not hidden behind packing.
    const uint32_t K = n >= 2048 ? 4u : 1u;
    std::vector<uint32_t> lo(K + 1);
    for (uint32_t c = 0; c < K; ++c) lo[c] = (uint32_t)((uint64_t)n * (2u * c) / (2u * K - 1u));
    lo[K] = n;
    std::vector<Layout> Ls(K);
    std::vector<size_t> soff(K);
    size_t stage = 0, arena_max = 0, scratch_max = 0;
    for (uint32_t c = 0; c < K; ++c) {
        Ls[c] = layout_from(sizes.data() + lo[c], lo[c + 1] - lo[c]);
        soff[c] = stage;
        stage += align_to(Ls[c].arena_bytes, 256);
        arena_max = std::max(arena_max, Ls[c].arena_bytes);
        scratch_max = std::max(scratch_max, Ls[c].scratch_bytes);
    }
    // the previous call on this workspace may still be reading the staging buffer
    GR_CUDA(cudaStreamSynchronize(st));
    if ((s = ensure_pinned(&ws->host_arena, &ws->host_arena_cap, stage)) != GR_OK) return s;
    if ((s = ws->arena.ensure(arena_max)) != GR_OK) return s;
    if ((s = ws->scratch.ensure(scratch_max)) != GR_OK) return s;
    if ((s = ws->out.ensure((size_t)n * sizeof(gr_repair_result))) != GR_OK) return s;
    if ((s = ws->aux.ensure(256)) != GR_OK) return s;
    gr_repair_result *d_out = static_cast<gr_repair_result *>(ws->out.p);
    uint32_t *d_perm_bad = static_cast<uint32_t *>(ws->aux.p);
    bool any_perm = false;
    for (uint32_t p = 0; p < n && !any_perm; ++p) any_perm = progs[p].perm && progs[p].perm_len;
    if (any_perm) GR_CUDA(cudaMemsetAsync(d_perm_bad, 0, 4, st));
    // Permutation tables: the packer checks the range of every entry while
    // converting; that each index occurs once is checked on the device
    // (k_perm_check) and read back before the results are copied.  Either way
    // the lowest bad program is reported and `out` stays untouched.
    auto bad_stmt = [&](uint32_t p) -> uint32_t {  // the first bad permutation window of p, or ~0u
        return first_bad_window(progs[p], launches[p]);
    };
    auto device_bad = [&](uint32_t *p_out) -> gr_status {  // waits for the stream
        uint32_t word = 0;
        if (any_perm) GR_CUDA(cudaMemcpyAsync(&word, d_perm_bad, 4, cudaMemcpyDeviceToHost, st));
        GR_CUDA(cudaStreamSynchronize(st));
        *p_out = word ? ~word : 0xFFFFFFFFu;
        return GR_OK;
    };
    const size_t rb = (size_t)n * sizeof(gr_repair_result);
    if ((s = ensure_pinned(&ws->host_out, &ws->host_out_cap, rb + 16)) != GR_OK) return s;
    std::vector<uint32_t> bad;
    for (uint32_t c = 0; c < K; ++c) {
        const uint32_t n_c = lo[c + 1] - lo[c];
        uint8_t *staging = ws->host_arena + soff[c];
        bad.assign(n_c, 0xFFFFFFFFu);
        pack_into(progs + lo[c], launches + lo[c], modes ? modes + lo[c] : nullptr, n_c, Ls[c], staging, bad.data(),
                  true);
        for (uint32_t p = 0; p < n_c; ++p)
            if (bad[p] != 0xFFFFFFFFu) {
                // an entry out of range: a lower program may hold a repeat, in
                // an earlier chunk (the device check has run) or in this one
                uint32_t low = 0xFFFFFFFFu;
                if ((s = device_bad(&low)) != GR_OK) return s;
                for (uint32_t q = lo[c]; q < lo[c] + p && low == 0xFFFFFFFFu; ++q)
                    if (bad_stmt(q) != 0xFFFFFFFFu) low = q;
                if (low < lo[c] + p)
                    return fail(GR_EINVAL, "program %u stmt %u: the permutation entries it reads are not distinct indices below M", low, bad_stmt(low));
                return fail(GR_EINVAL, "program %u stmt %u: the permutation entries it reads are not distinct indices below M", lo[c] + p, bad[p]);
            }
        GR_CUDA(cudaMemcpyAsync(ws->arena.p, staging, Ls[c].arena_bytes, cudaMemcpyHostToDevice, st));
        if (any_perm) GR_CUDA(launch_perm_check(ws->arena.p, n_c, lo[c], d_perm_bad, (uint32_t)ws->sms, st));
        const uint32_t skip = skip_bits(*reinterpret_cast<const ArenaHeader *>(staging));
        const uint64_t sb = Ls[c].scratch_bytes;
        // the chunk's size class picks the CTA shapes; the first batch of a class tunes them
        const SizeClass cls = size_class(progs + lo[c], launches + lo[c], n_c);
        auto it = ws->class_shape.find(cls);
        if (it == ws->class_shape.end()) {
            // tuning clears the scratch control words: report an earlier chunk's error first
            if (c > 0 && (s = finish_sync(ws->scratch.p, st)) != GR_OK) return s;
            GR_CUDA(cudaMemsetAsync(ws->scratch.p, 0, 256, st));
            if (!(skip & kSkipGeneral))
                GR_CUDA(launch_expand(ws->arena.p, ws->scratch.p, sb, true, expand_grid(*ws), st));
            Tuned t;
            gr_status ts = tune_cfg(*ws, ws->arena.p, n_c, ws->scratch.p, sb, st, cls.s_max, skip, &t);
            if (ts != GR_OK) return ts;
            t.skip = 0;  // per chunk below
            it = ws->class_shape.emplace(cls, t).first;
        }
        Tuned tc = it->second;
        tc.skip = skip;
        tc.simple = (reinterpret_cast<const ArenaHeader *>(staging)->flags & kArenaSimple) ? 1u : 0u;
        tc.rel_off = Ls[c].rel_off;
        const LaunchCfg cfg = full_cfg(*ws, n_c, tc);
        // the queue counters (and, for the first chunk, the error word) are cleared first
        GR_CUDA(enqueue_repair(ws->arena.p, n_c, opts_or_default(opts), ws->scratch.p, sb, d_out + lo[c], cfg,
                               expand_grid(*ws), true, c == 0, st));
        // the chunk's results start back while the host packs the next one
        GR_CUDA(cudaMemcpyAsync(ws->host_out + (size_t)lo[c] * sizeof(gr_repair_result), d_out + lo[c],
                                (size_t)n_c * sizeof(gr_repair_result), cudaMemcpyDeviceToHost, st));
    }
    // The results (above, per chunk), the permutation word and the device
    // error word come back through pinned staging (DMAs at full speed, and no
    // copy into pageable memory, which would block the host until the stream
    // reaches it) with one synchronisation; `out` is written only if both
    // words are clean.
    uint32_t *words = reinterpret_cast<uint32_t *>(ws->host_out + rb);
    words[0] = 0;
    if (any_perm) GR_CUDA(cudaMemcpyAsync(&words[0], d_perm_bad, 4, cudaMemcpyDeviceToHost, st));
    GR_CUDA(cudaMemcpyAsync(&words[1], static_cast<uint32_t *>(ws->scratch.p) + 1, 4, cudaMemcpyDeviceToHost, st));
    GR_CUDA(cudaStreamSynchronize(st));
    if (words[0]) {
        const uint32_t low = ~words[0];
        return fail(GR_EINVAL, "program %u stmt %u: the permutation entries it reads are not distinct indices below M",
                    low, bad_stmt(low));
    }
    if (words[1]) return fail(GR_ECUDA, "device error word 0x%x (%s)", words[1], device_error_text(words[1]));
    const uint8_t *staged = ws->host_out;
    parallel_over(n, [&](uint32_t a, uint32_t b) {
        memcpy(out + a, staged + (size_t)a * sizeof(gr_repair_result), (size_t)(b - a) * sizeof(gr_repair_result));
    });
    return GR_OK;
}

gr_status gr_check_batch(const gr_program *progs, const gr_launch *launches, const uint32_t *masks, uint32_t n,
                         gr_witnesses *out, void *stream) {
    if (!out || !masks) return fail(GR_EINVAL, "out or masks is NULL");
    gr_status s = validate_all(progs, launches, n, false);
    if (s != GR_OK) return s;
    for (uint32_t p = 0; p < n; ++p) {
        const uint32_t nsl = slots_of(progs[p]);
        if (nsl < 32 && (masks[p] >> nsl)) return fail(GR_EINVAL, "program %u: mask has bits beyond slot %u", p, nsl);
    }
    Workspace *ws;
    if ((s = current_ws(&ws)) != GR_OK) return s;
    std::lock_guard<std::mutex> g(ws->mu);
    if ((s = ensure_configured(*ws)) != GR_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Layout L;
    if ((s = upload_batch(*ws, progs, launches, nullptr, n, st, &L)) != GR_OK) return s;
    const size_t mask_bytes = align_to((size_t)n * 4, 256);
    if ((s = ws->out.ensure((size_t)n * sizeof(gr_witnesses))) != GR_OK) return s;
    if ((s = ws->aux.ensure(mask_bytes)) != GR_OK) return s;
    GR_CUDA(cudaMemcpyAsync(ws->aux.p, masks, (size_t)n * 4, cudaMemcpyHostToDevice, st));
    const SizeClass cls = size_class(progs, launches, n);
    auto it = ws->class_shape.find(cls);
    LaunchCfg cfg = it == ws->class_shape.end() ? choose_cfg(*ws, n, cls.s_max) : full_cfg(*ws, n, it->second);
    cfg.skip = skip_bits(*reinterpret_cast<const ArenaHeader *>(ws->host_arena));
    GR_CUDA(enqueue_check(ws->arena.p, n, static_cast<const uint32_t *>(ws->aux.p), ws->scratch.p, L.scratch_bytes,
                          static_cast<gr_witnesses *>(ws->out.p), cfg, expand_grid(*ws), true, st));
    GR_CUDA(cudaMemcpyAsync(out, ws->out.p, (size_t)n * sizeof(gr_witnesses), cudaMemcpyDeviceToHost, st));
    return finish_sync(ws->scratch.p, st);
}

gr_status gr_check(const gr_program *prog, gr_launch launch, uint32_t mask, gr_witnesses *out) {
    return gr_check_batch(prog, &launch, &mask, 1, out, nullptr);
}

gr_status gr_repair(const gr_program *prog, gr_launch launch, int32_t mode, const gr_options *opts,
                    gr_repair_result *out) {
    return gr_repair_batch(prog, &launch, &mode, 1, opts, out, nullptr);
}

gr_status gr_repair_plain(const gr_program *prog, gr_launch launch, int32_t mode, const gr_options *opts,
                          gr_repair_result *out) {
    return gr_repair_plain_timed(prog, launch, mode, opts, out, nullptr);
}

gr_status gr_repair_plain_timed(const gr_program *prog, gr_launch launch, int32_t mode, const gr_options *opts,
                                gr_repair_result *out, float *loop_ms) {
    if (!out) return fail(GR_EINVAL, "out is NULL");
    gr_status s = validate_all(prog, &launch, 1, false);
    if (s != GR_OK) return s;
    if ((s = validate_opts(opts)) != GR_OK) return s;
    if (mode != GR_MODE_REPAIR && mode != GR_MODE_REMOVE) return fail(GR_EINVAL, "bad mode %d", mode);
    Workspace *ws;
    if ((s = current_ws(&ws)) != GR_OK) return s;
    std::lock_guard<std::mutex> g(ws->mu);
    if ((s = ensure_configured(*ws)) != GR_OK) return s;
    cudaStream_t st = nullptr;
    Layout L;
    if ((s = upload_batch(*ws, prog, &launch, &mode, 1, st, &L)) != GR_OK) return s;
    const size_t state_bytes = align_to(sizeof(LoopState), 256);
    const size_t wit_bytes = align_to(sizeof(gr_witnesses), 256);
    if ((s = ws->aux.ensure(state_bytes + wit_bytes + sizeof(gr_repair_result))) != GR_OK) return s;
    LoopState *d_state = static_cast<LoopState *>(ws->aux.p);
    gr_witnesses *d_wit = reinterpret_cast<gr_witnesses *>(static_cast<uint8_t *>(ws->aux.p) + state_bytes);
    gr_repair_result *d_out =
        reinterpret_cast<gr_repair_result *>(static_cast<uint8_t *>(ws->aux.p) + state_bytes + wit_bytes);
    // events bracket the launch loop alone: expansion, the per-iteration
    // launches and the host's read of the done flag, not validation,
    // packing or the upload
    struct Events {
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~Events() {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } events;
    cudaEvent_t *ev = events.e;
    if (loop_ms) {
        GR_CUDA(cudaEventCreate(&ev[0]));
        GR_CUDA(cudaEventCreate(&ev[1]));
        GR_CUDA(cudaEventRecord(ev[0], st));
    }
    GR_CUDA(cudaMemsetAsync(ws->scratch.p, 0, 256, st));
    GR_CUDA(launch_expand(ws->arena.p, ws->scratch.p, L.scratch_bytes, false, expand_grid(*ws), st));
    const gr_options o = opts_or_default(opts);
    GR_CUDA(launch_plain_init(ws->arena.p, 0, o, d_state, st));
    const LaunchCfg cfg = choose_cfg(*ws, 1);
    uint32_t done = 0;
    GR_CUDA(cudaMemcpy(&done, &d_state->done, 4, cudaMemcpyDeviceToHost));
    for (uint32_t guard = 0; !done && guard <= GR_MAX_ITERS; ++guard) {
        GR_CUDA(cudaMemsetAsync(d_wit, 0, sizeof(gr_witnesses), st));
        GR_CUDA(launch_plain_check(ws->arena.p, 0, ws->scratch.p, d_state, d_wit, launch.blocks, cfg.table_bytes, st));
        GR_CUDA(launch_plain_solve(ws->arena.p, 0, d_state, d_wit, d_out, st));
        GR_CUDA(cudaMemcpy(&done, &d_state->done, 4, cudaMemcpyDeviceToHost));
    }
    if (!done) return fail(GR_ECUDA, "plain loop did not terminate");
    if (L.n_segments == 0) return fail(GR_ECUDA, "empty layout");
    // a program that ended in the initial solve still needs its result written
    GR_CUDA(launch_plain_solve(ws->arena.p, 0, d_state, d_wit, d_out, st));
    if (loop_ms) {
        GR_CUDA(cudaEventRecord(ev[1], st));
        GR_CUDA(cudaEventSynchronize(ev[1]));
        GR_CUDA(cudaEventElapsedTime(loop_ms, ev[0], ev[1]));
    }
    GR_CUDA(cudaMemcpy(out, d_out, sizeof(gr_repair_result), cudaMemcpyDeviceToHost));
    return GR_OK;
}

gr_status gr_solve(uint32_t n_vars, const uint32_t *w, const uint32_t *pos, uint32_t n_pos, const uint32_t *neg,
                   uint32_t n_neg, uint32_t forced, uint32_t forbidden, uint32_t *mask_out, uint32_t *weight_out) {
    if (!mask_out || !weight_out || !w) return fail(GR_EINVAL, "NULL argument");
    if (n_vars < 1 || n_vars > GR_MAX_SLOTS) return fail(GR_EINVAL, "n_vars %u outside 1..%d", n_vars, GR_MAX_SLOTS);
    if (n_pos + n_neg > GR_MAX_CLAUSES) return fail(GR_EINVAL, "more than %d clauses", GR_MAX_CLAUSES);
    if ((n_pos && !pos) || (n_neg && !neg)) return fail(GR_EINVAL, "NULL clause array");
    const uint32_t full = n_vars == 32 ? 0xFFFFFFFFu : ((1u << n_vars) - 1u);
    for (uint32_t k = 0; k < n_vars; ++k)
        if (w[k] < 1 || w[k] > GR_MAX_WEIGHT) return fail(GR_EINVAL, "weight %u outside 1..2^24", k);
    for (uint32_t i = 0; i < n_pos; ++i)
        if (pos[i] & ~full) return fail(GR_EINVAL, "positive clause %u uses a variable >= n_vars", i);
    for (uint32_t i = 0; i < n_neg; ++i)
        if ((neg[i] & ~full) || neg[i] == 0) return fail(GR_EINVAL, "negative clause %u empty or out of range", i);
    if ((forced | forbidden) & ~full) return fail(GR_EINVAL, "forced/forbidden use a variable >= n_vars");
    std::vector<uint32_t> in(5 + GR_MAX_SLOTS + n_pos + n_neg, 0);
    in[0] = n_vars;
    in[1] = n_pos;
    in[2] = n_neg;
    in[3] = forced;
    in[4] = forbidden;
    for (uint32_t k = 0; k < n_vars; ++k) in[5 + k] = w[k];
    for (uint32_t i = 0; i < n_pos; ++i) in[5 + GR_MAX_SLOTS + i] = pos[i];
    for (uint32_t i = 0; i < n_neg; ++i) in[5 + GR_MAX_SLOTS + n_pos + i] = neg[i];
    gr_status s;
    Workspace *ws;
    if ((s = current_ws(&ws)) != GR_OK) return s;
    std::lock_guard<std::mutex> g(ws->mu);
    if ((s = ensure_configured(*ws)) != GR_OK) return s;
    const size_t in_bytes = align_to(in.size() * 4, 256);
    if ((s = ws->aux.ensure(in_bytes + 256)) != GR_OK) return s;
    uint32_t *d_in = static_cast<uint32_t *>(ws->aux.p);
    uint32_t *d_out = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(ws->aux.p) + in_bytes);
    GR_CUDA(cudaMemcpy(d_in, in.data(), in.size() * 4, cudaMemcpyHostToDevice));
    GR_CUDA(launch_solve(d_in, d_out, nullptr));
    uint32_t res[3];
    GR_CUDA(cudaMemcpy(res, d_out, sizeof(res), cudaMemcpyDeviceToHost));
    *mask_out = res[1];
    *weight_out = res[2];
    return res[0] ? GR_OK : GR_UNSAT;
}

}  // extern "C"
