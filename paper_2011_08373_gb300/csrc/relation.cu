// relation.cu — the check kernel (Verify of Algorithm 1, Section 2.4) for
// programs whose statements all address the shared array and whose blocks
// see one access pattern: the same-block witnesses of every block are block
// 0's, and no pair of blocks shares an array, so one owner-table pass over
// block 0 decides every candidate pair.
//
// Each CTA takes programs from a work queue, three at a time in three
// program buffers: while warps 2.. (the workers) check program k, warp 1
// fetches and sets up program k+1 and warp 0 writes out program k-1, so that
// the setup's loads and arithmetic and the output overlap the table pass
// (and each other: on one warp, setup and output took longer than a
// program's install).  Per program:
//   setup   — (warp 1) the candidate pairs: under a mask, the instance pairs
//             (i <= j) with a write and no enabled barrier between them (one
//             phase, Section 2.2); for the repair loop, every pair with a
//             write (the empty mask), which gives the program's whole
//             conflict relation.  Instances with the same map and guard touch
//             the same words from the same threads and share one table row.
//   install — (workers) every access computes its word address from the map
//             (affine or strided arithmetic, or one permutation-table load),
//             writes its thread into its row's owner entry at that word (two
//             threads of a row on one word leave MULTI: a compare-and-swap,
//             only for rows whose map is not injective on the block's
//             threads), then marks its row in the word's column mask with an
//             acquire-release atomic that returns the rows already there, and
//             compares its thread with their entries.  Two rows conflict at a
//             word unless both hold the same single thread there (another
//             thread, or MULTI, is a second thread on the word: the race
//             definition of Section 1 made concrete — two distinct threads,
//             one word, at least one write, no barrier between them).  Of the
//             accesses of two rows to a word, the one whose atomic comes last
//             sees the other row's final entry, so every conflicting pair is
//             found; a row whose pairs are all decided stops installing.
//   reset   — (workers) the column masks used go back to empty; entries
//             carry the window's epoch, so stale ones read as empty.
// Install works in units of one table row and 64 consecutive active threads
// (two per lane), a warp per unit, so that a unit's map, guard and row are
// the same for the whole warp: the per-unit arithmetic is done once and each
// access costs a multiply and a reduction.  The table covers the array in windows when it
// does not fit.
#include <cuda_runtime.h>

#include <cstdint>

#include "device.cuh"
#include "loop.cuh"

namespace gr {

constexpr uint32_t kRelAllOnes = 0xFFFFFFFFu;

// One program's state (warp 1 fills one, the workers use one, warp 0 writes
// one out).
struct RelProg {
    DevProg prog;
    uint32_t cand[32];      // table row q: candidate partner rows (bit j, j >= q)
    uint32_t open[32];      // table row q: candidate partners in either direction not found yet
    uint32_t pend[32];      // instance i: candidate partners (bit j, j >= i)
    uint32_t rep_conf[32];  // the conflicts by pattern representative
    // table row q's access map (its representative's statement, block 0):
    // {am, bm, po, gk | gr << 16}: the address of thread t is (am t + bm)
    // mod M, or perm[po + (t + bm) mod M] when po != ~0; the guard holds iff
    // gk == 0 or t mod gk == gr
    uint4 row_map[32];
    uint32_t row_nact[32];  // threads of a block the row's guard lets through
    uint32_t nact[32];      // active threads of each instance (for the pair count)
    uint32_t involved, n_rows, W, pitch, n_win, inj_rows, bad, p, mask;
    uint32_t M, Mmagic;     // the shared array's words; floor((2^32 - 1) / M)
};

// Warps 0 and 1 are the control warps (warp 0 writes programs out, warp 1
// fetches and sets them up); the others are the workers.
constexpr uint32_t kRelCtl = 2;

struct RelSmem {
    RelProg buf[3];  // program k - 1 (output), k (install), k + 1 (setup), by k mod 3
};

constexpr size_t kRelFixed = (sizeof(RelSmem) + 15) / 16 * 16;
size_t rel_fixed_bytes() { return kRelFixed; }

// Column of word a within a window row: the low five bits are XOR-ed with
// the next five, so that 32 words spaced 32 apart (stride-32 maps) fall on
// 32 different banks; the window width is a multiple of 64, so a column
// stays within its row.
__device__ __forceinline__ uint32_t swizzle(uint32_t c) { return c ^ ((c >> 5) & 31u); }

// The owner table: an entry area of u16 entries (rows of one program, W + 2
// entries each) and, after it, a mask area of u32 column masks.  An entry
// carries an epoch (bits 11-15; one per window, 1..31, 0 = cleared), the
// MULTI flag (bit 10) and a thread (bits 0-9, T <= 1,024), so entries left by
// earlier windows read as empty without being cleared; the mask area is
// cleared after each window.  The areas never overlap, whatever the rows and
// widths of consecutive programs.
constexpr uint32_t kEntEpochShift = 11, kEntMulti = 1u << 10, kEntThread = kEntMulti - 1u, kMaxEpoch = 31;

__device__ __forceinline__ uint32_t rel_col_cap(uint32_t table_bytes) {  // column masks (words)
    return min(4096u, (table_bytes / 20u) & ~63u);
}
__device__ __forceinline__ uint32_t rel_entry_bytes(uint32_t table_bytes) {  // a multiple of 256
    return table_bytes - 4u * rel_col_cap(table_bytes);
}

// x mod M for x < 2^31 by a reciprocal multiply: q = floor(x * magic / 2^32)
// with magic = floor((2^32 - 1) / M) is floor(x / M) or one less, so one
// correction gives the remainder (M = 1 included).
__device__ __forceinline__ uint32_t mod_by(uint32_t x, uint32_t M, uint32_t magic) {
    uint32_t r = x - __umulhi(x, magic) * M;
    return r >= M ? r - M : r;
}

// The word at shared-memory address a &= v, returning the old value, with
// acquire-release order at CTA scope: the caller's earlier shared-memory
// writes are visible to any thread whose atomic on the word comes later, and
// its later reads see every write made before the atomics that precede its
// own.
__device__ __forceinline__ uint32_t and_acq_rel(uint32_t a, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.cta.shared::cta.and.b32 %0, [%1], %2;" : "=r"(old) : "r"(a), "r"(v) : "memory");
    return old;
}

// Per-program setup by warp 1: the program record, candidate pairs, table
// rows and their maps, window size.
__device__ void rel_setup(RelProg &sm, const DevProg *gp, uint32_t mask, uint32_t table_bytes) {
    const uint32_t lane = threadIdx.x & 31u;
    {
        // every load in flight before the first store
        constexpr uint32_t kN16 = sizeof(DevProg) / 16, kPer = (kN16 + 31u) / 32u;
        const uint4 *src = reinterpret_cast<const uint4 *>(gp);
        uint4 *d4 = reinterpret_cast<uint4 *>(&sm.prog);
        uint4 v[kPer];
#pragma unroll
        for (uint32_t k = 0; k < kPer; ++k)
            if (lane + 32u * k < kN16) v[k] = src[lane + 32u * k];
#pragma unroll
        for (uint32_t k = 0; k < kPer; ++k)
            if (lane + 32u * k < kN16) d4[lane + 32u * k] = v[k];
    }
    __syncwarp();
    const DevProg &P = sm.prog;
    const uint32_t S = P.n_stmts;
    const uint32_t gaps = gap_mask(P, mask);
    uint32_t pend = 0;
    if (lane < S) {
        const bool w = (P.write_mask >> lane) & 1u;
        pend = range_mask(lane, S) & phase_of(lane, gaps, S) & (w ? kRelAllOnes : P.write_mask);
    }
    sm.pend[lane] = pend;
    // pattern pairs pending (lower representative -> higher); when every
    // instance is its own representative they are the pending pairs
    uint32_t rp = pend;
    if (!__all_sync(0xFFFFFFFFu, P.rep[lane] == lane)) {
        sm.rep_conf[lane] = 0;
        __syncwarp();
        for (uint32_t t = pend; t; t &= t - 1u) {
            const uint32_t ri = P.rep[lane], rj = P.rep[__ffs(t) - 1u];
            atomicOr(&sm.rep_conf[min(ri, rj)], 1u << max(ri, rj));
        }
        __syncwarp();
        rp = sm.rep_conf[lane];
    }
    {
        // Pairs decided without the table: a map injective on the block's
        // threads gives distinct threads distinct words, so two instances
        // with that one map (whatever their guards; the self pair included)
        // never race.  Dropping them lets a row retire once its other pairs
        // are found.
        const DevStmt &st = P.stmts[lane];
        const unsigned long long key = st.kind == GR_PERM
                                           ? (1ull << 63) | st.perm_off
                                           : ((unsigned long long)st.am << 32) | st.bm;
        const uint32_t same = __match_any_sync(0xFFFFFFFFu, key);
        if (lane < S && (st.flags & kStmtInjective)) rp &= ~same;
    }
    uint32_t involved = rp | (rp ? (1u << lane) : 0u);
    involved = __reduce_or_sync(0xFFFFFFFFu, involved);
    const bool keep = (involved >> lane) & 1u;
    const uint32_t row = __popc(involved & ((1u << lane) - 1u));
    const uint32_t R = __popc(involved);
    // open pairs in both directions: the representative's candidates plus the
    // representatives that have it as a candidate (the transpose, a ballot
    // per representative), all in statement bits
    uint32_t sym = rp;
    for (uint32_t t = involved; t; t &= t - 1u) {
        const uint32_t l = __ffs(t) - 1u;
        const uint32_t col = __ballot_sync(0xFFFFFFFFu, (rp >> l) & 1u);
        if (lane == l) sym |= col;
    }
    // rows in increasing representative order, so that a representative mask
    // compresses to a row mask by bit extraction
    if (keep) {
        const DevStmt &st = P.stmts[lane];
        sm.cand[row] = pext32(rp, involved);
        sm.open[row] = pext32(sym, involved);
        sm.row_map[row] = make_uint4(st.am, st.bm, st.kind == GR_PERM ? st.perm_off : kRelAllOnes,
                                     (uint32_t)st.gk | ((uint32_t)st.gr << 16));
        sm.row_nact[row] = guard_count(P.threads, st.gk, st.gr);
    }
    const uint32_t inj =
        __reduce_or_sync(0xFFFFFFFFu, keep && (P.stmts[lane].flags & kStmtInjective) ? 1u << row : 0u);
    if (lane == 0) {
        const uint32_t M = P.m_shared;
        // R rows of W + 2 u16 entries (the extra word shifts each row by one
        // bank) in the entry area, W u32 column masks in the mask area
        uint32_t W = 0, n_win = 0;
        if (R) {
            const uint32_t cap = rel_col_cap(table_bytes), ent = rel_entry_bytes(table_bytes);
            const uint32_t per = ent / (2u * R);
            const uint32_t wmax = per > 2u ? min(cap, (per - 2u) & ~63u) : 0u;
            const uint32_t mr = (M + 63u) & ~63u;
            W = min(wmax, mr);
            n_win = W ? (M + W - 1u) / W : 0u;
        }
        sm.involved = involved;
        sm.M = M;
        sm.Mmagic = 0xFFFFFFFFu / M;
        sm.n_rows = R;
        sm.W = W;
        sm.pitch = W + 2u;
        sm.n_win = n_win;
        sm.inj_rows = inj;
        sm.bad = (R && W == 0) ? 1u : 0u;
        sm.mask = mask;
    }
}

// Install and check the accesses of the words [lo, lo + W): unit u (one per
// worker warp at a time) covers table row q = u mod R, active threads
// 64 c .. 64 c + 63 of the row with c = u / R (R rows, cpr chunks of 64
// threads each; a guarded row's active threads are its guard's residue
// class, numbered in order); lane l takes active threads 64 c + l and
// 64 c + 32 + l.  (q, c) steps from unit
// to unit without a division, and every reduction is a reciprocal multiply.
// When the array takes several windows, an affine unit whose 64 words (a
// run of 63 am + 1 positions, cyclically) miss the window is skipped whole.
// A unit of a row with no open pair is skipped too: no other row needs its
// entries.
constexpr uint32_t kRelTPL = 2;  // threads per lane of an install unit

struct RelAccess {
    uint32_t t, a;
    bool on;  // thread active and its word in the window
};

// One access: the thread into its row's entry, then the rows already at the
// word compared with it; returns the partners it conflicts with.
__device__ __forceinline__ uint32_t rel_access(RelProg &sm, uint16_t *tab, uint32_t colrows_s, uint32_t lo,
                                               uint32_t qq, uint32_t openq, bool injective, RelAccess x,
                                               uint32_t epoch) {
    const uint32_t qbit = 1u << qq, pitch = sm.pitch, t = x.t;
    const uint32_t tag = epoch << kEntEpochShift;
    const uint32_t col = swizzle(x.a - lo);
    uint16_t *e = tab + (size_t)qq * pitch + col;
    bool multi = false;  // a second thread of this row on the word
    if (injective) {
        *e = (uint16_t)(tag | t);
    } else {
        // the first thread of this window installs itself over the stale
        // entry it read; any other finds this window's epoch
        const uint16_t old = *(volatile uint16_t *)e;
        if ((uint32_t)(old >> kEntEpochShift) == epoch || atomicCAS(e, old, (uint16_t)(tag | t)) != old) {
            *e = (uint16_t)(tag | kEntMulti);
            multi = true;
        }
    }
    // the rows present before this access (their bits are clear)
    uint32_t part = ~and_acq_rel(colrows_s + 4u * col, ~qbit) & openq & ~qbit;
    // two threads of this row here: the self pair, and a thread other than
    // each partner's
    if (multi) return (openq & qbit) | part;
    uint32_t found = 0;
    for (; part; part &= part - 1u) {
        const uint32_t j = __ffs(part) - 1u;
        // another thread, or MULTI (bit 10, above every thread)
        if ((tab[(size_t)j * pitch + col] & (kEntMulti | kEntThread)) != t) found |= 1u << j;
    }
    return found;
}

template <uint32_t NT>
__device__ __forceinline__ void rel_install(RelProg &sm, const uint16_t *__restrict__ perm, uint16_t *tab,
                                            uint32_t *colrows, uint32_t lo, uint32_t epoch) {
    constexpr uint32_t NWK = NT / 32 - kRelCtl;  // worker warps
    const uint32_t lane = threadIdx.x & 31u, wk = (threadIdx.x >> 5) - kRelCtl;
    const uint32_t T = sm.prog.threads, M = sm.M, magic = sm.Mmagic, W = sm.W;
    // every row gets the chunks of the unguarded width; a guarded row's
    // later chunks are empty and skipped at once
    const uint32_t cpr = (T + 32u * kRelTPL - 1u) / (32u * kRelTPL), n_units = sm.n_rows * cpr, inj = sm.inj_rows;
    const bool windows = sm.n_win > 1;
    // units chunk by chunk across the rows (u = c R + q): a pair that
    // conflicts near the low threads is found early, its rows retire, and
    // their later chunks are skipped
    const uint32_t R = sm.n_rows, dc = NWK / R, dq = NWK - dc * R;
    uint32_t c = wk / R, q = wk - c * R;
    for (uint32_t u = wk; u < n_units; u += NWK) {  // uniform over the warp
        const uint32_t tb = c * (32u * kRelTPL), qq = q;
        q += dq;
        c += dc;
        if (q >= R) {
            q -= R;
            ++c;
        }
        const uint32_t nq = sm.row_nact[qq];
        if (tb >= nq) continue;  // past the row's active threads
        const uint32_t openq = *(volatile uint32_t *)&sm.open[qq];
        if (!openq) continue;  // every pair of this row is decided
        const uint4 mp = sm.row_map[qq];
        const uint32_t am = mp.x, bm = mp.y, po = mp.z, gk = mp.w & 0xFFFFu;
        // the unit's threads are the row's active ones: t = gr + g i, i in
        // [tb, tb + 64) below nq (g = gk, or 1 with no guard)
        const uint32_t g = gk ? gk : 1u, gr = mp.w >> 16;
        if (windows && po == kRelAllOnes) {
            // am (gr + g tb) < 2^16 2^10: the unit's first word; its words step
            // by am g mod M, a run of 63 steps
            const uint32_t start = mod_by(am * (gr + g * tb) + bm, M, magic);
            const uint32_t step = mod_u32(am * g, M, magic);
            if (step * (32u * kRelTPL - 1u) + 1u < M) {
                const uint32_t d = lo >= start ? lo - start : lo + M - start;  // (lo - start) mod M
                const uint32_t e = start >= lo ? start - lo : start + M - lo;  // (start - lo) mod M
                if (d > step * (32u * kRelTPL - 1u) && e >= W) continue;
            }
        }
        RelAccess x[kRelTPL];
#pragma unroll
        for (uint32_t h = 0; h < kRelTPL; ++h) {
            const uint32_t i = tb + 32u * h + lane;
            const bool on = i < nq;
            const uint32_t t = on ? gr + g * i : 0u;  // < T
            uint32_t a;
            if (po != kRelAllOnes) {
                // t + bm < 2^10 + 2^16
                a = on ? (uint32_t)__ldg(perm + po + mod_by(t + bm, M, magic)) : 0u;
            } else {
                // am, bm < M <= 2^16, t < 2^10: am t + bm < 2^27
                a = mod_by(am * t + bm, M, magic);
            }
            x[h].t = t;
            x[h].a = a;
            x[h].on = on && a - lo < W;
        }
        const bool injective = (inj >> qq) & 1u;
        const uint32_t colrows_s = (uint32_t)__cvta_generic_to_shared(colrows);
        uint32_t found = 0;
#pragma unroll
        for (uint32_t h = 0; h < kRelTPL; ++h)
            if (x[h].on) found |= rel_access(sm, tab, colrows_s, lo, qq, openq, injective, x[h], epoch);
        found = __reduce_or_sync(0xFFFFFFFFu, found);
        if (found) {  // uniform: close the pairs in both directions
            const uint32_t qbit = 1u << qq;
            if (lane == 0) atomicAnd(&sm.open[qq], ~found);
            if (((found & ~qbit) >> lane) & 1u) atomicAnd(&sm.open[lane], ~qbit);
        }
    }
}

// The window's column masks back to empty (all ones), in 16-byte stores (W
// is a multiple of 64 and the mask area 256-byte aligned).
template <uint32_t NT>
__device__ __forceinline__ void rel_reset(const RelProg &sm, uint32_t *colrows) {
    uint4 *c4 = reinterpret_cast<uint4 *>(colrows);
    for (uint32_t i = threadIdx.x - 32u * kRelCtl; i < sm.W / 4u; i += NT - 32u * kRelCtl)
        c4[i] = make_uint4(kRelAllOnes, kRelAllOnes, kRelAllOnes, kRelAllOnes);
}

// The entry area back to epoch 0 (every entry empty), before the epochs wrap.
template <uint32_t NT>
__device__ __forceinline__ void rel_clear_entries(uint16_t *tab, uint32_t table_bytes) {
    uint4 *t4 = reinterpret_cast<uint4 *>(tab);
    for (uint32_t i = threadIdx.x - 32u * kRelCtl; i < rel_entry_bytes(table_bytes) / 16u; i += NT - 32u * kRelCtl)
        t4[i] = make_uint4(0u, 0u, 0u, 0u);
}

// The program's witness rows (race_intra; one array per block, so no
// cross-block pairs) from the row conflicts, and under a mask its divergent
// slots and pair count.  Warp 0.
__device__ void rel_output(RelProg &sm, gr_witnesses *dst, bool with_mask, uint32_t *done) {
    const uint32_t lane = threadIdx.x & 31u;
    const DevProg &P = sm.prog;
    const uint32_t involved = sm.involved, p = sm.p;
    uint32_t rc = 0;
    if ((involved >> lane) & 1u) {
        const uint32_t row = __popc(involved & ((1u << lane) - 1u));
        rc = pdep32(sm.cand[row] & ~sm.open[row], involved);
    }
    uint32_t rows;
    if (__all_sync(0xFFFFFFFFu, P.rep[lane] == lane)) {
        rows = sm.pend[lane] & rc;  // every instance its own representative
    } else {
        sm.rep_conf[lane] = rc;
        __syncwarp();
        rows = 0;
        for (uint32_t t = sm.pend[lane]; t; t &= t - 1u) {
            const uint32_t j = __ffs(t) - 1u;
            const uint32_t ri = P.rep[lane], rj = P.rep[j];
            if ((sm.rep_conf[min(ri, rj)] >> max(ri, rj)) & 1u) rows |= 1u << j;
        }
    }
    gr_witnesses &wo = dst[p];
    wo.race_intra[lane] = rows;
    wo.race_inter[lane] = 0u;
    uint32_t dv = 0;
    unsigned long long pairs = 0;
    if (with_mask) {
        const uint32_t mask = sm.mask;
        dv = diverge_warp(P, mask, lane);
        const uint32_t S = P.n_stmts, gaps = gap_mask(P, mask);
        sm.nact[lane] = lane < S ? guard_count(P.threads, P.stmts[lane].gk, P.stmts[lane].gr) : 0u;
        __syncwarp();
        for (uint32_t idx = lane; idx < S * S; idx += 32u) {
            const uint32_t i = idx / S, j = idx - i * S;
            if (j < i || (gaps & range_mask(i, j))) continue;
            uint64_t same, cross;
            pair_count(P, sm.nact, i, j, same, cross);
            pairs += same;
        }
        pairs = warp_sum_u64(pairs);
    }
    if (lane == 0) {
        wo.diverge = dv;
        wo.n_stmts = P.n_stmts;
        wo.access_pairs = pairs;
    }
    if (done) {
        // the rows before the flag, for the warps of other CTAs that wait on it
        __threadfence();
        __syncwarp();
        if (lane == 0) *(volatile uint32_t *)&done[p] = 1u;
    }
    __syncwarp();
}

// Warp 1's place in the work queue, kept two programs ahead so
// that neither the queue's atomic nor the order table's load is waited on:
// `p_next` is the program of the next fetch (its order entry was loaded a
// fetch ago), `item_next` the queue item after it (lane 0's atomic result,
// read a fetch later).
struct RelQueue {
    uint32_t p_next, item_next;
};

__device__ __forceinline__ uint32_t rel_grab(uint32_t *ctrl) {
    return (threadIdx.x & 31u) == 0 ? atomicAdd(&ctrl[2], 1u) : 0u;
}

__device__ __forceinline__ RelQueue rel_queue_start(const ArenaView &V, uint32_t *ctrl, uint32_t n_fast) {
    RelQueue Q;
    const uint32_t item = __shfl_sync(0xFFFFFFFFu, rel_grab(ctrl), 0);
    Q.p_next = item < n_fast ? V.order[item] : kRelAllOnes;
    Q.item_next = rel_grab(ctrl);
    return Q;
}

// Warp 1: the next program from the queue into `b`, set up.
__device__ __forceinline__ void rel_fetch(RelProg &b, RelQueue &Q, const ArenaView &V, uint32_t *ctrl,
                                          uint32_t n_fast, const uint32_t *masks, uint32_t table_bytes) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t p = Q.p_next;
    const uint32_t item = __shfl_sync(0xFFFFFFFFu, Q.item_next, 0);
    Q.p_next = item < n_fast ? V.order[item] : kRelAllOnes;
    if (item < n_fast) Q.item_next = rel_grab(ctrl);  // once past the end, no further atomics
    if (p != kRelAllOnes) rel_setup(b, &V.progs[p], masks ? masks[p] : 0u, table_bytes);
    // the record of the program after it into L2 (its order entry has
    // arrived by now), so that the next setup's loads do not wait on DRAM
    if (Q.p_next != kRelAllOnes && lane < (sizeof(DevProg) + 127u) / 128u) {
        const char *line = reinterpret_cast<const char *>(&V.progs[Q.p_next]) + 128u * lane;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(line));
    }
    __syncwarp();
    if (lane == 0) b.p = p;
    __syncwarp();
}

// The relation kernel.  FUSED: once the relation queue is empty and this
// CTA's programs are written out, every warp runs Algorithm 1 for programs
// from the loop queue (one warp each, as the loop kernel does), its record in
// the freed table; a program's loop starts after its relation's done flag,
// set by the CTA that took it (a CTA that is running: it took the item), so
// the wait ends; it is bounded all the same, and running out sets the error
// word.
template <uint32_t NT, uint32_t MINB, bool FUSED>
__global__ void __launch_bounds__(NT, MINB)
    k_relation(const uint8_t *__restrict__ arena, uint32_t n, const uint32_t *__restrict__ masks,
               uint8_t *__restrict__ scratch, uint64_t scratch_bytes, gr_witnesses *__restrict__ out,
               uint32_t table_bytes, gr_options opts, gr_repair_result *__restrict__ results) {
    extern __shared__ uint4 rel_raw[];
    // a dependent launch (the loop kernel) may be placed as this kernel's
    // CTAs exit; it waits for this kernel's completion before reading
    // anything it writes.  Every CTA is resident from the start (the grid
    // is at most the SMs' capacity), so nothing waits on the dependent.
    asm volatile("griddepcontrol.launch_dependents;");
    RelSmem &sm = *reinterpret_cast<RelSmem *>(rel_raw);
    uint16_t *tab = reinterpret_cast<uint16_t *>(reinterpret_cast<uint8_t *>(rel_raw) + kRelFixed);
    const ArenaView V = view(arena);
    uint32_t *ctrl = reinterpret_cast<uint32_t *>(scratch);
    if (!launch_matches(V, n, scratch_bytes)) {
        if (threadIdx.x == 0) atomicOr(&ctrl[1], kErrArgs);
        return;
    }
    gr_witnesses *dst = out ? out : reinterpret_cast<gr_witnesses *>(scratch + V.h->scratch_rel_off);
    uint32_t *done = FUSED ? reinterpret_cast<uint32_t *>(scratch + rel_flags_off(V.h->scratch_rel_off, n)) : nullptr;
    const uint32_t n_fast = V.h->n_fast;
    const uint32_t warp = threadIdx.x >> 5;
    constexpr uint32_t kWorkers = NT - 32u * kRelCtl;
    static_assert(NT / 32 > kRelCtl, "the relation kernel needs a worker warp");
    // entries at epoch 0 (empty), column masks empty (all ones)
    uint32_t *colrows = reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(tab) + rel_entry_bytes(table_bytes));
    for (uint32_t i = threadIdx.x; i < table_bytes / 16u; i += NT) {
        const uint32_t v = i < rel_entry_bytes(table_bytes) / 16u ? 0u : kRelAllOnes;
        reinterpret_cast<uint4 *>(tab)[i] = make_uint4(v, v, v, v);
    }
    uint32_t epoch = 0;  // the workers' window count, modulo the epochs
    RelQueue Q{kRelAllOnes, 0u};
    if (warp == 1) {
        Q = rel_queue_start(V, ctrl, n_fast);
        rel_fetch(sm.buf[0], Q, V, ctrl, n_fast, masks, table_bytes);
    } else if (threadIdx.x == 0) {
        sm.buf[1].p = kRelAllOnes;
        sm.buf[2].p = kRelAllOnes;
    }
    __syncthreads();
    for (uint32_t k = 0, ic = 0;; ++k, ic = ic == 2u ? 0u : ic + 1u) {  // ic = k mod 3
        RelProg &cur = sm.buf[ic], &nxt = sm.buf[ic == 2u ? 0u : ic + 1u], &prv = sm.buf[ic == 0u ? 2u : ic - 1u];
        const bool have_cur = cur.p != kRelAllOnes, have_prv = prv.p != kRelAllOnes;
        if (!have_cur && !have_prv) break;  // uniform
        if (warp == 0) {
            // program k-1 out (its buffer is set up again in the next round)
            if (have_prv) rel_output(prv, dst, masks != nullptr, done);
        } else if (warp == 1) {
            // program k+1 into the third buffer
            if (have_cur) {
                rel_fetch(nxt, Q, V, ctrl, n_fast, masks, table_bytes);
            } else if ((threadIdx.x & 31u) == 0) {
                nxt.p = kRelAllOnes;
            }
        } else if (have_cur) {
            const uint32_t R = cur.n_rows, W = cur.W, n_win = cur.n_win;
            if (cur.bad) {
                if (threadIdx.x == 32u * kRelCtl) atomicOr(&ctrl[1], kErrTableTooSmall);
            } else if (R) {
                for (uint32_t w = 0; w < n_win; ++w) {
                    if (++epoch > kMaxEpoch) {  // uniform over the workers
                        rel_clear_entries<NT>(tab, table_bytes);
                        asm volatile("bar.sync 1, %0;" ::"r"(kWorkers) : "memory");
                        epoch = 1;
                    }
                    rel_install<NT>(cur, V.perm, tab, colrows, w * W, epoch);
                    asm volatile("bar.sync 1, %0;" ::"r"(kWorkers) : "memory");
                    rel_reset<NT>(cur, colrows);
                    // the last window's reset is ordered before the next
                    // program's install by the CTA barrier below
                    if (w + 1u < n_win) asm volatile("bar.sync 1, %0;" ::"r"(kWorkers) : "memory");
                }
            }
        }
        __syncthreads();
    }
    if constexpr (FUSED) {
        // the pipeline has drained: the table area holds a loop record per warp
        const uint32_t lane = threadIdx.x & 31u;
        LoopWarpSimple &lw = *reinterpret_cast<LoopWarpSimple *>(reinterpret_cast<uint8_t *>(tab) +
                                                                 warp_smem<LoopWarpSimple>() * warp);
        const uint32_t max_iters =
            opts.max_iters == 0 ? GR_MAX_ITERS : min(opts.max_iters, (uint32_t)GR_MAX_ITERS);
        const uint64_t deadline_ns = opts.deadline_us * 1000ull;
        constexpr uint32_t kWaitLimit = 1u << 23;  // about half a second of 64 ns sleeps
        for (;;) {
            uint32_t item = 0;
            if (lane == 0) item = atomicAdd(&ctrl[3], 1u);
            item = __shfl_sync(0xFFFFFFFFu, item, 0);
            if (item >= n) break;
            const uint32_t p = V.order[item];
            uint32_t ok = 1;
            if (lane == 0) {
                for (uint32_t it = 0; *(volatile uint32_t *)&done[p] == 0u; ++it) {
                    if (it >= kWaitLimit) {
                        atomicOr(&ctrl[1], kErrStall);
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
                __threadfence();  // the relation rows after the flag
            }
            if (!__shfl_sync(0xFFFFFFFFu, ok, 0)) return;
            loop_program(lw, V, p, dst, opts, max_iters, deadline_ns, results, ctrl);
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

// CTA shapes of the relation kernel: {threads, CTAs per SM}.
const LaunchShape kRelShapes[kNumRelShapes] = {{512, 3}, {256, 4}, {512, 2}, {1024, 1}, {256, 6}, {128, 8}};

template <typename F>
static cudaError_t rel_set_smem(F *f, uint32_t max_dynamic_smem) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, (const void *)f);
    if (e != cudaSuccess) return e;
    const size_t cap = max_dynamic_smem > a.sharedSizeBytes ? max_dynamic_smem - a.sharedSizeBytes : 0;
    return cudaFuncSetAttribute((const void *)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
}

cudaError_t configure_relation(uint32_t max_dynamic_smem) {
    cudaError_t e;
    if ((e = rel_set_smem(k_relation<512, 3, false>, max_dynamic_smem)) != cudaSuccess) return e;
    if ((e = rel_set_smem(k_relation<256, 4, false>, max_dynamic_smem)) != cudaSuccess) return e;
    if ((e = rel_set_smem(k_relation<512, 2, false>, max_dynamic_smem)) != cudaSuccess) return e;
    if ((e = rel_set_smem(k_relation<1024, 1, false>, max_dynamic_smem)) != cudaSuccess) return e;
    if ((e = rel_set_smem(k_relation<256, 6, false>, max_dynamic_smem)) != cudaSuccess) return e;
    if ((e = rel_set_smem(k_relation<128, 8, false>, max_dynamic_smem)) != cudaSuccess) return e;
    if ((e = rel_set_smem(k_relation<512, 2, true>, max_dynamic_smem)) != cudaSuccess) return e;
    return cudaSuccess;
}

bool relation_loop_fits(uint32_t table_bytes) {
    return (size_t)table_bytes >= warp_smem<LoopWarpSimple>() * (512u / 32u);
}

cudaError_t launch_relation_loop(const void *d_arena, uint32_t n, void *d_scratch, uint64_t scratch_bytes,
                                 const gr_options &opts, gr_repair_result *d_out, RelCfg cfg, cudaStream_t st) {
    const size_t smem = kRelFixed + cfg.table_bytes;
    k_relation<512, 2, true><<<cfg.grid, 512, smem, st>>>(static_cast<const uint8_t *>(d_arena), n, nullptr,
                                                         static_cast<uint8_t *>(d_scratch), scratch_bytes, nullptr,
                                                         cfg.table_bytes, opts, d_out);
    return cudaGetLastError();
}

cudaError_t launch_relation(const void *d_arena, uint32_t n, const uint32_t *d_masks, void *d_scratch,
                            uint64_t scratch_bytes, gr_witnesses *d_out, RelCfg cfg, cudaStream_t st) {
    const uint8_t *a = static_cast<const uint8_t *>(d_arena);
    uint8_t *sc = static_cast<uint8_t *>(d_scratch);
    const size_t smem = kRelFixed + cfg.table_bytes;
    switch (cfg.shape) {
        case 1: k_relation<256, 4, false><<<cfg.grid, 256, smem, st>>>(a, n, d_masks, sc, scratch_bytes, d_out, cfg.table_bytes, gr_options{}, nullptr); break;
        case 2: k_relation<512, 2, false><<<cfg.grid, 512, smem, st>>>(a, n, d_masks, sc, scratch_bytes, d_out, cfg.table_bytes, gr_options{}, nullptr); break;
        case 3: k_relation<1024, 1, false><<<cfg.grid, 1024, smem, st>>>(a, n, d_masks, sc, scratch_bytes, d_out, cfg.table_bytes, gr_options{}, nullptr); break;
        case 4: k_relation<256, 6, false><<<cfg.grid, 256, smem, st>>>(a, n, d_masks, sc, scratch_bytes, d_out, cfg.table_bytes, gr_options{}, nullptr); break;
        case 5: k_relation<128, 8, false><<<cfg.grid, 128, smem, st>>>(a, n, d_masks, sc, scratch_bytes, d_out, cfg.table_bytes, gr_options{}, nullptr); break;
        default: k_relation<512, 3, false><<<cfg.grid, 512, smem, st>>>(a, n, d_masks, sc, scratch_bytes, d_out, cfg.table_bytes, gr_options{}, nullptr); break;
    }
    return cudaGetLastError();
}

}  // namespace gr
