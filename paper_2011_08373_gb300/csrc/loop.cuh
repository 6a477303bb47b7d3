// loop.cuh — the repair loop of Algorithm 1 (Section 2.4), one warp per
// program, over each program's conflict relation.
//
// The relation (race_intra / race_inter rows of the check under the empty
// mask: every instance pair with a write that conflicts somewhere, same-block
// or across blocks) is computed once per program by the check kernels.  A
// check under any mask m then needs no further table pass: a witness (i, j)
// exists under m iff the pair conflicts and no enabled barrier runs between
// i and j (for a cross-block pair, no enabled grid barrier), i.e. iff m
// misses the pair's exact clause (the slots whose barriers run in gaps
// i..j-1).  So Verify(m) = the relation restricted to the phases of m, plus
// the divergent enabled slots, both exact; the loop below is Algorithm 1 on
// those witnesses:
//   check    — witnesses under the proposal; a clean proposal ends the loop
//              (the mhs strategy first asks the exact solver once more);
//   clauses  — each witness's clause (GenerateClause), kept as a sorted set;
//              a divergent slot becomes a negative unit clause (forbidden);
//   solve    — the next proposal: the minimum-weight hitting set with ties
//              to the lowest mask (Solve as weighted MaxSAT), or Johnson's
//              greedy set under the mhs strategy, the exact solve as its
//              fallback;
// until a proposal is clean (repaired), no hitting set exists (unrepairable),
// or the iteration cap or the deadline is reached.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "device.cuh"

namespace gr {

// Two builds of the kernel: the general one (four warps per CTA, clause
// buffers for the largest clause sets) and, for batches of simple programs
// (straight-line, shared array only: every clause an interval [i, j), at
// most 25 * 24 / 2 + 1 of them, no sort, at most 25 row minima), one with
// small buffers and twice the warps per CTA, so that more programs are in
// flight per SM.
constexpr uint32_t kListCap = 704;        // >= GR_MAX_CLAUSES (656), a multiple of 32
constexpr uint32_t kSimpleListCap = 320;  // >= 301 interval clauses
constexpr uint32_t kSimpleScratch = 64;   // >= 32 kept clauses (the register subsumption)
constexpr uint32_t kSimpleWarps = 8;

template <uint32_t CAPC, uint32_t CAPA>
struct LoopWarpT {
    static constexpr uint32_t kCapC = CAPC, kCapA = CAPA;
    DevProg prog;
    uint32_t traj[GR_MAX_ITERS];
    uint32_t tg[GR_MAX_ITERS], tgg[GR_MAX_ITERS];  // gaps of each checked mask (all slots / grid slots)
    uint32_t cl[CAPC];  // the clause set, sorted
    uint32_t A[CAPA];   // scratch: candidate clauses, filtered clauses, kept high parts
    uint32_t B[CAPA];   // scratch: sort buffer, size-ordered clauses, kept low patterns
    uint32_t nhi[32], nlo[32];
    uint32_t wc[32], wlo[32], lb[34];
    uint32_t w4[8][16];     // weight of each nibble of the high part
    uint32_t size_at[34];
    unsigned long long pk[32];  // instance fields for the pair count: guard k, r, active threads, write, space
};

using LoopWarp = LoopWarpT<kListCap, kListCap>;
using LoopWarpSimple = LoopWarpT<kSimpleListCap, kSimpleScratch>;
constexpr uint32_t kLoopWarps = kLoopThreads / 32;  // programs in flight per CTA (one per warp)

template <class LW>
constexpr size_t warp_smem() { return (sizeof(LW) + 15) / 16 * 16; }
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
    for (uint32_t o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xFFFFFFFFu, v, o);
        v = u < v ? u : v;
    }
    return v;
}

// ---- sorted sets of clauses --------------------------------------------------

// Sort src[0..m) ascending into dst (src is used as scratch); m <= kListCap.
// Runs of 32 are sorted in registers (bitonic network over the lanes), then
// merged pairwise: each element's place in the merged run is its rank in its
// own run plus the number of elements of the other run before it (ties:
// the left run first).
__device__ inline uint32_t *warp_sort(uint32_t *src, uint32_t *dst, uint32_t m) {
    const uint32_t lane = lane_id();
    for (uint32_t base = 0; base < m; base += 32u) {
        uint32_t x = base + lane < m ? src[base + lane] : 0xFFFFFFFFu;
        for (uint32_t k = 2; k <= 32; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, j);
                const bool up = ((lane & k) == 0);
                const bool lower = (lane & j) == 0;
                const uint32_t lo = min(x, y), hi = max(x, y);
                x = (lower == up) ? lo : hi;
            }
        }
        if (base + lane < m) src[base + lane] = x;
    }
    __syncwarp();
    uint32_t *a = src, *b = dst;
    for (uint32_t w = 32; w < m; w <<= 1) {
        for (uint32_t i = lane; i < m; i += 32u) {
            const uint32_t run = i / (2u * w) * (2u * w);
            const uint32_t mid = min(run + w, m), end = min(run + 2u * w, m);
            const uint32_t x = a[i];
            uint32_t pos;
            if (i < mid) {  // left run: elements of the right run strictly below x
                uint32_t lo = mid, hi = end;
                while (lo < hi) {
                    const uint32_t md = (lo + hi) >> 1;
                    if (a[md] < x) lo = md + 1u; else hi = md;
                }
                pos = i + (lo - mid);
            } else {  // right run: elements of the left run not above x
                uint32_t lo = run, hi = mid;
                while (lo < hi) {
                    const uint32_t md = (lo + hi) >> 1;
                    if (a[md] <= x) lo = md + 1u; else hi = md;
                }
                pos = (i - mid) + lo;
            }
            b[pos] = x;
        }
        __syncwarp();
        uint32_t *t = a;
        a = b;
        b = t;
    }
    if (a != dst) {
        for (uint32_t i = lane; i < m; i += 32u) dst[i] = a[i];
        __syncwarp();
    }
    return dst;
}

// Distinct values of the sorted src[0..m) into dst, in order; returns how many.
__device__ inline uint32_t warp_unique(const uint32_t *src, uint32_t m, uint32_t *dst) {
    const uint32_t lane = lane_id();
    uint32_t n = 0;
    for (uint32_t base = 0; base < m; base += 32u) {
        const uint32_t i = base + lane;
        const bool keep = i < m && (i == 0 || src[i] != src[i - 1u]);
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
        if (keep) dst[n + __popc(bal & ((1u << lane) - 1u))] = src[i];
        n += __popc(bal);
    }
    __syncwarp();
    return n;
}

// The clause set from the witnesses seen so far (GenerateClause): a same-block
// witness (i, j) gives the slots whose barriers run in gaps i..j-1, a
// cross-block witness the grid slots among them.  Lane i holds row i of both.
// Returns the number of distinct clauses, sorted in lw.cl.
template <class LW>
__device__ uint32_t build_clause_set(LW &lw, uint32_t acc_i, uint32_t acc_x) {
    const DevProg &P = lw.prog;
    const uint32_t lane = lane_id();
    uint32_t m = 0;
    if (!P.general && !__any_sync(0xFFFFFFFFu, acc_x != 0u)) {
        // Without loops or explicit places and without cross-block witnesses
        // the clause of (i, j) is the slot interval [i, j): 2^j - 2^i, all
        // distinct, and in increasing order when sorted by j, then by
        // decreasing i (the values for j lie in [2^(j-1), 2^j)); a
        // same-statement witness gives the empty clause 0, first.
        if (__any_sync(0xFFFFFFFFu, (acc_i >> lane) & 1u)) lw.cl[m++] = 0u;
        const uint32_t rows = __reduce_or_sync(0xFFFFFFFFu, acc_i);
        for (uint32_t t = rows & ~1u; t; t &= t - 1u) {
            const uint32_t j = __ffs(t) - 1u;
            const bool has = lane < j && ((acc_i >> j) & 1u);
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, has);
            if (has) lw.cl[m + __popc(bal >> lane) - 1u] = (1u << j) - (1u << lane);
            m += __popc(bal);
        }
        __syncwarp();
        return m;
    }
    // lane i emits its row's clauses one per round, in increasing j
    uint32_t ti = acc_i, tx = acc_x;
    while (__any_sync(0xFFFFFFFFu, (ti | tx) != 0u)) {
        uint32_t c = 0;
        bool has = false;
        if (ti) {
            const uint32_t j = __ffs(ti) - 1u;
            ti &= ti - 1u;
            c = slots_of_gaps(P, range_mask(lane, j));
            has = true;
        } else if (tx) {
            const uint32_t j = __ffs(tx) - 1u;
            tx &= tx - 1u;
            c = slots_of_gaps(P, range_mask(lane, j)) & P.grid_mask;
            has = true;
        }
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, has);
        if (has) lw.A[m + __popc(bal & ((1u << lane) - 1u))] = c;
        m += __popc(bal);
    }
    __syncwarp();
    if (m == 0) return 0;
    const uint32_t *s = warp_sort(lw.A, lw.B, m);
    return warp_unique(s, m, lw.cl);
}

// ---- Solve: exact minimum-weight hitting set --------------------------------

// Least (weight, mask) with forced <= mask, mask & forbidden == 0, hitting
// every clause of cl[0..n) and containing no negative clause of the
// program.  Ties go to the lowest mask.  Returns false when none exists.
//   1. clauses hit by a forced slot are met; the others lose their forbidden
//      slots (an emptied clause: unsatisfiable);
//   2. in order of size, a clause containing an earlier one is dropped;
//      unit clauses join the forced set; R = the slots left in some clause
//      (any other slot stays off in a minimum);
//   3. the R slots are renumbered in order (so the lowest mask stays the
//      lowest); the five lowest ride in the 32 bits of a word — each clause
//      becomes, per assignment of the high slots, a 32-bit set of low
//      assignments that hit it — and the high slots are enumerated by size
//      (Gosper's order), lanes taking contiguous ranges, stopping at the first
//      size whose lightest member is heavier than the best key found.
template <class LW>
__device__ bool warp_solve(LW &lw, const uint32_t *cl, uint32_t n, uint32_t forced, uint32_t forbidden,
                           uint32_t &mask_out, uint32_t &weight_out) {
    const DevProg &P = lw.prog;
    const uint32_t *w = P.weights;
    const uint32_t lane = lane_id();
    if (forced & forbidden) return false;
    uint32_t n_kept = 0, U = 0, R = 0;
    if (n <= 32u) {
        // one clause per lane, in registers: drop a clause hit by a forced
        // slot, remove forbidden slots (an emptied clause: unsatisfiable),
        // then keep a clause unless another is a strict subset of it or an
        // equal one sits on a lower lane (the same kept set as the size-ordered
        // pass below)
        uint32_t pc = 0;
        bool bad = false;
        if (lane < n) {
            const uint32_t c = cl[lane];
            if (!(c & forced)) {
                pc = c & ~forbidden;
                bad = pc == 0u;
            }
        }
        if (__any_sync(0xFFFFFFFFu, bad)) return false;
        bool keep = pc != 0u;
        for (uint32_t j = 0; j < n; ++j) {
            const uint32_t d = __shfl_sync(0xFFFFFFFFu, pc, j);
            keep = keep && !(d != 0u && (d & ~pc) == 0u && (d != pc || j < lane));
        }
        const bool unit = keep && (pc & (pc - 1u)) == 0u;
        U = __reduce_or_sync(0xFFFFFFFFu, unit ? pc : 0u);
        const bool multi = keep && !unit;
        R = __reduce_or_sync(0xFFFFFFFFu, multi ? pc : 0u);
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, multi);
        if (multi) lw.A[__popc(bal & ((1u << lane) - 1u))] = pc;
        n_kept = __popc(bal);
        __syncwarp();
    } else {
    lw.size_at[lane] = 0;
    if (lane < 2) lw.size_at[32 + lane] = 0;
    __syncwarp();
    bool bad = false;
    for (uint32_t i = lane; i < n; i += 32u) {
        const uint32_t c = cl[i];
        uint32_t pc = 0;
        if (!(c & forced)) {
            pc = c & ~forbidden;
            if (!pc) bad = true;
            else atomicAdd(&lw.size_at[__popc(pc)], 1u);
        }
        lw.A[i] = pc;
    }
    if (__any_sync(0xFFFFFFFFu, bad)) return false;
    __syncwarp();
    // start of each size class (sizes 1..32) by an exclusive scan
    {
        const uint32_t v = lw.size_at[lane + 1u];
        uint32_t incl = v;
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += t;
        }
        __syncwarp();
        lw.size_at[lane + 1u] = incl - v;
        if (lane == 31) lw.size_at[33] = incl;
    }
    __syncwarp();
    const uint32_t n_sorted = lw.size_at[33];
    for (uint32_t i = lane; i < n; i += 32u) {
        const uint32_t pc = lw.A[i];
        if (pc) lw.B[atomicAdd(&lw.size_at[__popc(pc)], 1u)] = pc;
    }
    __syncwarp();
    // subsumption, in size order: keep a clause unless an earlier one is a
    // subset of it (of two equal clauses the later one goes)
    for (uint32_t base = 0; base < n_sorted; base += 32u) {
        const uint32_t i = base + lane;
        bool keep = false, unit = false;
        uint32_t c = 0;
        if (i < n_sorted) {
            c = lw.B[i];
            keep = true;
            for (uint32_t j = 0; j < i && keep; ++j) keep = (lw.B[j] & ~c) != 0u;
            unit = keep && (c & (c - 1u)) == 0u;
        }
        U |= __reduce_or_sync(0xFFFFFFFFu, unit ? c : 0u);
        const bool multi = keep && !unit;
        R |= __reduce_or_sync(0xFFFFFFFFu, multi ? c : 0u);
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, multi);
        if (multi) lw.A[n_kept + __popc(bal & ((1u << lane) - 1u))] = c;
        n_kept += __popc(bal);
    }
    __syncwarp();
    }
    // a kept clause never contains a unit's slot (the unit subsumes it)
    forced |= U;
    // negative clauses: a forbidden slot in one keeps it satisfied; one inside
    // the forced set is violated by every mask; one with a slot outside R is
    // never violated (that slot stays off)
    uint32_t n_negk = 0;
    {
        bool unsat = false, keepn = false;
        uint32_t v = 0;
        if (lane < P.n_neg) {
            const uint32_t N = P.neg[lane];
            if (!(N & forbidden)) {
                v = N & ~forced;
                if (!v) unsat = true;
                else keepn = (v & ~R) == 0u;
            }
        }
        if (__any_sync(0xFFFFFFFFu, unsat)) return false;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keepn);
        if (keepn) lw.nhi[__popc(bal & ((1u << lane) - 1u))] = v;
        n_negk = __popc(bal);
    }
    const uint32_t r = __popc(R);
    const uint32_t L = r < 5 ? r : 5;
    const uint32_t rh = r - L;
    if (r <= 5) {
        // no high part: lane l tries the low assignment l itself (the slots
        // of R in order; l < 2^r), every lane at once
        const uint32_t l = lane;
        bool ok = l < (1u << r);
        uint32_t x = 0, wt = 0;
        if (ok) {
            uint32_t t = R;
            for (uint32_t b = 0; b < r; ++b, t &= t - 1u) {
                if ((l >> b) & 1u) {
                    const uint32_t k = __ffs(t) - 1u;
                    x |= 1u << k;
                    wt += w[k];
                }
            }
            for (uint32_t c = 0; c < n_kept && ok; ++c) ok = (lw.A[c] & x) != 0u;
            for (uint32_t c = 0; c < n_negk && ok; ++c) ok = (lw.nhi[c] & ~x) != 0u;
        }
        // the key compares (weight, compact mask): the compact mask of x is l
        const unsigned long long key = ok ? (((unsigned long long)wt << 32) | l) : ~0ull;
        const unsigned long long best = warp_min_u64(key);
        __syncwarp();
        if (best == ~0ull) return false;
        mask_out = pdep32((uint32_t)best, R) | forced;
        uint32_t wf = (uint32_t)(best >> 32);
        for (uint32_t t = forced; t; t &= t - 1u) wf += w[__ffs(t) - 1u];
        weight_out = wf;
        return true;
    }
    {
        uint32_t v = 0;
        if (lane < r) {  // the weight of R's lane-th slot
            uint32_t t = R;
            for (uint32_t q = 0; q < lane; ++q) t &= t - 1u;
            v = w[__ffs(t) - 1u];
        }
        lw.wc[lane] = v;
    }
    __syncwarp();
    if (n_negk == 0) {
        // Interval clauses: when every kept clause is a run of consecutive
        // slots of R (a straight-line program's same-block clauses are the
        // slots between two instances) and no negative clause is left, the
        // minimum-weight stabbing set comes from a dynamic program over the
        // compact slots, from the highest down.  g[k] = the least key of a
        // set whose lowest member is k and that stabs every clause starting
        // above k: key(k) plus the least g[j], k < j <= B_k (B_k = the least
        // end of a clause starting above k), or key(k) alone when no clause
        // starts above k.  The answer is the least g[k] over k <= the least
        // clause end.  Keys add (weights; disjoint mask bits) and k's bit is
        // below every bit of its continuation, so the least continuation
        // gives the least key: the same (weight, lowest mask) minimum as the
        // enumeration below.
        bool ivl = true;
        for (uint32_t c = lane; c < n_kept; c += 32u) {
            const uint32_t x = pext32(lw.A[c], R);
            const uint32_t lo = __ffs(x) - 1u, y = x >> lo;
            const uint32_t hi = lo + 31u - __clz(y);
            ivl = ivl && (y & (y + 1u)) == 0u;
            lw.B[c] = lo | (hi << 8);
        }
        if (__all_sync(0xFFFFFFFFu, ivl)) {
            __syncwarp();
            uint32_t bk = 0xFFFFFFFFu, H = 0xFFFFFFFFu;
            for (uint32_t c = 0; c < n_kept; ++c) {
                const uint32_t e = lw.B[c], lo = e & 255u, hi = e >> 8;
                H = min(H, hi);
                if (lo > lane && hi < bk) bk = hi;
            }
            // With the weights of R summing below 2^(32 - r), a key packs in
            // 32 bits, (weight << r) | compact mask, in the same order, and
            // each step's minimum is one warp reduction.  The clamp keeps the
            // sum exact: a weight at or above the cap fails the test alone.
            const uint32_t cap = 1u << (32u - r);  // 5 < r <= 32
            const uint32_t sumw = __reduce_add_sync(0xFFFFFFFFu, min(lw.wc[lane], cap));
            if (sumw + 1u < cap) {  // uniform; then r < 32 and no key reaches ~0u
                const uint32_t key32 = lane < r ? (lw.wc[lane] << r) | (1u << lane) : 0u;
                uint32_t g32 = 0xFFFFFFFFu;
                for (int k = (int)r - 1; k >= 0; --k) {  // uniform
                    const uint32_t b = __shfl_sync(0xFFFFFFFFu, bk, k);
                    const uint32_t m = __reduce_min_sync(
                        0xFFFFFFFFu, lane > (uint32_t)k && lane <= b && lane < r ? g32 : 0xFFFFFFFFu);
                    if (lane == (uint32_t)k) g32 = b == 0xFFFFFFFFu ? key32 : (m == 0xFFFFFFFFu ? m : key32 + m);
                }
                const uint32_t best = __reduce_min_sync(0xFFFFFFFFu, lane < r && lane <= H ? g32 : 0xFFFFFFFFu);
                __syncwarp();
                if (best == 0xFFFFFFFFu) return false;
                mask_out = pdep32(best & ((1u << r) - 1u), R) | forced;
                uint32_t wt = best >> r;
                for (uint32_t t = forced; t; t &= t - 1u) wt += w[__ffs(t) - 1u];
                weight_out = wt;
                return true;
            }
            const unsigned long long keyk = ((unsigned long long)lw.wc[lane] << 32) | (1ull << lane);
            unsigned long long g = ~0ull;
            for (int k = (int)r - 1; k >= 0; --k) {  // uniform
                const uint32_t b = __shfl_sync(0xFFFFFFFFu, bk, k);
                const unsigned long long m =
                    warp_min_u64(lane > (uint32_t)k && lane <= b && lane < r ? g : ~0ull);
                if (lane == (uint32_t)k) g = b == 0xFFFFFFFFu ? keyk : (m == ~0ull ? ~0ull : keyk + m);
            }
            const unsigned long long best = warp_min_u64(lane < r && lane <= H ? g : ~0ull);
            __syncwarp();
            if (best == ~0ull) return false;
            mask_out = pdep32((uint32_t)best, R) | forced;
            uint32_t wt = (uint32_t)(best >> 32);
            for (uint32_t t = forced; t; t &= t - 1u) wt += w[__ffs(t) - 1u];
            weight_out = wt;
            return true;
        }
        __syncwarp();
    }
    for (uint32_t k = lane; k < n_kept; k += 32u) {
        const uint32_t c = pext32(lw.A[k], R);
        uint32_t lo = 0;
        for (uint32_t b = 0; b < L; ++b)
            if ((c >> b) & 1u) lo |= low_pattern(b);
        lw.A[k] = c >> L;
        lw.B[k] = lo;
    }
    if (lane < n_negk) {
        const uint32_t c = pext32(lw.nhi[lane], R);
        uint32_t lo = 0xFFFFFFFFu;
        for (uint32_t b = 0; b < L; ++b)
            if ((c >> b) & 1u) lo &= low_pattern(b);
        lw.nhi[lane] = c >> L;
        lw.nlo[lane] = lo;
    }
    {
        uint32_t v = 0;
        for (uint32_t b = 0; b < L; ++b)
            if ((lane >> b) & 1u) v += lw.wc[b];
        lw.wlo[lane] = v;
    }
    for (uint32_t e = lane; e < 8u * 16u; e += 32u) {
        const uint32_t q = e >> 4, nib = e & 15u;
        uint32_t v = 0;
        for (uint32_t b = 0; b < 4; ++b) {
            const uint32_t hb = q * 4u + b;
            if (((nib >> b) & 1u) && hb < rh) v += lw.wc[L + hb];
        }
        lw.w4[q][nib] = v;
    }
    {
        // lb[k] = the sum of the k lightest high weights: each lane puts its
        // weight at its rank (ties by index), then an inclusive scan
        const uint32_t v = lane < rh ? lw.wc[L + lane] : 0u;
        if (lane < rh) {
            uint32_t rank = 0;
            for (uint32_t j = 0; j < rh; ++j) {
                const uint32_t u = lw.wc[L + j];
                rank += (u < v || (u == v && j < lane)) ? 1u : 0u;
            }
            lw.lb[rank + 1u] = v;
        }
        __syncwarp();
        uint32_t acc = lane < rh ? lw.lb[lane + 1u] : 0u;
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, acc, o);
            if (lane >= o) acc += t;
        }
        __syncwarp();
        if (lane < rh) lw.lb[lane + 1u] = acc;
        if (lane == 0) lw.lb[0] = 0;
    }
    __syncwarp();
    const uint32_t VL = L == 5 ? 0xFFFFFFFFu : ((1u << (1u << L)) - 1u);
    unsigned long long best = ~0ull;
    for (uint32_t kh = 0; kh <= rh; ++kh) {
        if (best != ~0ull && (unsigned long long)lw.lb[kh] > (best >> 32)) break;  // uniform
        const uint32_t total = c_binom.v[rh][kh];
        const uint32_t per = (total + 31u) / 32u;
        const uint32_t start = lane * per;
        const uint32_t end = min(total, start + per);
        unsigned long long local = best;
        if (start < end) {
            uint32_t h = unrank_colex(start, kh, rh);
            for (uint32_t idx = start; idx < end; ++idx) {
                uint32_t wh = 0;
#pragma unroll
                for (uint32_t q = 0; q < 8; ++q) wh += lw.w4[q][(h >> (4u * q)) & 15u];
                const uint64_t lwt = local >> 32;
                const bool skip = (uint64_t)wh > lwt || ((uint64_t)wh == lwt && (h << L) > (uint32_t)local);
                if (!skip) {
                    uint32_t F = VL;
                    for (uint32_t c = 0; c < n_kept; ++c) {
                        if ((lw.A[c] & h) == 0) {
                            F &= lw.B[c];
                            if (!F) break;
                        }
                    }
                    if (F)
                        for (uint32_t c = 0; c < n_negk; ++c)
                            if ((lw.nhi[c] & ~h) == 0) F &= ~lw.nlo[c];
                    while (F) {
                        const uint32_t l = __ffs(F) - 1u;
                        F &= F - 1u;
                        const unsigned long long key =
                            ((unsigned long long)(wh + lw.wlo[l]) << 32) | (unsigned long long)((h << L) | l);
                        if (key < local) local = key;
                    }
                }
                if (idx + 1u < end) h = gosper_next(h);
            }
        }
        best = warp_min_u64(local);
    }
    __syncwarp();
    if (best == ~0ull) return false;
    mask_out = pdep32((uint32_t)best, R) | forced;
    uint32_t wt = (uint32_t)(best >> 32);
    for (uint32_t t = forced; t; t &= t - 1u) wt += w[__ffs(t) - 1u];
    weight_out = wt;
    return true;
}

// ---- Solve: the mhs strategy's greedy proposal ------------------------------

// Johnson's greedy hitting set (Section 2.4's mhs strategy): from the forced
// slots, repeatedly take the allowed slot that hits the most clauses not yet
// hit per unit of weight (ratios compared by cross-multiplication, ties to
// the lower slot), then drop, from the highest slot down, every non-forced
// slot whose removal leaves every clause hit.  Returns false when some
// clause has no allowed slot (or a forced slot is forbidden).
template <class LW>
__device__ bool warp_greedy(LW &lw, uint32_t n, uint32_t forced, uint32_t forbidden, uint32_t &mask_out,
                            uint32_t &weight_out) {
    const DevProg &P = lw.prog;
    const uint32_t *w = P.weights;
    const uint32_t lane = lane_id(), n_vars = P.n_slots;
    const uint32_t *cl = lw.cl;
    if (forced & forbidden) return false;
    bool bad = false;
    for (uint32_t i = lane; i < n; i += 32u)
        if (!(cl[i] & forced) && !(cl[i] & ~forbidden)) bad = true;
    if (__any_sync(0xFFFFFFFFu, bad)) return false;
    uint32_t x = forced;
    const uint32_t rounds = (n + 31u) >> 5;
    for (;;) {
        // lane v: the clauses not yet hit that slot v would hit
        uint32_t hits = 0;
        for (uint32_t r = 0; r < rounds; ++r) {
            const uint32_t i = r * 32u + lane;
            const uint32_t m = (i < n && !(cl[i] & x)) ? (cl[i] & ~forbidden) : 0u;
            for (uint32_t vs = __reduce_or_sync(0xFFFFFFFFu, m); vs; vs &= vs - 1u) {
                const uint32_t v = __ffs(vs) - 1u;
                const uint32_t c = __popc(__ballot_sync(0xFFFFFFFFu, (m >> v) & 1u));
                if (lane == v) hits += c;
            }
        }
        uint32_t h = (lane < n_vars && !((x >> lane) & 1u) && !((forbidden >> lane) & 1u)) ? hits : 0u;
        uint32_t wk = lane < n_vars ? w[lane] : 1u, k = lane;
        for (uint32_t o = 16; o > 0; o >>= 1) {
            const uint32_t h2 = __shfl_down_sync(0xFFFFFFFFu, h, o);
            const uint32_t w2 = __shfl_down_sync(0xFFFFFFFFu, wk, o);
            const uint32_t k2 = __shfl_down_sync(0xFFFFFFFFu, k, o);
            const uint64_t a = (uint64_t)h2 * wk, b = (uint64_t)h * w2;
            if (h2 && (!h || a > b || (a == b && k2 < k))) {
                h = h2;
                wk = w2;
                k = k2;
            }
        }
        h = __shfl_sync(0xFFFFFFFFu, h, 0);
        k = __shfl_sync(0xFFFFFFFFu, k, 0);
        if (!h) break;  // every clause is hit
        x |= 1u << k;
    }
    for (int k = (int)n_vars - 1; k >= 0; --k) {
        if (!((x >> k) & 1u) || ((forced >> k) & 1u)) continue;
        const uint32_t y = x & ~(1u << k);
        bool ok = true;
        for (uint32_t i = lane; i < n && ok; i += 32u) ok = (cl[i] & y) != 0;
        if (__all_sync(0xFFFFFFFFu, ok)) x = y;
    }
    uint32_t wt = 0;
    for (uint32_t t = x; t; t &= t - 1u) wt += w[__ffs(t) - 1u];
    mask_out = x;
    weight_out = wt;
    return true;
}

// For the exact solve: one clause per witness row and kind, the one of the
// row's nearest partner.  The clause of (i, j) only grows with j (it holds
// the slots of gaps i..j-1), so it is contained in every other clause of row
// i of its kind, and a mask hits all of them iff it hits this one: the
// minimum-weight hitting sets of the whole clause set and of these (at most
// 2 x 25) are the same.  Into lw.cl; returns how many.
template <class LW>
__device__ uint32_t build_row_minima(LW &lw, uint32_t acc_i, uint32_t acc_x) {
    const DevProg &P = lw.prog;
    const uint32_t lane = lane_id();
    uint32_t ci = 0, cx = 0;
    const bool hi = acc_i != 0u, hx = acc_x != 0u;
    if (hi) ci = slots_of_gaps(P, range_mask(lane, __ffs(acc_i) - 1u));
    if (hx) cx = slots_of_gaps(P, range_mask(lane, __ffs(acc_x) - 1u)) & P.grid_mask;
    const uint32_t bi = __ballot_sync(0xFFFFFFFFu, hi), bx = __ballot_sync(0xFFFFFFFFu, hx);
    const uint32_t below = (1u << lane) - 1u;
    if (hi) lw.cl[__popc(bi & below)] = ci;
    if (hx) lw.cl[__popc(bi) + __popc(bx & below)] = cx;
    __syncwarp();
    return __popc(bi) + __popc(bx);
}

// ---- the loop ---------------------------------------------------------------

// Algorithm 1 for program p by the calling warp, over its conflict relation
// rel[p]; writes out[p].  lw: the warp's record in shared memory.
// Program p's record into the warp's shared copy (from the arena: it does
// not depend on the relations).
template <class LW>
__device__ __forceinline__ void loop_load_record(LW &lw, const ArenaView &V, uint32_t p) {
    const uint4 *src = reinterpret_cast<const uint4 *>(&V.progs[p]);
    uint4 *d4 = reinterpret_cast<uint4 *>(&lw.prog);
    for (uint32_t i = lane_id(); i < sizeof(DevProg) / 16; i += 32u) d4[i] = src[i];
}

// have_record: loop_load_record(lw, V, p) has run already.
template <class LW>
__device__ __forceinline__ void loop_program(LW &lw, const ArenaView &V, uint32_t p, const gr_witnesses *rel,
                                             const gr_options &opts, uint32_t max_iters, uint64_t deadline_ns,
                                             gr_repair_result *out, uint32_t *ctrl, bool have_record = false) {
    const uint32_t lane = lane_id();
    const DevProg &P = lw.prog;
    if (!have_record) loop_load_record(lw, V, p);
    // at L2 (not L1): in the relation kernel's own loop, another CTA wrote them
    const uint32_t conf_i = __ldcg(&rel[p].race_intra[lane]), conf_x = __ldcg(&rel[p].race_inter[lane]);
    __syncwarp();
    if (LW::kCapC < kListCap && (P.general || P.global_rows)) {
        // the small build only takes batches the packer marked simple
        if (lane == 0) atomicOr(&ctrl[1], kErrArgs);
        return;
    }
    const uint32_t S = P.n_stmts, E = P.existing;
    const uint64_t t_start = globaltimer();
    uint32_t forced = P.mode == GR_MODE_REPAIR ? E : 0u;
    uint32_t forbidden = opts.grid_enabled ? 0u : P.grid_mask;
    uint32_t mask = E, iters = 0, n_cl = 0, status = GR_REPAIRED;
    bool probe = P.mode == GR_MODE_REMOVE, greedy = opts.strategy == GR_STRATEGY_MHS, done = false;
    uint32_t acc_i = 0, acc_x = 0;
    if (P.mode != GR_MODE_REMOVE) {
        // Solve over no positive clause: the forced set itself, unless it
        // meets a forbidden slot or holds a negative clause whole
        bool ok = (forced & forbidden) == 0u;
        const bool viol = lane < P.n_neg && (forced & P.neg[lane]) == P.neg[lane];
        ok = ok && !__any_sync(0xFFFFFFFFu, viol);
        if (ok) {
            mask = forced;
        } else {
            status = GR_UNREPAIRABLE;
            done = true;
        }
    }
    while (!done) {
        // Verify(mask): the relation within the phases of mask, and the
        // divergent enabled slots
        const uint32_t gaps = gap_mask(P, mask), ggaps = gap_mask(P, mask & P.grid_mask);
        const uint32_t rows_i = lane < S ? conf_i & phase_of(lane, gaps, S) : 0u;
        const uint32_t rows_x = lane < S ? conf_x & phase_of(lane, ggaps, S) : 0u;
        const uint32_t dv = diverge_warp(P, mask, lane);
        const bool clean = !__any_sync(0xFFFFFFFFu, (rows_i | rows_x) != 0u) && !dv && !probe;
        if (lane == 0) lw.traj[iters] = mask;
        ++iters;
        uint32_t step = 0;  // 0: a new proposal is needed; 1: the exact query after a clean greedy one
        if (clean) {
            if (greedy) {
                greedy = false;
                step = 1;
            } else {
                status = GR_REPAIRED;
                break;
            }
        } else {
            acc_i |= rows_i;
            acc_x |= rows_x;
            probe = false;
            forbidden |= dv;
        }
        bool found = false, solved = false;
        uint32_t smask = 0, sweight = 0;
        if (step == 0 && greedy) {
            // the greedy counts every distinct clause
            n_cl = build_clause_set(lw, acc_i, acc_x);
            found = warp_greedy(lw, n_cl, forced, forbidden, smask, sweight);
            // a greedy set that holds a negative clause whole falls back to the MaxSAT solve
            const bool viol = found && lane < P.n_neg && (smask & P.neg[lane]) == P.neg[lane];
            solved = found && !__any_sync(0xFFFFFFFFu, viol);
        }
        if (!solved) {
            const uint32_t n_min = build_row_minima(lw, acc_i, acc_x);
            found = warp_solve(lw, lw.cl, n_min, forced, forbidden, smask, sweight);
        }
        if (step == 1 && (!found || smask == mask)) {
            status = GR_REPAIRED;  // the greedy proposal is the minimum
            done = true;
        } else if (!found) {
            status = GR_UNREPAIRABLE;
            done = true;
        } else {
            mask = smask;
            if (iters >= max_iters) {
                status = GR_ITER_CAP;
                done = true;
            } else if (deadline_ns && globaltimer() - t_start >= deadline_ns) {
                status = GR_TIMEOUT;
                done = true;
            }
        }
    }
    __syncwarp();
    // the result, with the sorted set of every clause built
    n_cl = build_clause_set(lw, acc_i, acc_x);
    gr_repair_result &o = out[p];
    for (uint32_t k = lane; k < GR_MAX_ITERS; k += 32u) {
        const uint32_t m = k < iters ? lw.traj[k] : 0u;
        o.traj[k] = m;
        if (k < iters) {
            lw.tg[k] = gap_mask(P, m);
            lw.tgg[k] = gap_mask(P, m & P.grid_mask);
        }
    }
    for (uint32_t i = lane; i < GR_MAX_CLAUSES; i += 32u) o.clauses[i] = i < n_cl ? lw.cl[i] : 0u;
    __syncwarp();
    // thread pairs a pairwise checker examines, summed over the checks;
    // each instance's fields packed in one shared word
    {
        uint64_t pk = 0;
        if (lane < S) {
            const DevStmt &st = P.stmts[lane];
            const uint32_t na = guard_count(P.threads, st.gk, st.gr);
            pk = (uint64_t)st.gk | ((uint64_t)st.gr << 16) | ((uint64_t)na << 32) |
                 ((uint64_t)(st.op == GR_W) << 48) | ((uint64_t)st.space << 49);
        }
        lw.pk[lane] = pk;
    }
    __syncwarp();
    // the gaps of up to four checked masks in registers (most programs)
    uint32_t g[4], x[4];
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k) {
        g[k] = k < iters ? lw.tg[k] : 0u;
        x[k] = k < iters ? lw.tgg[k] : 0u;
    }
    // Pairs (i <= j) ordered by j, then i: pair idx = j (j + 1) / 2 + i, so
    // the pairs of S instances are idx < S (S + 1) / 2, about ten per
    // lane.  Per pair, thread counts without the block factors:
    //   a1 += (n_i n_j - n_ij) c_s  (i < j),  n_i (n_i - 1) / 2 c_s  (i == j)
    //   a2 += n_i n_j c_x  (i < j, global),  a3 += n_i^2 c_x  (i == j, global)
    // with c_s / c_x the checks whose same-block / cross-block phase holds
    // both; the block factors B, B (B - 1) and B (B - 1) / 2 at the end.
    unsigned long long a1 = 0, a2 = 0, a3 = 0;
    const uint32_t n_pairs = S * (S + 1u) / 2u;
    for (uint32_t idx = lane; idx < n_pairs; idx += 32u) {
        // j = floor((sqrt(8 idx + 1) - 1) / 2), corrected for rounding
        uint32_t j = (uint32_t)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
        while (j * (j + 1u) / 2u > idx) --j;
        while ((j + 1u) * (j + 2u) / 2u <= idx) ++j;
        const uint32_t i = idx - j * (j + 1u) / 2u;
        const uint64_t mi = lw.pk[i], mj = lw.pk[j];
        const bool wi = (mi >> 48) & 1u, wj = (mj >> 48) & 1u;
        const uint32_t spi = (uint32_t)((mi >> 49) & 1u);
        if (((mj >> 49) & 1u) != spi || (!wi && !wj)) continue;
        const uint32_t ni = (uint32_t)((mi >> 32) & 0xFFFFu), nj = (uint32_t)((mj >> 32) & 0xFFFFu);
        const uint32_t rg = range_mask(i, j);
        uint32_t cs = 0, cx = 0;
        if (iters <= 4) {
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) {
                cs += (k < iters && (g[k] & rg) == 0u) ? 1u : 0u;
                cx += (k < iters && (x[k] & rg) == 0u) ? 1u : 0u;
            }
        } else {
            for (uint32_t k = 0; k < iters; ++k) {
                cs += (lw.tg[k] & rg) == 0u ? 1u : 0u;
                cx += (lw.tgg[k] & rg) == 0u ? 1u : 0u;
            }
        }
        const bool global = spi == GR_GLOBAL;
        if (i == j) {
            a1 += (unsigned long long)(ni * (ni - 1u) / 2u) * cs;  // n_i <= 1,024: 32-bit products
            if (global) a3 += (unsigned long long)(ni * ni) * cx;
        } else {
            const uint32_t gki = (uint32_t)(mi & 0xFFFFu), gri = (uint32_t)((mi >> 16) & 0xFFFFu);
            const uint32_t gkj = (uint32_t)(mj & 0xFFFFu), grj = (uint32_t)((mj >> 16) & 0xFFFFu);
            // threads active at both: one side unguarded or both under one guard needs no count
            const uint32_t nij = gki == 0 ? nj
                                 : (gkj == 0 || (gki == gkj && gri == grj))
                                       ? ni
                                       : guard_both(P.threads, gki, gri, gkj, grj);
            a1 += (unsigned long long)(ni * nj - nij) * cs;
            if (global) a2 += (unsigned long long)(ni * nj) * cx;
        }
    }
    a1 = warp_sum_u64(a1);
    a2 = warp_sum_u64(a2);
    a3 = warp_sum_u64(a3);
    const unsigned long long Bq = P.blocks;
    const unsigned long long pairs = Bq * a1 + Bq * (Bq - 1ull) * a2 + (Bq * (Bq - 1ull) / 2ull) * a3;
    if (lane == 0) {
        const bool ok = status == GR_REPAIRED;
        const uint32_t m = ok ? mask : 0u;
        uint32_t wt = 0;
        for (uint32_t t = m; t; t &= t - 1u) wt += P.weights[__ffs(t) - 1u];
        o.status = (int32_t)status;
        o.mask = m;
        o.weight = wt;
        o.added = m & ~E;
        o.removed = ok ? (E & ~m) : 0u;
        o.iters = iters;
        o.n_clauses = n_cl;
        o.forbidden = forbidden;
        o._pad = 0;
        o.access_pairs = pairs;
        o.t_start_ns = t_start;
        o.t_end_ns = globaltimer();
    }
    __syncwarp();
}

}  // namespace gr
