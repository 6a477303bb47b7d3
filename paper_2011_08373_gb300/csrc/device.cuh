// device.cuh — device helpers shared by the kernels of libgpurepair: the
// packed arena view, bit operations over statement and slot masks (phases,
// gaps, clause ranges), the bit-sliced solver's small helpers, and the
// closed-form thread-pair counts.  Internal; not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "engine.cuh"

namespace gr {

struct ArenaView {
    const ArenaHeader *h;
    const DevProg *progs;
    const uint32_t *order;
    const uint64_t *segbase;
    const uint16_t *perm;  // permutation tables, entries below 65,536
};

__device__ __forceinline__ ArenaView view(const uint8_t *arena) {
    ArenaView v;
    v.h = reinterpret_cast<const ArenaHeader *>(arena);
    v.progs = reinterpret_cast<const DevProg *>(arena + v.h->progs_off);
    v.order = reinterpret_cast<const uint32_t *>(arena + v.h->order_off);
    v.segbase = reinterpret_cast<const uint64_t *>(arena + v.h->segbase_off);
    v.perm = reinterpret_cast<const uint16_t *>(arena + v.h->perm_off);
    return v;
}

// The launch's program count and scratch size against the arena header: a
// kernel given a count or a scratch buffer that does not match the arena it
// reads would index past the caller's buffers, so it does no work and
// raises kErrArgs in the device error word instead.  Every CTA decides the
// same way.
__device__ __forceinline__ bool launch_matches(const ArenaView &V, uint32_t n, uint64_t scratch_bytes) {
    return V.h->magic == kArenaMagic && V.h->n_progs == n && scratch_bytes >= V.h->scratch_bytes;
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// x mod M for any 32-bit x by a reciprocal multiply: with magic =
// floor((2^32 - 1) / M), q = floor(x magic / 2^32) is floor(x / M) or at most
// two less (x magic / 2^32 > x / M - (1 + M) / M), so two corrections give
// the remainder (M = 1 included).
__device__ __forceinline__ uint32_t mod_u32(uint32_t x, uint32_t M, uint32_t magic) {
    uint32_t r = x - __umulhi(x, magic) * M;
    if (r >= M) r -= M;
    if (r >= M) r -= M;
    return r;
}

__device__ __forceinline__ uint32_t range_mask(uint32_t i, uint32_t j) {  // bits [i, j)
    const uint32_t hi = j >= 32 ? 0xFFFFFFFFu : ((1u << j) - 1u);
    return hi & ~((1u << i) - 1u);
}

// Gaps between executed instances where an enabled barrier (of the slots in
// `mask`) runs: gap k (between instances k and k+1) runs the barriers of the
// slots gapslots[k].  Without loops or explicit places gap k is slot k.
__device__ __forceinline__ uint32_t gap_mask(const DevProg &P, uint32_t mask) {
    if (!P.general) return mask;
    uint32_t g = 0;
    for (uint32_t k = 0; k + 1 < P.n_stmts; ++k)
        if (P.gapslots[k] & mask) g |= 1u << k;
    return g;
}

// The slots whose barriers run in the gaps `gaps`.
__device__ __forceinline__ uint32_t slots_of_gaps(const DevProg &P, uint32_t gaps) {
    if (!P.general) return gaps;
    uint32_t m = 0;
    for (uint32_t t = gaps; t; t &= t - 1u) m |= P.gapslots[__ffs(t) - 1u];
    return m;
}

// Instances in the same phase as s when the gaps in `cut` hold an enabled
// barrier: gap k separates instances k and k+1.
__device__ __forceinline__ uint32_t phase_of(uint32_t s, uint32_t cut, uint32_t S) {
    const uint32_t below = cut & ((1u << s) - 1u);
    const uint32_t start = below ? 32u - __clz(below) : 0u;
    const uint32_t above = cut >> s;
    const uint32_t end = above ? s + __ffs(above) - 1u : S - 1u;
    return range_mask(start, end + 1u);
}

__device__ __forceinline__ uint32_t pext32(uint32_t x, uint32_t m) {
    uint32_t out = 0, j = 0;
    for (uint32_t t = m; t; t &= t - 1u, ++j)
        if (x & (t & (0u - t))) out |= 1u << j;
    return out;
}

__device__ __forceinline__ uint32_t pdep32(uint32_t x, uint32_t m) {
    uint32_t out = 0, j = 0;
    for (uint32_t t = m; t; t &= t - 1u, ++j)
        if ((x >> j) & 1u) out |= t & (0u - t);
    return out;
}

// Low assignments l in [0,32) with bit k set, k < 5.
__device__ __forceinline__ uint32_t low_pattern(uint32_t k) {
    const uint32_t p[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u, 0xFFFF0000u};
    return p[k];
}

__device__ __forceinline__ void or_row(uint32_t *rows, uint32_t i, uint32_t bits) {
    volatile uint32_t *vr = rows;
    if (bits & ~vr[i]) atomicOr(&rows[i], bits);
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
    for (uint32_t o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Next k-subset in colex order (Gosper's step).
__device__ __forceinline__ uint32_t gosper_next(uint32_t h) {
    const uint32_t c = h & (0u - h);
    const uint32_t r = h + c;
    return (((r ^ h) >> 2) >> (__ffs(c) - 1u)) | r;
}

struct BinomTable {
    uint32_t v[GR_MAX_SLOTS + 1][GR_MAX_SLOTS + 1];  // C(n, k), n <= 32: at most C(32, 16) < 2^32
    constexpr BinomTable() : v() {
        for (int n = 0; n <= GR_MAX_SLOTS; ++n) {
            v[n][0] = 1;
            for (int k = 1; k <= n; ++k) v[n][k] = v[n - 1][k - 1] + (k <= n - 1 ? v[n - 1][k] : 0);
        }
    }
};
static __constant__ BinomTable c_binom = BinomTable();

// The k-subset of {0..n-1} of colex rank `rank`.
__device__ __forceinline__ uint32_t unrank_colex(uint32_t rank, uint32_t k, uint32_t n) {
    uint32_t h = 0;
    int c = (int)n - 1;
    for (uint32_t i = k; i >= 1; --i) {
        while (c >= 0 && c_binom.v[c][i] > rank) --c;
        h |= 1u << c;
        rank -= c_binom.v[c][i];
        --c;
    }
    return h;
}

// ---- thread-pair counts in closed form --------------------------------------

// Threads t in [0, T) with t % k == r (k == 0: every thread).
__device__ __forceinline__ uint32_t guard_count(uint32_t T, uint32_t k, uint32_t r) {
    if (k == 0) return T;
    return r < T ? (T - 1u - r) / k + 1u : 0u;
}

// Inverse of a modulo m (gcd(a, m) == 1, 2 <= m < 2^16), by the extended
// Euclidean algorithm (32-bit: every remainder and coefficient is below m).
__device__ __forceinline__ uint32_t mod_inverse(uint32_t a, uint32_t m) {
    int32_t r0 = (int32_t)m, r1 = (int32_t)(a % m), s0 = 0, s1 = 1;
    while (r1 != 0) {
        const int32_t q = r0 / r1;
        const int32_t r2 = r0 - q * r1;
        r0 = r1;
        r1 = r2;
        const int32_t s2 = s0 - q * s1;
        s0 = s1;
        s1 = s2;
    }
    return (uint32_t)(s0 < 0 ? s0 + (int32_t)m : s0);
}

// Threads t in [0, T) active under both guards (k1, r1) and (k2, r2).  Both
// congruences t = r1 (mod k1), t = r2 (mod k2) hold on one residue class
// modulo lcm(k1, k2) when r1 = r2 (mod gcd(k1, k2)) (Chinese remainder
// theorem) and on none otherwise; the class's least member t0 is
// r1 + k1 q0 with k1 q0 = r2 - r1 (mod k2), q0 found with the inverse of
// k1 / g modulo k2 / g.  Guards have k < 2^16, so t0 < lcm <= k1 k2 / g
// < 2^32: 32-bit arithmetic throughout.
__device__ __forceinline__ uint32_t guard_both(uint32_t T, uint32_t k1, uint32_t r1, uint32_t k2, uint32_t r2) {
    if (k1 == 0) return guard_count(T, k2, r2);
    if (k2 == 0) return guard_count(T, k1, r1);
    // one modulus a multiple of the other (powers of two, equal moduli): the
    // finer congruence decides, and it must agree with the coarser one
    if (k2 % k1 == 0) return r2 % k1 == r1 ? guard_count(T, k2, r2) : 0u;
    if (k1 % k2 == 0) return r1 % k2 == r2 ? guard_count(T, k1, r1) : 0u;
    uint32_t a = k1, b = k2;
    while (b) {
        const uint32_t t = a % b;
        a = b;
        b = t;
    }
    const uint32_t g = a;
    const uint32_t dr = r2 >= r1 ? r2 - r1 : r1 - r2;
    if (dr % g != 0) return 0u;
    const uint32_t m = k2 / g;
    uint32_t q0 = 0;
    if (m > 1) {
        const uint32_t dq = (dr / g) % m;
        const uint32_t d = r2 >= r1 ? dq : (dq ? m - dq : 0u);  // (r2 - r1) / g mod m
        q0 = d * mod_inverse((k1 / g) % m, m) % m;
    }
    const uint32_t t0 = r1 + k1 * q0;
    const uint32_t l = k1 * m;  // lcm(k1, k2)
    return t0 < T ? (T - 1u - t0) / l + 1u : 0u;
}

// Thread pairs of instance pair (i <= j) that a pairwise checker examines
// when nothing orders them: same-block and cross-block, for pairs of one
// array with a write (0 otherwise).  i < j: ordered pairs of distinct
// threads, B (n_i n_j - n_ij) in one block, B (B - 1) n_i n_j across blocks
// (global array only); i == j: unordered pairs, B n_i (n_i - 1) / 2 and
// B (B - 1) / 2 n_i^2.
// nact: the active threads of each instance (guard_count).
__device__ __forceinline__ void pair_count(const DevProg &P, const uint32_t *nact, uint32_t i, uint32_t j,
                                           uint64_t &same, uint64_t &cross) {
    const DevStmt &a = P.stmts[i], &b = P.stmts[j];
    same = 0;
    cross = 0;
    if (a.space != b.space || (a.op != GR_W && b.op != GR_W)) return;
    const uint64_t T = P.threads, B = P.blocks;
    const uint64_t ni = nact[i];
    const bool global = a.space == GR_GLOBAL;
    if (i < j) {
        const uint64_t nj = nact[j];
        // threads active at both: one side unguarded or both under one guard needs no count
        const uint64_t nij = a.gk == 0 ? nj
                             : (b.gk == 0 || (a.gk == b.gk && a.gr == b.gr))
                                   ? ni
                                   : guard_both(P.threads, a.gk, a.gr, b.gk, b.gr);
        same = B * (ni * nj - nij);
        cross = global ? B * (B - 1) * ni * nj : 0;
    } else {
        same = B * (ni * (ni - 1) / 2);
        cross = global ? (B * (B - 1) / 2) * ni * ni : 0;
    }
    (void)T;
}

// Divergent enabled slots under mask: an enabled slot whose guard holds for
// some tid in [0, T) and fails for another.  Lane k of the calling warp
// decides slot k; every lane returns the mask.
__device__ __forceinline__ uint32_t diverge_warp(const DevProg &P, uint32_t mask, uint32_t lane) {
    bool dv = false;
    if (((mask & P.guarded_slots) >> lane) & 1u) {
        const uint32_t cnt = guard_count(P.threads, P.slot_gk[lane], P.slot_gr[lane]);
        dv = cnt > 0 && cnt < P.threads;
    }
    return __ballot_sync(0xFFFFFFFFu, dv);
}

}  // namespace gr
