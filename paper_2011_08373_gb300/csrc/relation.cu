// relation.cu — the check kernel (Verify of Algorithm 1, Section 2.4) for
// programs whose statements all address the shared array and whose blocks
// see one access pattern: the same-block witnesses of every block are block
// 0's, and no pair of blocks shares an array, so one owner-table pass over
// block 0 decides every candidate pair.
//
// Each CTA takes programs from a work queue and, per program:
//   setup   — the candidate pairs: under a mask, the instance pairs (i <= j)
//             with a write and no enabled barrier between them (one phase,
//             Section 2.2); for the repair loop, every pair with a write (the
//             empty mask), which gives the program's whole conflict
//             relation.  Instances with the same map and guard touch the same
//             words from the same threads and share one table row.
//   install — every access computes its word address from the map (affine
//             or strided arithmetic, or one permutation-table load) and
//             writes its thread into its row's owner entry; two threads of a
//             row on one word leave MULTI (a compare-and-swap, only for rows
//             whose map is not injective on the block's threads).  Per column
//             a bit per row marks the rows holding an entry there.
//   probe   — an access (thread t, word a) of row q and a pending partner row
//             j conflict iff j's entry at a is not empty and is not t: an
//             entry of another thread, or MULTI.  This is the race
//             definition of Section 1 made concrete: two distinct threads,
//             one word, at least one write, no barrier between them.
//   reset   — every access puts its entries back to empty, so the table is
//             clean for the next program without a clear of the whole array.
// The table covers the array in windows when it does not fit; the addresses
// of up to kRelCache accesses per thread stay in registers across the passes.
#include <cuda_runtime.h>

#include <cstdint>

#include "device.cuh"

namespace gr {

constexpr uint32_t kRelCache = 16;  // accesses a thread keeps in registers across the passes
constexpr uint32_t kRelAllOnes = 0xFFFFFFFFu;

struct RelSmem {
    DevProg prog;
    uint32_t cand[32];      // table row q: partner rows (bit j, j >= q) still to decide
    uint32_t conf[32];      // table row q: partner rows found to conflict
    uint32_t pend[32];      // instance i: candidate partners (bit j, j >= i)
    uint32_t rep_conf[32];  // the conflicts by pattern representative
    uint32_t rep_list[32];  // representative of table row q
    uint32_t involved, n_rows, use_col, W, n_win, inj_rows, item, bad;
};

constexpr size_t kRelFixed = (sizeof(RelSmem) + 15) / 16 * 16;
size_t rel_fixed_bytes() { return kRelFixed; }

// Column of word a within a window row: the low five bits are XOR-ed with
// the next five, so that 32 words spaced 32 apart (stride-32 maps) fall on
// 32 different banks; the window width is a multiple of 32, so a column
// stays within its row.
__device__ __forceinline__ uint32_t swizzle(uint32_t c) { return c ^ ((c >> 5) & 31u); }

// Per-program setup by warp 0: candidate pairs, table rows, window size.
__device__ void rel_setup(RelSmem &sm, uint32_t mask, uint32_t table_bytes) {
    const DevProg &P = sm.prog;
    const uint32_t lane = threadIdx.x & 31u, S = P.n_stmts;
    const uint32_t gaps = gap_mask(P, mask);
    uint32_t pend = 0;
    if (lane < S) {
        const bool w = (P.write_mask >> lane) & 1u;
        pend = range_mask(lane, S) & phase_of(lane, gaps, S) & (w ? kRelAllOnes : P.write_mask);
    }
    sm.pend[lane] = pend;
    sm.rep_conf[lane] = 0;  // pattern pairs pending (lower representative -> higher)
    __syncwarp();
    for (uint32_t t = pend; t; t &= t - 1u) {
        const uint32_t ri = P.rep[lane], rj = P.rep[__ffs(t) - 1u];
        atomicOr(&sm.rep_conf[min(ri, rj)], 1u << max(ri, rj));
    }
    __syncwarp();
    const uint32_t rp = sm.rep_conf[lane];
    uint32_t involved = rp | (rp ? (1u << lane) : 0u);
    involved = __reduce_or_sync(0xFFFFFFFFu, involved);
    const bool keep = (involved >> lane) & 1u;
    const uint32_t row = __popc(involved & ((1u << lane) - 1u));
    // rows in increasing representative order, so that a representative mask
    // compresses to a row mask by bit extraction
    if (keep) {
        sm.rep_list[row] = lane;
        sm.cand[row] = pext32(rp, involved);
        sm.conf[row] = 0;
    }
    const uint32_t inj = __ballot_sync(0xFFFFFFFFu, keep && (P.stmts[lane].flags & kStmtInjective));
    const uint32_t n_pairs = __reduce_add_sync(0xFFFFFFFFu, __popc(rp));
    if (lane == 0) {
        const uint32_t R = __popc(involved);
        // a bit per row per column pays when rows have three or more pending
        // partners on average (fewer are cheaper to probe one by one)
        const uint32_t use_col = n_pairs >= 3u * R ? 1u : 0u;
        const uint32_t per_col = R + 2u * use_col;  // u16 entries per column
        const uint32_t M = P.m_shared;
        uint32_t W = 0, n_win = 0;
        if (R) {
            const uint32_t wmax = (table_bytes / 2u / per_col) & ~31u;
            const uint32_t mr = (M + 31u) & ~31u;
            W = min(wmax, mr);
            n_win = W ? (M + W - 1u) / W : 0u;
        }
        sm.involved = involved;
        sm.n_rows = R;
        sm.use_col = use_col;
        sm.W = W;
        sm.n_win = n_win;
        sm.inj_rows = pext32(inj, involved);
        sm.bad = (R && W == 0) ? 1u : 0u;
    }
}

// The accesses of round `base` this thread takes: u = base + tid + k NT over
// (table row q, thread t), q = u / T; key = word | t << 16 | q << 26, all ones
// for no access (guard false, or past the end).
template <uint32_t NT>
__device__ __forceinline__ void rel_keys(const RelSmem &sm, const uint16_t *__restrict__ perm, uint32_t base,
                                         uint32_t total, uint32_t (&key)[kRelCache]) {
    const DevProg &P = sm.prog;
    const uint32_t T = P.threads;
#pragma unroll
    for (uint32_t k = 0; k < kRelCache; ++k) {
        const uint32_t u = base + threadIdx.x + k * NT;
        key[k] = kRelAllOnes;
        if (u < total) {
            const uint32_t q = u / T, t = u - q * T;
            const DevStmt &st = P.stmts[sm.rep_list[q]];
            if (st.gk == 0 || t % st.gk == st.gr) {
                const uint32_t M = st.m;
                // 32-bit arithmetic: am, bm < M <= 65,536 and t < 1,024
                const uint32_t a = st.kind == GR_PERM ? (uint32_t)__ldg(perm + st.perm_off + (t + st.bm) % M)
                                                      : (st.am * t + st.bm) % M;
                key[k] = a | (t << 16) | (q << 26);
            }
        }
    }
}

template <uint32_t NT, uint32_t MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_relation(const uint8_t *__restrict__ arena, uint32_t n, const uint32_t *__restrict__ masks,
               uint8_t *__restrict__ scratch, uint64_t scratch_bytes, gr_witnesses *__restrict__ out,
               uint32_t table_bytes) {
    extern __shared__ uint4 rel_raw[];
    RelSmem &sm = *reinterpret_cast<RelSmem *>(rel_raw);
    uint16_t *tab = reinterpret_cast<uint16_t *>(reinterpret_cast<uint8_t *>(rel_raw) + kRelFixed);
    const ArenaView V = view(arena);
    uint32_t *ctrl = reinterpret_cast<uint32_t *>(scratch);
    if (!launch_matches(V, n, scratch_bytes)) {
        if (threadIdx.x == 0) atomicOr(&ctrl[1], kErrArgs);
        return;
    }
    gr_witnesses *dst = out ? out : reinterpret_cast<gr_witnesses *>(scratch + V.h->scratch_rel_off);
    const uint32_t n_fast = V.h->n_fast;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    // every table entry is empty (all ones) between programs
    for (uint32_t i = threadIdx.x; i < table_bytes / 16u; i += NT)
        reinterpret_cast<uint4 *>(tab)[i] = make_uint4(kRelAllOnes, kRelAllOnes, kRelAllOnes, kRelAllOnes);
    for (;;) {
        if (threadIdx.x == 0) sm.item = atomicAdd(&ctrl[2], 1u);
        __syncthreads();  // also: the previous program's reset is complete
        const uint32_t item = sm.item;
        if (item >= n_fast) break;
        const uint32_t p = V.order[item];
        {
            const uint4 *src = reinterpret_cast<const uint4 *>(&V.progs[p]);
            uint4 *d4 = reinterpret_cast<uint4 *>(&sm.prog);
            for (uint32_t i = threadIdx.x; i < sizeof(DevProg) / 16; i += NT) d4[i] = src[i];
        }
        __syncthreads();
        const uint32_t mask = masks ? masks[p] : 0u;
        if (warp == 0) rel_setup(sm, mask, table_bytes);
        __syncthreads();
        const uint32_t R = sm.n_rows, W = sm.W, n_win = sm.n_win, use_col = sm.use_col, inj = sm.inj_rows;
        if (sm.bad) {
            if (threadIdx.x == 0) atomicOr(&ctrl[1], kErrTableTooSmall);
        } else if (R) {
            const uint32_t total = R * sm.prog.threads;
            const uint32_t per_round = NT * kRelCache;
            const uint32_t rounds = (total + per_round - 1u) / per_round;
            uint32_t *colrows = reinterpret_cast<uint32_t *>(tab + (size_t)R * W);
            uint32_t key[kRelCache];
            if (rounds == 1) rel_keys<NT>(sm, V.perm, 0, total, key);
            for (uint32_t w = 0; w < n_win; ++w) {
                const uint32_t lo = w * W;
                // install
                for (uint32_t rd = 0; rd < rounds; ++rd) {
                    if (rounds > 1) rel_keys<NT>(sm, V.perm, rd * per_round, total, key);
#pragma unroll
                    for (uint32_t k = 0; k < kRelCache; ++k) {
                        const uint32_t x = key[k];
                        if (x == kRelAllOnes || (x & 0xFFFFu) - lo >= W) continue;
                        const uint32_t col = swizzle((x & 0xFFFFu) - lo), q = x >> 26;
                        const uint16_t t = (uint16_t)((x >> 16) & 0x3FFu);
                        uint16_t *e = tab + (size_t)q * W + col;
                        if ((inj >> q) & 1u) {
                            *e = t;
                        } else if (atomicCAS(e, kEmpty, t) != kEmpty) {
                            *e = kMulti;  // a second thread of this row on the word
                        }
                        if (use_col) atomicAnd(&colrows[col], ~(1u << q));
                    }
                }
                __syncthreads();
                // probe
                for (uint32_t rd = 0; rd < rounds; ++rd) {
                    if (rounds > 1) rel_keys<NT>(sm, V.perm, rd * per_round, total, key);
#pragma unroll
                    for (uint32_t k = 0; k < kRelCache; ++k) {
                        const uint32_t x = key[k];
                        if (x == kRelAllOnes || (x & 0xFFFFu) - lo >= W) continue;
                        const uint32_t col = swizzle((x & 0xFFFFu) - lo), q = x >> 26;
                        const uint32_t t = (x >> 16) & 0x3FFu;
                        uint32_t todo = sm.cand[q] & ~*(volatile uint32_t *)&sm.conf[q];
                        if (!todo) continue;
                        if (use_col) todo &= ~colrows[col];
                        uint32_t hits = 0;
                        for (; todo; todo &= todo - 1u) {
                            const uint32_t j = __ffs(todo) - 1u;
                            const uint32_t o = tab[(size_t)j * W + col];
                            hits |= (o != kEmpty && o != t) ? (1u << j) : 0u;
                        }
                        if (hits) or_row(sm.conf, q, hits);
                    }
                }
                __syncthreads();
                // reset
                for (uint32_t rd = 0; rd < rounds; ++rd) {
                    if (rounds > 1) rel_keys<NT>(sm, V.perm, rd * per_round, total, key);
#pragma unroll
                    for (uint32_t k = 0; k < kRelCache; ++k) {
                        const uint32_t x = key[k];
                        if (x == kRelAllOnes || (x & 0xFFFFu) - lo >= W) continue;
                        const uint32_t col = swizzle((x & 0xFFFFu) - lo), q = x >> 26;
                        tab[(size_t)q * W + col] = kEmpty;
                        if (use_col) colrows[col] = kRelAllOnes;
                    }
                }
                __syncthreads();
            }
        }
        if (warp == 0) {
            // row conflicts back to representatives, then to instance pairs
            const DevProg &P = sm.prog;
            const uint32_t involved = sm.involved;
            uint32_t rc = 0;
            if ((involved >> lane) & 1u) rc = pdep32(sm.conf[__popc(involved & ((1u << lane) - 1u))], involved);
            sm.rep_conf[lane] = rc;
            __syncwarp();
            uint32_t rows = 0;
            for (uint32_t t = sm.pend[lane]; t; t &= t - 1u) {
                const uint32_t j = __ffs(t) - 1u;
                const uint32_t ri = P.rep[lane], rj = P.rep[j];
                if ((sm.rep_conf[min(ri, rj)] >> max(ri, rj)) & 1u) rows |= 1u << j;
            }
            gr_witnesses &wo = dst[p];
            wo.race_intra[lane] = rows;
            wo.race_inter[lane] = 0u;  // one array per block: no cross-block pairs
            uint32_t dv = 0;
            unsigned long long pairs = 0;
            if (masks) {
                dv = diverge_warp(P, mask, lane);
                const uint32_t S = P.n_stmts, gaps = gap_mask(P, mask);
                for (uint32_t idx = lane; idx < S * S; idx += 32u) {
                    const uint32_t i = idx / S, j = idx - i * S;
                    if (j < i || (gaps & range_mask(i, j))) continue;
                    uint64_t same, cross;
                    pair_count(P, i, j, same, cross);
                    pairs += same;
                }
                pairs = warp_sum_u64(pairs);
            }
            if (lane == 0) {
                wo.diverge = dv;
                wo.n_stmts = P.n_stmts;
                wo.access_pairs = pairs;
            }
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
    if ((e = rel_set_smem(k_relation<512, 3>, max_dynamic_smem)) != cudaSuccess) return e;
    if ((e = rel_set_smem(k_relation<256, 4>, max_dynamic_smem)) != cudaSuccess) return e;
    if ((e = rel_set_smem(k_relation<512, 2>, max_dynamic_smem)) != cudaSuccess) return e;
    if ((e = rel_set_smem(k_relation<1024, 1>, max_dynamic_smem)) != cudaSuccess) return e;
    if ((e = rel_set_smem(k_relation<256, 6>, max_dynamic_smem)) != cudaSuccess) return e;
    if ((e = rel_set_smem(k_relation<128, 8>, max_dynamic_smem)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t launch_relation(const void *d_arena, uint32_t n, const uint32_t *d_masks, void *d_scratch,
                            uint64_t scratch_bytes, gr_witnesses *d_out, RelCfg cfg, cudaStream_t st) {
    const uint8_t *a = static_cast<const uint8_t *>(d_arena);
    uint8_t *sc = static_cast<uint8_t *>(d_scratch);
    const size_t smem = kRelFixed + cfg.table_bytes;
    switch (cfg.shape) {
        case 1: k_relation<256, 4><<<cfg.grid, 256, smem, st>>>(a, n, d_masks, sc, scratch_bytes, d_out, cfg.table_bytes); break;
        case 2: k_relation<512, 2><<<cfg.grid, 512, smem, st>>>(a, n, d_masks, sc, scratch_bytes, d_out, cfg.table_bytes); break;
        case 3: k_relation<1024, 1><<<cfg.grid, 1024, smem, st>>>(a, n, d_masks, sc, scratch_bytes, d_out, cfg.table_bytes); break;
        case 4: k_relation<256, 6><<<cfg.grid, 256, smem, st>>>(a, n, d_masks, sc, scratch_bytes, d_out, cfg.table_bytes); break;
        case 5: k_relation<128, 8><<<cfg.grid, 128, smem, st>>>(a, n, d_masks, sc, scratch_bytes, d_out, cfg.table_bytes); break;
        default: k_relation<512, 3><<<cfg.grid, 512, smem, st>>>(a, n, d_masks, sc, scratch_bytes, d_out, cfg.table_bytes); break;
    }
    return cudaGetLastError();
}

}  // namespace gr
