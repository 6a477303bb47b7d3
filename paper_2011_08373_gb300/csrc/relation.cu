// relation.cu — the check kernel (Verify of Algorithm 1, Section 2.4) for
// programs whose statements all address the shared array and whose blocks
// see one access pattern: the same-block witnesses of every block are block
// 0's, and no pair of blocks shares an array, so one owner-table pass over
// block 0 decides every candidate pair.
//
// Each CTA takes programs from a work queue.  Warp 0 is the control warp: it
// runs one program ahead of the others (two program buffers), fetching and
// setting up program k+1 and writing out program k-1 while warps 1.. (the
// workers) check program k, so that the setup's loads and the output overlap
// the table passes.  Per program:
//   setup   — (control) the candidate pairs: under a mask, the instance pairs
//             (i <= j) with a write and no enabled barrier between them (one
//             phase, Section 2.2); for the repair loop, every pair with a
//             write (the empty mask), which gives the program's whole
//             conflict relation.  Instances with the same map and guard touch
//             the same words from the same threads and share one table row.
//   install — (workers) every access computes its word address from the map
//             (affine or strided arithmetic, or one permutation-table load)
//             and writes its thread into its row's owner entry at that word;
//             two threads of a row on one word leave MULTI (a compare-and-
//             swap, only for rows whose map is not injective on the block's
//             threads).  A bit per row and column marks the rows holding an
//             entry there.
//   scan    — (workers) each thread takes whole columns: two rows holding an
//             entry at a column conflict unless both entries name the same
//             single thread (an entry of another thread, or MULTI, is a
//             second thread on the word: the race definition of Section 1
//             made concrete — two distinct threads, one word, at least one
//             write, no barrier between them).  The scan puts every entry it
//             read back to empty, so the table is clean for the next program
//             without a clear of the whole array.
// Install works in units of one table row and 32 consecutive threads, a warp
// per unit, so that a unit's map, guard and row are the same for the whole
// warp: the per-unit arithmetic (a division or two) is done once and each
// access costs a multiply and a reduction.  The table covers the array in
// windows when it does not fit.
#include <cuda_runtime.h>

#include <cstdint>

#include "device.cuh"

namespace gr {

constexpr uint32_t kRelAllOnes = 0xFFFFFFFFu;

// One program's state (the control warp fills one while the workers use the
// other).
struct RelProg {
    DevProg prog;
    uint32_t cand[32];      // table row q: partner rows (bit j, j >= q) to decide
    uint32_t conf[32];      // table row q: partner rows found to conflict
    uint32_t pend[32];      // instance i: candidate partners (bit j, j >= i)
    uint32_t rep_conf[32];  // the conflicts by pattern representative
    // table row q's access map (its representative's statement, block 0):
    uint32_t row_am[32];    // address of thread t: (am t + bm) mod M, or
    uint32_t row_bm[32];    //   perm[po + (t + bm) mod M] when po != ~0
    uint32_t row_po[32];
    uint32_t row_gk[32], row_gr[32];  // guard (gk == 0: none)
    uint32_t row_gmag[32];  // floor((2^32 - 1) / gk)
    uint32_t nact[32];      // active threads of each instance (for the pair count)
    uint32_t involved, n_rows, W, pitch, n_win, inj_rows, bad, p, mask;
    uint32_t M, Mmagic;     // the shared array's words; floor((2^32 - 1) / M)
};

struct RelSmem {
    RelProg buf[2];
};

constexpr size_t kRelFixed = (sizeof(RelSmem) + 15) / 16 * 16;
size_t rel_fixed_bytes() { return kRelFixed; }

// Column of word a within a window row: the low five bits are XOR-ed with
// the next five, so that 32 words spaced 32 apart (stride-32 maps) fall on
// 32 different banks; the window width is a multiple of 64, so a column
// stays within its row.
__device__ __forceinline__ uint32_t swizzle(uint32_t c) { return c ^ ((c >> 5) & 31u); }

// x mod M for x < 2^31 by a reciprocal multiply: q = floor(x * magic / 2^32)
// with magic = floor((2^32 - 1) / M) is floor(x / M) or one less, so one
// correction gives the remainder (M = 1 included).
__device__ __forceinline__ uint32_t mod_by(uint32_t x, uint32_t M, uint32_t magic) {
    uint32_t r = x - __umulhi(x, magic) * M;
    return r >= M ? r - M : r;
}

// Per-program setup by warp 0: the program record, candidate pairs, table
// rows and their maps, window size.
__device__ void rel_setup(RelProg &sm, const DevProg *gp, uint32_t mask, uint32_t table_bytes) {
    const uint32_t lane = threadIdx.x & 31u;
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(gp);
        uint4 *d4 = reinterpret_cast<uint4 *>(&sm.prog);
        for (uint32_t i = lane; i < sizeof(DevProg) / 16; i += 32u) d4[i] = src[i];
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
        const DevStmt &st = P.stmts[lane];
        sm.cand[row] = pext32(rp, involved);
        sm.conf[row] = 0;
        sm.row_am[row] = st.am;
        sm.row_bm[row] = st.bm;
        sm.row_po[row] = st.kind == GR_PERM ? st.perm_off : kRelAllOnes;
        sm.row_gk[row] = st.gk;
        sm.row_gr[row] = st.gr;
        sm.row_gmag[row] = st.gk ? 0xFFFFFFFFu / st.gk : 0u;
    }
    const uint32_t inj = __ballot_sync(0xFFFFFFFFu, keep && (P.stmts[lane].flags & kStmtInjective));
    if (lane == 0) {
        const uint32_t R = __popc(involved);
        const uint32_t M = P.m_shared;
        // R rows of W + 2 u16 entries (the extra word shifts each row by one
        // bank) and W u32 column masks
        uint32_t W = 0, n_win = 0;
        if (R) {
            const uint32_t wmax = table_bytes > 4u * R ? ((table_bytes - 4u * R) / (2u * R + 4u)) & ~63u : 0u;
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
        sm.inj_rows = pext32(inj, involved);
        sm.bad = (R && W == 0) ? 1u : 0u;
        sm.mask = mask;
    }
}

// Install the accesses of the words [lo, lo + W) into the table: unit u (one
// per worker warp at a time) covers table row q = u / cpr, threads
// 32 c .. 32 c + 31 with c = u mod cpr (cpr = chunks of 32 threads per row);
// lane l takes thread 32 c + l.  (q, c) steps from unit to unit without a
// division, and every reduction is a reciprocal multiply.  When the array
// takes several windows, an affine unit whose 32 words (a run of 31 am + 1
// positions, cyclically) miss the window is skipped whole.
template <uint32_t NT>
__device__ __forceinline__ void rel_install(const RelProg &sm, const uint16_t *__restrict__ perm, uint16_t *tab,
                                            uint32_t *colrows, uint32_t lo) {
    constexpr uint32_t NWK = NT / 32 - 1;  // worker warps
    const uint32_t lane = threadIdx.x & 31u, wk = (threadIdx.x >> 5) - 1u;
    const uint32_t T = sm.prog.threads, M = sm.M, magic = sm.Mmagic, W = sm.W, pitch = sm.pitch;
    const uint32_t cpr = (T + 31u) >> 5, n_units = sm.n_rows * cpr, inj = sm.inj_rows;
    const bool windows = sm.n_win > 1;
    const uint32_t dq = NWK / cpr, dc = NWK - dq * cpr;
    uint32_t q = wk / cpr, c = wk - q * cpr;
    for (uint32_t u = wk; u < n_units; u += NWK) {  // uniform over the warp
        const uint32_t tb = c << 5, t = tb + lane;
        const uint32_t gk = sm.row_gk[q], am = sm.row_am[q], bm = sm.row_bm[q], po = sm.row_po[q];
        const uint32_t qq = q;
        c += dc;
        q += dq;
        if (c >= cpr) {
            c -= cpr;
            ++q;
        }
        if (windows && po == kRelAllOnes && am * 31u + 1u < M) {
            // am * tb + bm < 2^27: the unit's first word and the run to its last
            const uint32_t start = mod_by(am * tb + bm, M, magic);
            const uint32_t d = lo >= start ? lo - start : lo + M - start;  // (lo - start) mod M
            const uint32_t e = start >= lo ? start - lo : start + M - lo;  // (start - lo) mod M
            if (d > am * 31u && e >= W) continue;
        }
        bool on = t < T;
        if (gk) {
            const uint32_t gr = sm.row_gr[qq];
            on = on && ((gk & (gk - 1u)) == 0u ? (t & (gk - 1u)) : mod_by(t, gk, sm.row_gmag[qq])) == gr;
        }
        uint32_t a;
        if (po != kRelAllOnes) {
            // t + bm < 2^10 + 2^16
            a = on ? (uint32_t)__ldg(perm + po + mod_by(t + bm, M, magic)) : 0u;
        } else {
            // am, bm < M <= 2^16, t < 2^10: am t + bm < 2^27
            a = mod_by(am * t + bm, M, magic);
        }
        if (!on || a - lo >= W) continue;
        const uint32_t col = swizzle(a - lo);
        uint16_t *e = tab + (size_t)qq * pitch + col;
        if ((inj >> qq) & 1u) {
            *e = (uint16_t)t;
        } else if (atomicCAS(e, kEmpty, (uint16_t)t) != kEmpty) {
            *e = kMulti;  // a second thread of this row on the word
        }
        atomicAnd(&colrows[col], ~(1u << qq));
    }
}

// Scan the window's columns (worker threads): two rows holding an entry at a
// column conflict unless both entries are the same single thread; a row's
// MULTI entry is its own race.  Each pair is compared once, from its lower
// row (the candidates of a row are its pairs with higher rows).  Every
// entry read, and the column mask, go back to empty.
template <uint32_t NT>
__device__ __forceinline__ void rel_scan(RelProg &sm, uint16_t *tab, uint32_t *colrows) {
    const uint32_t W = sm.W, pitch = sm.pitch;
    for (uint32_t c = threadIdx.x - 32u; c < W; c += NT - 32u) {
        const uint32_t present = ~colrows[c];
        if (!present) continue;
        colrows[c] = kRelAllOnes;
        for (uint32_t t = present; t; t &= t - 1u) {
            const uint32_t qi = __ffs(t) - 1u;
            uint16_t *ei = tab + (size_t)qi * pitch + c;
            // the partners of row qi at this column (itself and the higher rows
            // present) whose pair is a candidate not found yet; none: skip
            const uint32_t open =
                sm.cand[qi] & ~*(volatile uint32_t *)&sm.conf[qi] & (t & ~((1u << qi) - 1u));
            if (!open) {
                *ei = kEmpty;
                continue;
            }
            const uint32_t oi = *ei;
            *ei = kEmpty;  // no later row of this column reads it again
            uint32_t bits = oi == kMulti ? (1u << qi) : 0u;
            for (uint32_t t2 = open & ~(1u << qi); t2; t2 &= t2 - 1u) {
                const uint32_t qj = __ffs(t2) - 1u;
                const uint32_t oj = tab[(size_t)qj * pitch + c];
                bits |= (oi != oj || oi == kMulti) ? (1u << qj) : 0u;
            }
            bits &= open;
            if (bits) or_row(sm.conf, qi, bits);
        }
    }
}

// The program's witness rows (race_intra; one array per block, so no
// cross-block pairs) from the row conflicts, and under a mask its divergent
// slots and pair count.  Warp 0.
__device__ void rel_output(RelProg &sm, gr_witnesses *dst, bool with_mask) {
    const uint32_t lane = threadIdx.x & 31u;
    const DevProg &P = sm.prog;
    const uint32_t involved = sm.involved, p = sm.p;
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
    __syncwarp();
}

// The control warp: the next program from the queue into `b`, set up.
__device__ __forceinline__ void rel_fetch(RelProg &b, const ArenaView &V, uint32_t *ctrl, uint32_t n_fast,
                                          const uint32_t *masks, uint32_t table_bytes) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(&ctrl[2], 1u);
    item = __shfl_sync(0xFFFFFFFFu, item, 0);
    const uint32_t p = item < n_fast ? V.order[item] : kRelAllOnes;
    if (p != kRelAllOnes) rel_setup(b, &V.progs[p], masks ? masks[p] : 0u, table_bytes);
    __syncwarp();
    if (lane == 0) b.p = p;
    __syncwarp();
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
    const uint32_t warp = threadIdx.x >> 5;
    constexpr uint32_t kWorkers = NT - 32u;
    // every table entry is empty (all ones) between programs
    for (uint32_t i = threadIdx.x; i < table_bytes / 16u; i += NT)
        reinterpret_cast<uint4 *>(tab)[i] = make_uint4(kRelAllOnes, kRelAllOnes, kRelAllOnes, kRelAllOnes);
    if (warp == 0) {
        rel_fetch(sm.buf[0], V, ctrl, n_fast, masks, table_bytes);
        if ((threadIdx.x & 31u) == 0) sm.buf[1].p = kRelAllOnes;
    }
    __syncthreads();
    for (uint32_t k = 0;; ++k) {
        RelProg &cur = sm.buf[k & 1u], &prv = sm.buf[(k & 1u) ^ 1u];
        const bool have_cur = cur.p != kRelAllOnes, have_prv = prv.p != kRelAllOnes;
        if (!have_cur && !have_prv) break;  // uniform
        if (warp == 0) {
            // program k-1 out, then program k+1 into its buffer
            if (have_prv) rel_output(prv, dst, masks != nullptr);
            if (have_cur) {
                rel_fetch(prv, V, ctrl, n_fast, masks, table_bytes);
            } else if ((threadIdx.x & 31u) == 0) {
                prv.p = kRelAllOnes;
            }
        } else if (have_cur) {
            const uint32_t R = cur.n_rows, W = cur.W, n_win = cur.n_win;
            if (cur.bad) {
                if (threadIdx.x == 32) atomicOr(&ctrl[1], kErrTableTooSmall);
            } else if (R) {
                uint32_t *colrows = reinterpret_cast<uint32_t *>(tab + (size_t)R * cur.pitch);
                for (uint32_t w = 0; w < n_win; ++w) {
                    rel_install<NT>(cur, V.perm, tab, colrows, w * W);
                    asm volatile("bar.sync 1, %0;" ::"r"(kWorkers) : "memory");
                    rel_scan<NT>(cur, tab, colrows);
                    asm volatile("bar.sync 1, %0;" ::"r"(kWorkers) : "memory");
                }
            }
        }
        __syncthreads();
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
