// kernels.cu — sm_103a kernels of the repair loop (Algorithm 1 of GPURepair,
// Section 2.4) over concrete access programs.
//
//   k_expand        : address traces, one u16 word address per (statement,
//                     thread), layout [S][B][t_pad] with a segment's threads in
//                     unit order (8 per unit, spaced so that the 32 units of a
//                     warp read 32 consecutive threads at a time), plus per
//                     (statement, block) the 1,024-word chunks touched and the
//                     address range.
//   owner tables    : the check (Verify).  For each address of a chunk tile, a
//                     shared-memory table holds per statement the one thread
//                     (same-block pass) or block (cross-block pass) that touched
//                     it, or MULTI: a CAS installs each access.  A probe pass
//                     then reads, at every access, the entries of the pending
//                     partner statements and emits the witness bitmaps.
//   mhs_solve       : exact minimum-weight hitting set (Solve), bit-sliced: the
//                     low 5 compact variables ride in the bits of a 32-bit word,
//                     the rest are enumerated by popcount level (Gosper order)
//                     with a weight bound; ties go to the lowest mask.
//   k_check         : persistent work-queue kernel, one CTA per program, one
//                     check per program of the batch's general part (a
//                     global array, or blocks that differ); under the empty
//                     mask it gives the conflict relation the loop kernel
//                     (loop.cu) filters.  Programs on the shared array with
//                     alike blocks go to the relation kernel (relation.cu).
//   k_plain_*       : the same stages as separate launches, one check launch
//                     per iteration (host-driven loop).
#include <cuda_runtime.h>

#include <cstdint>

#include "device.cuh"

namespace gr {

// ---------------------------------------------------------------------------
// Shared memory
// ---------------------------------------------------------------------------

struct MhsSmem {
    uint32_t cl[kClauseCap];   // raw clause list (shares the table region: never live during a check)
    uint32_t pc[kClauseCap];   // preprocessed positive clauses (0 = dropped)
    uint32_t khi[kClauseCap];  // kept clauses: compact high part
    uint32_t klo[kClauseCap];  // kept clauses: low-part hit pattern over 32 low assignments
    uint32_t set[kClauseSet];  // open-addressing set of the clauses built so far; the
                               // solver's size-sorted clauses after that
    uint32_t nhi[kClauseCap];
    uint32_t nlo[kClauseCap];
    uint32_t w8[4][256];       // weight of each byte of the high part
    uint32_t wlo[32];          // weight of each low assignment
    uint32_t lb[GR_MAX_SLOTS + 2];  // sum of the k smallest high weights
    uint32_t wc[GR_MAX_SLOTS]; // compact weights
    uint32_t n_kept, n_negk, R, U, unsat;
    uint32_t full_seen;  // the clause of all 32 slots (the set's empty marker) was built
    uint32_t size_at[33];  // counting sort of the positive clauses by size
};

struct Smem {
    DevProg prog;
    uint32_t act[GR_MAX_STMTS][32];  // active-thread bitmaps per statement
    uint32_t nact[32];               // active threads per statement
    uint32_t rows_intra[32], rows_inter[32];
    uint32_t acc_intra[32], acc_inter[32];
    uint32_t ph_intra[32], ph_inter[32];
    uint32_t traj[GR_MAX_ITERS];
    uint32_t row_list[32];
    uint32_t pend_row[32];  // pending partners of each statement in the current pass
    uint32_t rep_pend[32], rep_conf[32];  // pending / witnessed pattern pairs (lower -> higher)
    uint32_t n_seg_list, pass_rows, pass_pend;
    uint32_t rlo[32], rhi[32], clo[32], chi[32];
    uint32_t seg_list[kSegCap];
    unsigned long long bchunk[2][64];
    unsigned long long npair[2][325];  // per statement pair: same-block / cross-block thread pairs
    uint32_t scan[32];
    uint8_t chunk_slot[64];
    unsigned long long best;
    unsigned long long pairs;
    unsigned long long access_pairs;
    unsigned long long t_start;
    unsigned long long chunk_acc;
    // loop state
    uint32_t mask, probe, done, status, iters, forced, forbidden, max_iters;
    uint32_t greedy, step;  // mhs strategy: greedy proposals pending; kind of this step
    unsigned long long deadline_ns;  // 0: none; else the loop's time limit (gr_options::deadline_us)
    uint32_t diverge, n_cl, n_rows, item;
    uint32_t rel_sh, rel_gi, rel_gx, sol_found, sol_mask, sol_weight;
    uint32_t *err;  // device error word (scratch control area)
};

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
constexpr size_t kFixedSmem = align_up(sizeof(Smem), 16);

// The clause list lives in the region the owner table uses during a check.
__device__ __forceinline__ uint32_t *mh_cl(Smem &sm) {
    return reinterpret_cast<MhsSmem *>(reinterpret_cast<uint8_t *>(&sm) + kFixedSmem)->cl;
}

size_t fixed_smem_bytes() { return kFixedSmem; }
size_t mhs_smem_bytes() { return align_up(sizeof(MhsSmem), 16); }

// ---------------------------------------------------------------------------
// Program load
// ---------------------------------------------------------------------------

__device__ void pair_counts(Smem &sm);

__device__ void load_program(Smem &sm, const DevProg *gp) {
    const uint4 *src = reinterpret_cast<const uint4 *>(gp);
    uint4 *dst = reinterpret_cast<uint4 *>(&sm.prog);
    for (uint32_t i = threadIdx.x; i < sizeof(DevProg) / 16; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    // active-thread bitmaps in the traces' unit order: byte v of a row holds
    // the 8 threads of unit v (unit v of group g: threads 256 g + (v mod 32) +
    // U e, U = the group's units); bytes past the units are zero
    const uint32_t S = sm.prog.n_stmts, T = sm.prog.threads, nv = sm.prog.t_pad >> 3;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (uint32_t s = warp; s < S; s += nwarps) {
        const uint32_t k = sm.prog.stmts[s].gk, r = sm.prog.stmts[s].gr, kk = k ? k : 1u;
        uint32_t n = 0;
        for (uint32_t g = 0; g < 4u; ++g) {  // unit v = 32 g + lane (at most 128 units)
            const uint32_t v = 32u * g + lane;
            uint32_t a8 = 0;
            if (v < nv) {
                const uint32_t U = min(32u, nv - 32u * g), t0 = 256u * g + lane;
                // t mod k advanced by U threads at a time
                const uint32_t du = U % kk;
                uint32_t m = t0 % kk;
                for (uint32_t e = 0; e < 8u; ++e) {
                    if (t0 + U * e < T && (k == 0 || m == r)) a8 |= 1u << e;
                    m += du;
                    if (m >= kk) m -= kk;
                }
            }
            n += __popc(a8);
            uint32_t word = a8 << ((lane & 3u) * 8u);
            word |= __shfl_xor_sync(0xFFFFFFFFu, word, 1);
            word |= __shfl_xor_sync(0xFFFFFFFFu, word, 2);
            if ((lane & 3u) == 0) sm.act[s][8u * g + (lane >> 2)] = word;
        }
        n = __reduce_add_sync(0xFFFFFFFFu, n);
        if (lane == 0) sm.nact[s] = n;
    }
    __syncthreads();
    pair_counts(sm);
}

// ---------------------------------------------------------------------------
// Check: owner tables
// ---------------------------------------------------------------------------

// One owner pass over the statements in `rows` (bit s = statement s), the
// accesses of blocks [blk_lo, blk_lo+nb) and the address chunks in `chunks`.
// The owner of an access is its tid (same-block pass, nb == 1) or its block
// (cross-block pass).  Witness bits go to rows_out (row i, bit j >= i) for
// pairs in one phase (ph) with at least one write.
//
// Only candidate pairs not yet in rows_out are pending, and only their
// statements get a table row.  Chunks are processed in tiles of up to `cap`
// chunks.  Per tile:
//   clear — each row's owner entries over its own address range;
//   build — every access installs its owner with a CAS on an empty entry and
//           turns an entry holding another owner into MULTI; only (statement,
//           block) segments whose chunk mask meets the tile are read;
//   probe — an access (owner o, address a) of statement i and a pending
//           partner j form a witness iff j's entry at a is neither empty nor
//           o (a MULTI entry always differs; j == i is the self race).  Each
//           thread probes its eight addresses per partner and skips partners
//           already witnessed.
// Statements with the same array, map and guard touch the same addresses from
// the same threads, so they share one row: the pass works on the lowest
// statement of each such class, and a pair inside one class conflicts iff the
// class's row holds a MULTI (its self pair).
template <bool kInter>
__device__ void owner_pass(Smem &sm, uint16_t *tab, uint32_t table_bytes, const uint16_t *trace,
                           const uint64_t *segmask, const uint32_t *segrange, uint32_t rows,
                           uint32_t blk_lo, uint32_t nb, uint64_t chunks, const uint32_t *ph,
                           uint32_t *rows_out) {
    const DevProg &P = sm.prog;
    const uint32_t S = P.n_stmts, B = P.blocks, tpad = P.t_pad, nv = tpad >> 3;
    if (rows == 0 || chunks == 0) return;  // uniform
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t wmask = P.write_mask;
    __syncthreads();  // row_list / pending / ranges are reused across passes
    if (warp == 0) {
        const uint32_t i = lane;
        const bool in = i < S && ((rows >> i) & 1u);
        // pending candidate partners: j >= i in i's phase (a read only with a
        // write), not yet witnessed
        uint32_t pend = 0;
        if (in) pend = rows & ph[i] & ~((1u << i) - 1u) & (((wmask >> i) & 1u) ? 0xFFFFFFFFu : wmask) & ~rows_out[i];
        sm.pend_row[i] = pend;
        // statements with the same access pattern have the same owner row: a
        // pending pair becomes a pair of pattern representatives (lower first)
        sm.rep_pend[lane] = 0;
        sm.rep_conf[lane] = 0;
        __syncwarp();
        for (uint32_t t = pend; t; t &= t - 1u) {
            const uint32_t ri = sm.prog.rep[i], rj = sm.prog.rep[__ffs(t) - 1u];
            atomicOr(&sm.rep_pend[min(ri, rj)], 1u << max(ri, rj));
        }
        __syncwarp();
        const uint32_t rp = sm.rep_pend[lane];
        uint32_t involved = rp | (rp ? (1u << lane) : 0u);
        for (uint32_t o = 16; o > 0; o >>= 1) involved |= __shfl_xor_sync(0xFFFFFFFFu, involved, o);
        const bool keep = (involved >> lane) & 1u;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
        if (keep) sm.row_list[__popc(bal & ((1u << lane) - 1u))] = lane;
        if (lane == 0) sm.pass_rows = involved;
        const uint32_t n_pend = __reduce_add_sync(0xFFFFFFFFu, __popc(rp));  // pending pattern pairs
        if (lane == 0) sm.pass_pend = n_pend;
        // address range of each row over the blocks of the pass: here for a
        // few blocks (each lane its own row), by the whole CTA below otherwise
        uint32_t lo = 0xFFFFu, hi = 0u;
        if (nb <= 32u && keep) {
            for (uint32_t bi = 0; bi < nb; ++bi) {
                const uint32_t r = segrange[(size_t)lane * B + blk_lo + bi];
                if ((r & 0xFFFFu) <= (r >> 16)) {
                    lo = min(lo, r & 0xFFFFu);
                    hi = max(hi, r >> 16);
                }
            }
        }
        sm.rlo[lane] = lo;
        sm.rhi[lane] = hi;
    }
    __syncthreads();
    rows = sm.pass_rows;
    const uint32_t n_rows = __popc(rows);
    if (n_rows == 0) return;  // every candidate pair already witnessed
    if (nb > 32u) {
        for (uint32_t u = threadIdx.x; u < S * nb; u += blockDim.x) {
            const uint32_t st = u / nb, bi = u - st * nb;
            if (!((rows >> st) & 1u)) continue;
            const uint32_t r = segrange[(size_t)st * B + blk_lo + bi];
            const uint32_t lo = r & 0xFFFFu, hi = r >> 16;
            if (lo <= hi) {
                atomicMin(&sm.rlo[st], lo);
                atomicMax(&sm.rhi[st], hi);
            }
        }
        __syncthreads();  // the ranges, before the column ranges of each tile
    }
    const uint32_t cap_rows = min(table_bytes / (2u * S * kChunkWords), kMaxTileChunks);
    if (cap_rows == 0) {  // the host sizes the table for at least one chunk; never loop without progress
        if (threadIdx.x == 0) atomicOr(sm.err, kErrTableTooSmall);
        return;
    }
    // With room for a 32-bit mask per column (the rows that hold an entry
    // there), the same-block probe pass reads only those rows' entries instead
    // of every pending partner's; taken when the program's blocks are alike
    // (one block pass probes every pending pair), rows have three or more
    // pending partners on average (fewer cost less than the masks do) and the
    // masks cost no extra tile.  (When blocks differ, or in the cross-block
    // pass, many block passes each probe a few pairs, which the per-partner
    // test below handles for less.)
    const uint32_t cap_masks = min(table_bytes / ((2u * S + 4u) * kChunkWords), kMaxTileChunks);
    const uint32_t n_chunks = __popcll(chunks);
    const bool col_rows = !kInter && P.blk_invariant && sm.pass_pend >= 3u * n_rows && cap_masks > 0 &&
                          (n_chunks + cap_masks - 1u) / cap_masks == (n_chunks + cap_rows - 1u) / cap_rows;
    const uint32_t cap = col_rows ? cap_masks : cap_rows;
    const uint32_t n_segs = n_rows * nb;
    const bool one_batch = n_segs <= kSegCap;
    uint64_t pending = chunks;
    while (pending) {
        uint64_t sel = 0;
        uint32_t k = 0;
        while (pending && k < cap) {
            const uint64_t low = pending & (~pending + 1ull);
            sel |= low;
            pending ^= low;
            ++k;
        }
        const uint32_t cols = k * kChunkWords;
        // tile slot of each chunk of the tile (0xFF: not in it); the column
        // ranges below take it from sel directly, so one barrier serves both
        auto slot_of = [sel](uint32_t ch) -> uint32_t {
            return ((sel >> ch) & 1ull) ? (uint32_t)__popcll(sel & ((1ull << ch) - 1ull)) : 0xFFu;
        };
        if (threadIdx.x < 64) sm.chunk_slot[threadIdx.x] = (uint8_t)slot_of(threadIdx.x);
        // column range of each row within this tile (the tile keeps address order)
        if (threadIdx.x < 32) {
            const uint32_t st = threadIdx.x;
            uint32_t c0 = 1, c1 = 0;
            const uint32_t lo = sm.rlo[st], hi = sm.rhi[st];
            if (st < S && ((rows >> st) & 1u) && lo <= hi) {
                const uint32_t k0 = lo >> kChunkShift, k1 = hi >> kChunkShift;
                for (uint32_t ch = k0; ch <= k1; ++ch) {
                    const uint32_t slot = slot_of(ch);
                    if (slot != 0xFFu) {
                        c0 = slot * kChunkWords + (ch == k0 ? (lo & (kChunkWords - 1u)) : 0u);
                        break;
                    }
                }
                for (uint32_t ch = k1 + 1; ch-- > k0;) {
                    const uint32_t slot = slot_of(ch);
                    if (slot != 0xFFu) {
                        c1 = slot * kChunkWords + (ch == k1 ? (hi & (kChunkWords - 1u)) : kChunkWords - 1u);
                        break;
                    }
                }
                if (c0 > c1) {
                    c0 = 1;
                    c1 = 0;
                }
            }
            sm.clo[st] = c0;
            sm.chi[st] = c1;
        }
        __syncthreads();
        // clear each row over the word-aligned span of its column range (a warp per row)
        for (uint32_t r = warp; r < n_rows; r += nwarps) {
            const uint32_t st = sm.row_list[r];
            const uint32_t c0 = sm.clo[st], c1 = sm.chi[st];
            if (c0 > c1) continue;
            uint32_t *row32 = reinterpret_cast<uint32_t *>(tab + (size_t)st * cols);
            for (uint32_t w = (c0 >> 1) + lane; w <= (c1 >> 1); w += 32) row32[w] = 0xFFFFFFFFu;
        }
        // the column masks follow the S rows: (2 S + 4) bytes per column in all
        uint32_t *colrows = reinterpret_cast<uint32_t *>(tab + (size_t)S * cols);
        if (col_rows)
            for (uint32_t w = threadIdx.x; w < cols; w += blockDim.x) colrows[w] = 0;
        // pass 0: each access installs its owner with a CAS on an empty entry;
        //         one that finds another owner stores MULTI (an entry only ever
        //         goes empty -> one owner -> MULTI, so the end state is exact);
        // pass 1: probe the pending partners.
        // When the tile holds every remaining chunk and they are chunks 0..k-1
        // of the address space, every access is in the tile and the column of
        // an address is the address itself.
        const bool identity = pending == 0 && sel == ((k >= 64) ? ~0ull : ((1ull << k) - 1ull));
        uint4 held0 = make_uint4(0, 0, 0, 0), held1 = held0;
        for (uint32_t pass = 0; pass < 2; ++pass) {
            for (uint32_t base = 0; base < n_segs; base += kSegCap) {
                // with every remaining chunk in the tile each segment meets it
                // (a segment with no active thread has none in any chunk), so
                // the identity tile needs no segment list
                if (!identity && (pass == 0 || !one_batch)) {
                    // segments of this batch whose chunks meet the tile
                    __syncthreads();
                    if (threadIdx.x == 0) sm.n_seg_list = 0;
                    __syncthreads();
                    const uint32_t end = min(n_segs, base + kSegCap);
                    for (uint32_t g = base + warp * 32u; g < end; g += nwarps * 32u) {
                        const uint32_t u = g + lane;
                        bool keep = false;
                        uint32_t code = 0;
                        if (u < end) {
                            const uint32_t r = u / nb, bi = u - r * nb;
                            const uint32_t st = sm.row_list[r];
                            keep = (segmask[(size_t)st * B + blk_lo + bi] & sel) != 0;
                            code = (st << 16) | bi;
                        }
                        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
                        uint32_t at = 0;
                        if (lane == 0 && bal) at = atomicAdd(&sm.n_seg_list, __popc(bal));
                        at = __shfl_sync(0xFFFFFFFFu, at, 0);
                        if (keep) sm.seg_list[at + __popc(bal & ((1u << lane) - 1u))] = code;
                    }
                }
                // publishes the segment list, or orders pass 0's installs after
                // the clear; pass 1 without a new list follows pass 0's barrier
                if (pass == 0 || (!identity && !one_batch)) __syncthreads();
                const uint32_t n_list = identity ? min(n_segs - base, kSegCap) : sm.n_seg_list;
                const uint32_t units = n_list * nv;
                const bool hold = one_batch && units <= 2u * blockDim.x;
                uint32_t slot_i = 0;
                for (uint32_t u = threadIdx.x; u < units; u += blockDim.x, ++slot_i) {
                    const uint32_t v = u % nv;
                    uint32_t st, blk;
                    if (identity) {
                        const uint32_t g = base + u / nv, r = g / nb;
                        st = sm.row_list[r];
                        blk = blk_lo + (g - r * nb);
                    } else {
                        const uint32_t code = sm.seg_list[u / nv];
                        st = code >> 16;
                        blk = blk_lo + (code & 0xFFFFu);
                    }
                    const uint32_t act8 = (sm.act[st][v >> 2] >> ((v & 3u) * 8u)) & 0xFFu;
                    if (!act8) continue;
                    uint32_t pend = 0;
                    if (pass == 1) {
                        pend = sm.rep_pend[st] & ~*(volatile uint32_t *)&sm.rep_conf[st];
                        if (!pend) continue;
                    }
                    uint4 q;
                    if (pass > 0 && hold) {
                        q = slot_i ? held1 : held0;
                    } else {
                        q = __ldg(reinterpret_cast<const uint4 *>(trace + ((size_t)st * B + blk) * tpad) + v);
                        if (slot_i) held1 = q; else held0 = q;
                    }
                    const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
                    if (pass == 0) {
                        uint16_t *row = tab + (size_t)st * cols;
#pragma unroll
                        for (uint32_t e = 0; e < 8; ++e) {
                            if (!((act8 >> e) & 1u)) continue;
                            const uint32_t a = (w4[e >> 1] >> ((e & 1u) * 16u)) & 0xFFFFu;
                            uint32_t idx;
                            if (identity) {
                                idx = a;
                            } else {
                                const uint32_t slot = sm.chunk_slot[a >> kChunkShift];
                                if (slot == 0xFFu) continue;
                                idx = slot * kChunkWords + (a & (kChunkWords - 1u));
                            }
                            const uint16_t owner = kInter ? (uint16_t)blk : (uint16_t)(v * 8u + e);
                            const uint16_t old = atomicCAS(row + idx, kEmpty, owner);
                            if (old == kEmpty) {
                                if (col_rows) atomicOr(&colrows[idx], 1u << st);  // the row's first entry here
                            } else if (old != owner) {
                                row[idx] = kMulti;
                            }
                        }
                    } else {
                        uint32_t col[8];
#pragma unroll
                        for (uint32_t e = 0; e < 8; ++e) {
                            const uint32_t a = (w4[e >> 1] >> ((e & 1u) * 16u)) & 0xFFFFu;
                            if (identity) {
                                col[e] = ((act8 >> e) & 1u) ? a : 0xFFFFFFFFu;
                            } else {
                                const uint32_t slot = sm.chunk_slot[a >> kChunkShift];
                                col[e] = (((act8 >> e) & 1u) && slot != 0xFFu)
                                             ? slot * kChunkWords + (a & (kChunkWords - 1u)) : 0xFFFFFFFFu;
                            }
                        }
                        if (col_rows) {
                            // at each access, the pending partners holding an
                            // entry at its column; an entry not its own is a hit
                            uint32_t hits = 0;
#pragma unroll
                            for (uint32_t e = 0; e < 8; ++e) {
                                const uint32_t c = col[e];
                                if (c == 0xFFFFFFFFu) continue;
                                const uint32_t mine = kInter ? blk : (v * 8u + e);
                                uint32_t t = colrows[c] & pend & ~hits;
                                if (t) t &= ~*(volatile uint32_t *)&sm.rep_conf[st];  // found by another unit
                                for (; t; t &= t - 1u) {
                                    const uint32_t j = __ffs(t) - 1u;
                                    const uint32_t o = tab[(size_t)j * cols + c];
                                    if (o != kEmpty && o != mine) hits |= 1u << j;
                                }
                            }
                            if (hits) atomicOr(&sm.rep_conf[st], hits);
                            continue;
                        }
                        for (uint32_t jt = pend; jt; jt &= jt - 1u) {
                            const uint32_t j = __ffs(jt) - 1u;
                            if ((*(volatile uint32_t *)&sm.rep_conf[st] >> j) & 1u) continue;
                            const uint32_t c0 = sm.clo[j], c1 = sm.chi[j];
                            const uint16_t *rj = tab + (size_t)j * cols;
                            bool hit = false;
#pragma unroll
                            for (uint32_t e = 0; e < 8; ++e) {
                                const uint32_t c = col[e];
                                if (c >= c0 && c <= c1) {  // j's entries outside its range are stale
                                    const uint32_t o = rj[c];
                                    const uint32_t mine = kInter ? blk : (v * 8u + e);
                                    hit |= o != kEmpty && o != mine;
                                }
                            }
                            if (hit) atomicOr(&sm.rep_conf[st], 1u << j);
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    // pattern conflicts back to statement pairs
    if (warp == 0) {
        const uint32_t i = lane;
        uint32_t conf = 0;
        for (uint32_t t = sm.pend_row[i]; t; t &= t - 1u) {
            const uint32_t j = __ffs(t) - 1u;
            const uint32_t ri = sm.prog.rep[i], rj = sm.prog.rep[j];
            if ((sm.rep_conf[min(ri, rj)] >> max(ri, rj)) & 1u) conf |= 1u << j;
        }
        if (conf) atomicOr(&rows_out[i], conf);
    }
    __syncthreads();
}

__device__ uint64_t block_chunks(const uint64_t *segmask, uint32_t B, uint32_t rows, uint32_t blk) {
    uint64_t m = 0;
    for (uint32_t t = rows; t; t &= t - 1u) m |= segmask[(size_t)(__ffs(t) - 1u) * B + blk];
    return m;
}

// Phase masks and the statements that share a phase with a write of their space.
__device__ void prepare_check(Smem &sm, uint32_t mask) {
    const DevProg &P = sm.prog;
    const uint32_t S = P.n_stmts;
    if (threadIdx.x < 32) {
        const uint32_t s = threadIdx.x, bit = 1u << s;
        sm.rows_intra[s] = 0;
        sm.rows_inter[s] = 0;
        uint32_t pi = 0, px = 0;
        if (s < S) {
            pi = phase_of(s, gap_mask(P, mask), S);
            px = phase_of(s, gap_mask(P, mask & P.grid_mask), S);
        }
        sm.ph_intra[s] = pi;
        sm.ph_inter[s] = px;
        // rows with a write in their phase (of their own array)
        const uint32_t sh = __ballot_sync(0xFFFFFFFFu, (P.shared_rows & bit) && (pi & P.shared_rows & P.write_mask));
        const uint32_t gi = __ballot_sync(0xFFFFFFFFu, (P.global_rows & bit) && (pi & P.global_rows & P.write_mask));
        const uint32_t gx = __ballot_sync(0xFFFFFFFFu, (P.global_rows & bit) && (px & P.global_rows & P.write_mask));
        if (s == 0) {
            sm.rel_sh = sh;
            sm.rel_gi = gi;
            sm.rel_gx = (P.blocks > 1) ? gx : 0u;
            sm.pairs = 0;
            sm.chunk_acc = 0;
            sm.diverge = 0;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ uint32_t tri_index(uint32_t i, uint32_t j, uint32_t S) {  // i <= j < S
    return i * S - (i * (i - 1u)) / 2u + (j - i);
}

// Thread pairs of each statement pair (i <= j, one space, a write): same-block
// and cross-block, independent of the mask; computed once per program.
__device__ void pair_counts(Smem &sm) {
    const DevProg &P = sm.prog;
    const uint32_t S = P.n_stmts;
    const uint64_t B = P.blocks;
    for (uint32_t idx = threadIdx.x; idx < S * S; idx += blockDim.x) {
        const uint32_t i = idx / S, j = idx - i * S;
        if (j < i) continue;
        const DevStmt &a = P.stmts[i], &b = P.stmts[j];
        uint64_t same = 0, cross = 0;
        if (a.space == b.space && (a.op == GR_W || b.op == GR_W)) {
            const uint64_t ni = sm.nact[i], nj = sm.nact[j];
            // threads active at both: one side unguarded, or one guard, needs no count
            uint64_t nij;
            if (a.gk == 0) nij = nj;
            else if (b.gk == 0 || (a.gk == b.gk && a.gr == b.gr)) nij = ni;
            else {
                nij = 0;
                const uint32_t nw = (P.threads + 31u) >> 5;
                for (uint32_t w = 0; w < nw; ++w) nij += __popc(sm.act[i][w] & sm.act[j][w]);
            }
            const bool global = a.space == GR_GLOBAL;
            if (i < j) {
                same = B * (ni * nj - nij);
                cross = global ? B * (B - 1) * ni * nj : 0;
            } else {
                same = B * (ni * (ni - 1) / 2);
                cross = global ? (B * (B - 1) / 2) * ni * ni : 0;
            }
        }
        const uint32_t t = tri_index(i, j, S);
        sm.npair[0][t] = same;
        sm.npair[1][t] = cross;
    }
    __syncthreads();
}

// Divergence (closed form over tid in [0, T)) and the access-pair count.
__device__ void check_misc(Smem &sm, uint32_t mask) {
    const DevProg &P = sm.prog;
    const uint32_t S = P.n_stmts, T = P.threads;
    if (threadIdx.x < 32) {  // lane k: does enabled guarded slot k diverge?
        const uint32_t k = threadIdx.x;
        bool dv = false;
        if (((mask & P.guarded_slots) >> k) & 1u) {
            const uint32_t gk = P.slot_gk[k], gr = P.slot_gr[k];
            const uint32_t cnt = T > gr ? (T - 1u - gr) / gk + 1u : 0u;
            dv = cnt > 0 && cnt < T;
        }
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, dv);
        if (k == 0) sm.diverge = b;
    }
    unsigned long long local = 0;
    const uint32_t gaps = gap_mask(P, mask), grid_gaps = gap_mask(P, mask & P.grid_mask);
    for (uint32_t idx = threadIdx.x; idx < S * S; idx += blockDim.x) {
        const uint32_t i = idx / S, j = idx - i * S;
        if (j < i) continue;
        const uint32_t rg = range_mask(i, j);
        const uint32_t t = tri_index(i, j, S);
        if ((gaps & rg) == 0) local += sm.npair[0][t];
        if ((grid_gaps & rg) == 0) local += sm.npair[1][t];
    }
    for (uint32_t o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xFFFFFFFFu, local, o);
    if ((threadIdx.x & 31u) == 0 && local) atomicAdd(&sm.pairs, local);
}

// Same-block passes for blocks [b0, b1) and, if requested, the cross-block pass.
// When every block sees one access pattern (blk_invariant: see the packer)
// the same-block witnesses of any block are block 0's, so only block 0 is
// checked.
__device__ void check_blocks(Smem &sm, uint16_t *tab, uint32_t table_bytes, const uint16_t *trace,
                             const uint64_t *segmask, const uint32_t *segrange, uint32_t b0, uint32_t b1,
                             bool inter) {
    const DevProg &P = sm.prog;
    const uint32_t B = P.blocks, S = P.n_stmts;
    if (P.blk_invariant) b1 = b0 == 0 ? min(b1, 1u) : b0;  // uniform
    const bool cached = b1 - b0 <= 64;
    if (cached) {  // chunk masks of every block of the range, OR-reduced in parallel
        __syncthreads();
        for (uint32_t u = threadIdx.x; u < 128; u += blockDim.x) (&sm.bchunk[0][0])[u] = 0;
        __syncthreads();
        const uint32_t nb = b1 - b0;
        for (uint32_t u = threadIdx.x; u < S * nb; u += blockDim.x) {
            const uint32_t s = u / nb, bi = u - s * nb;
            const uint32_t bit = 1u << s;
            if (!((sm.rel_sh | sm.rel_gi) & bit)) continue;
            const uint64_t m = segmask[(size_t)s * B + b0 + bi];
            if (m) atomicOr(&sm.bchunk[(sm.rel_sh & bit) ? 0 : 1][bi], m);
        }
        __syncthreads();
    }
    for (uint32_t blk = b0; blk < b1; ++blk) {
        if (sm.rel_sh) {
            const uint64_t ch = cached ? sm.bchunk[0][blk - b0] : block_chunks(segmask, B, sm.rel_sh, blk);
            owner_pass<false>(sm, tab, table_bytes, trace, segmask, segrange, sm.rel_sh, blk, 1, ch, sm.ph_intra,
                              sm.rows_intra);
        }
        if (sm.rel_gi) {
            const uint64_t ch = cached ? sm.bchunk[1][blk - b0] : block_chunks(segmask, B, sm.rel_gi, blk);
            owner_pass<false>(sm, tab, table_bytes, trace, segmask, segrange, sm.rel_gi, blk, 1, ch, sm.ph_intra,
                              sm.rows_intra);
        }
    }
    if (inter && sm.rel_gx) {
        __syncthreads();
        unsigned long long m = 0;
        for (uint32_t u = threadIdx.x; u < S * B; u += blockDim.x) {
            const uint32_t st = u / B;
            if ((sm.rel_gx >> st) & 1u) m |= segmask[u];
        }
        if (m) atomicOr(&sm.chunk_acc, m);
        __syncthreads();
        owner_pass<true>(sm, tab, table_bytes, trace, segmask, segrange, sm.rel_gx, 0, B, sm.chunk_acc, sm.ph_inter,
                         sm.rows_inter);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Exact minimum-weight hitting set
// ---------------------------------------------------------------------------

// Least (weight, mask) with forced <= mask, mask & forbidden == 0, hitting
// every clause of mh_cl(sm)[0..n_cl) and containing no negative clause neg[0..n_neg).
// Result in sm.sol_found / sol_mask / sol_weight.  All threads must call.
__device__ void mhs_solve(Smem &sm, MhsSmem &mh, uint32_t n_vars, const uint32_t *w, uint32_t n_cl,
                          const uint32_t *neg, uint32_t n_neg, uint32_t forced, uint32_t forbidden) {
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    __syncthreads();
    if (tid == 0) {
        mh.n_kept = 0;
        mh.n_negk = 0;
        mh.R = 0;
        mh.U = 0;
        mh.unsat = (forced & forbidden) ? 1u : 0u;
        sm.best = ~0ull;
    }
    if (tid < 33) mh.size_at[tid] = 0;
    __syncthreads();
    for (uint32_t i = tid; i < n_cl; i += nt) {
        const uint32_t c = mh_cl(sm)[i];
        uint32_t pc = 0;
        if (!(c & forced)) {
            pc = c & ~forbidden;
            if (!pc) mh.unsat = 1;
            else atomicAdd(&mh.size_at[__popc(pc)], 1u);
        }
        mh.pc[i] = pc;
    }
    __syncthreads();
    if (mh.unsat) {
        if (tid == 0) sm.sol_found = 0;
        __syncthreads();
        return;
    }
    // the remaining clauses in order of size (counting sort): the first of
    // each size by an exclusive scan, then each clause to its place
    if (tid < 32) {
        const uint32_t v = mh.size_at[tid + 1u];
        uint32_t incl = v;
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (tid >= o) incl += t;
        }
        mh.size_at[tid + 1u] = incl - v;
    }
    __syncthreads();
    for (uint32_t i = tid; i < n_cl; i += nt) {
        const uint32_t pc = mh.pc[i];
        if (pc) mh.set[atomicAdd(&mh.size_at[__popc(pc)], 1u)] = pc;
    }
    __syncthreads();
    // drop every clause that contains another one.  In size order only an
    // earlier clause can be a subset (of two equal clauses the later one is
    // dropped), and the small clauses that drop most others come first.
    const uint32_t n_sorted = mh.size_at[32];  // the end of the last size
    const uint32_t *sorted = mh.set;
    const uint4 *sorted4 = reinterpret_cast<const uint4 *>(mh.set);
    for (uint32_t i = tid; i < n_sorted; i += nt) {
        const uint32_t c = sorted[i];
        bool keep = true;
        for (uint32_t j = 0; j < i && keep; j += 4u) {
            const uint4 d = sorted4[j >> 2];
            keep = (d.x & ~c) != 0 && (j + 1u >= i || (d.y & ~c) != 0) && (j + 2u >= i || (d.z & ~c) != 0) &&
                   (j + 3u >= i || (d.w & ~c) != 0);
        }
        if (keep) {
            if ((c & (c - 1u)) == 0) {
                atomicOr(&mh.U, c);  // unit clause: its slot is on in every solution
            } else {
                const uint32_t k = atomicAdd(&mh.n_kept, 1u);
                mh.khi[k] = c;
                atomicOr(&mh.R, c);
            }
        }
    }
    __syncthreads();
    // a kept clause never contains a unit's slot (the unit subsumes it), so the
    // units join the forced set and the search runs over the other variables
    forced |= mh.U;
    const uint32_t R = mh.R;
    // variables outside every clause stay off; a negative clause with such a
    // variable can never be violated; one inside the forced set always is
    for (uint32_t i = tid; i < n_neg; i += nt) {
        const uint32_t N = neg[i];
        if (N & forbidden) continue;
        const uint32_t v = N & ~forced;
        if (!v) {
            mh.unsat = 1;
        } else if ((v & ~R) == 0) {
            const uint32_t k = atomicAdd(&mh.n_negk, 1u);
            mh.nhi[k] = v;
        }
    }
    __syncthreads();
    if (mh.unsat) {
        if (tid == 0) sm.sol_found = 0;
        __syncthreads();
        return;
    }
    const uint32_t r = __popc(R);
    const uint32_t L = r < 5 ? r : 5;
    const uint32_t rh = r - L;
    const uint32_t lomask = (1u << L) - 1u;
    if (tid < GR_MAX_SLOTS) {
        uint32_t v = 0;
        if (tid < r) {
            uint32_t t = R;
            for (uint32_t q = 0; q < tid; ++q) t &= t - 1u;
            v = w[__ffs(t) - 1u];
        }
        mh.wc[tid] = v;
    }
    __syncthreads();
    const uint32_t n_kept = mh.n_kept, n_negk = mh.n_negk;
    for (uint32_t k = tid; k < n_kept; k += nt) {
        const uint32_t c = pext32(mh.khi[k], R);
        uint32_t lo = 0;
        for (uint32_t b = 0; b < L; ++b)
            if ((c >> b) & 1u) lo |= low_pattern(b);
        mh.khi[k] = c >> L;
        mh.klo[k] = lo;
    }
    for (uint32_t k = tid; k < n_negk; k += nt) {
        const uint32_t c = pext32(mh.nhi[k], R);
        uint32_t lo = 0xFFFFFFFFu;
        for (uint32_t b = 0; b < L; ++b)
            if ((c >> b) & 1u) lo &= low_pattern(b);
        mh.nhi[k] = c >> L;
        mh.nlo[k] = lo;
    }
    if (tid < 32) {
        uint32_t v = 0;
        for (uint32_t b = 0; b < L; ++b)
            if ((tid >> b) & 1u) v += mh.wc[b];
        mh.wlo[tid] = v;
    }
    for (uint32_t e = tid; e < 4 * 256; e += nt) {
        const uint32_t q = e >> 8, byte = e & 255u;
        if (q * 8u >= rh && byte) continue;  // bytes past the high part are zero: only entry 0 is read
        uint32_t v = 0;
        for (uint32_t b = 0; b < 8; ++b) {
            const uint32_t hb = q * 8u + b;
            if (((byte >> b) & 1u) && hb < rh) v += mh.wc[L + hb];
        }
        mh.w8[q][byte] = v;
    }
    if (tid < 32) {
        // lb[k] = the sum of the k lightest high weights: each lane puts its
        // weight at its rank (ties by index), then an inclusive scan
        const uint32_t v = tid < rh ? mh.wc[L + tid] : 0u;
        if (tid < rh) {
            uint32_t rank = 0;
            for (uint32_t j = 0; j < rh; ++j) {
                const uint32_t u = mh.wc[L + j];
                rank += (u < v || (u == v && j < tid)) ? 1u : 0u;
            }
            mh.lb[rank + 1u] = v;
        }
        __syncwarp();
        uint32_t acc = tid < rh ? mh.lb[tid + 1u] : 0u;
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, acc, o);
            if (tid >= o) acc += t;
        }
        if (tid < rh) mh.lb[tid + 1u] = acc;
        if (tid == 0) mh.lb[0] = 0;
    }
    __syncthreads();
    const uint32_t VL = L == 5 ? 0xFFFFFFFFu : ((1u << (1u << L)) - 1u);
    (void)lomask;
    for (uint32_t kh = 0; kh <= rh; ++kh) {
        const unsigned long long cur = *(volatile unsigned long long *)&sm.best;
        if (cur != ~0ull && (unsigned long long)mh.lb[kh] > (cur >> 32)) break;  // uniform
        const uint32_t total = c_binom.v[rh][kh];
        const uint32_t per = (total + nt - 1u) / nt;
        const uint32_t start = tid * per;
        const uint32_t end = min(total, start + per);
        unsigned long long local = cur;
        if (start < end) {
            uint32_t h = unrank_colex(start, kh, rh);
            for (uint32_t idx = start; idx < end; ++idx) {
                const uint32_t wh = mh.w8[0][h & 255u] + mh.w8[1][(h >> 8) & 255u] + mh.w8[2][(h >> 16) & 255u] +
                                    mh.w8[3][h >> 24];
                const uint64_t lw = local >> 32;
                bool skip = (uint64_t)wh > lw || ((uint64_t)wh == lw && (h << L) > (uint32_t)local);
                if (!skip) {
                    uint32_t F = VL;
                    for (uint32_t c = 0; c < n_kept; ++c) {
                        if ((mh.khi[c] & h) == 0) {
                            F &= mh.klo[c];
                            if (!F) break;
                        }
                    }
                    if (F)
                        for (uint32_t c = 0; c < n_negk; ++c)
                            if ((mh.nhi[c] & ~h) == 0) F &= ~mh.nlo[c];
                    while (F) {
                        const uint32_t l = __ffs(F) - 1u;
                        F &= F - 1u;
                        const unsigned long long key =
                            ((unsigned long long)(wh + mh.wlo[l]) << 32) | (unsigned long long)((h << L) | l);
                        if (key < local) local = key;
                    }
                }
                if (idx + 1u < end) h = gosper_next(h);
            }
        }
        if (local < cur) atomicMin(&sm.best, local);
        __syncthreads();
    }
    if (tid == 0) {
        const unsigned long long b = sm.best;
        if (b == ~0ull) {
            sm.sol_found = 0;
        } else {
            const uint32_t x = pdep32((uint32_t)b, R) | forced;
            uint32_t wt = (uint32_t)(b >> 32);
            for (uint32_t t = forced; t; t &= t - 1u) wt += w[__ffs(t) - 1u];
            (void)n_vars;
            sm.sol_found = 1;
            sm.sol_mask = x;
            sm.sol_weight = wt;
        }
    }
    __syncthreads();
}

// The mhs strategy's proposal (Section 2.4, after Johnson 1974): starting from
// the forced slots, repeatedly take the allowed slot that hits the most clauses
// not yet hit per unit of weight (cross-multiplied ratios, ties to the lower
// slot), then drop, from the highest slot down, every non-forced slot whose
// removal leaves every clause hit.  sm.sol_found = 0 when a clause has no
// allowed slot (or a forced slot is forbidden).  All threads must call.
__device__ void mhs_greedy(Smem &sm, MhsSmem &mh, uint32_t n_vars, const uint32_t *w, uint32_t n_cl,
                           uint32_t forced, uint32_t forbidden) {
    const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = tid & 31u;
    const uint32_t *cl = mh.cl;
    uint32_t *cnt = mh.wlo;  // hit counts per slot (the exact solver's table is free here)
    __syncthreads();
    if (tid == 0) {
        mh.unsat = (forced & forbidden) ? 1u : 0u;
        mh.R = forced;
        mh.n_kept = 0;
    }
    __syncthreads();
    for (uint32_t i = tid; i < n_cl; i += nt)
        if (!(cl[i] & forced) && !(cl[i] & ~forbidden)) mh.unsat = 1;
    __syncthreads();
    if (mh.unsat) {
        if (tid == 0) sm.sol_found = 0;
        __syncthreads();
        return;
    }
    // every warp sweeps whole rounds of 32 clauses so that its ballots see full lanes
    const uint32_t rounds = (n_cl + 31u) >> 5;
    for (;;) {
        const uint32_t x = *(volatile uint32_t *)&mh.R;
        if (tid < 32) cnt[tid] = 0;
        __syncthreads();
        // lane v: the clauses not yet hit that slot v would hit, by one ballot
        // per slot present in 32 clauses, then one atomic per lane and warp
        uint32_t hits = 0;
        for (uint32_t r = tid >> 5; r < rounds; r += nt >> 5) {
            const uint32_t i = r * 32u + lane;
            const uint32_t m = (i < n_cl && !(cl[i] & x)) ? (cl[i] & ~forbidden) : 0u;
            for (uint32_t vs = __reduce_or_sync(0xFFFFFFFFu, m); vs; vs &= vs - 1u) {
                const uint32_t v = __ffs(vs) - 1u;
                const uint32_t n = __popc(__ballot_sync(0xFFFFFFFFu, (m >> v) & 1u));
                if (lane == v) hits += n;
            }
        }
        if (hits) atomicAdd(&cnt[lane], hits);
        __syncthreads();
        if (tid < 32) {
            // lane k's candidate; reduce to the best by hits/weight, ties to the lower slot
            uint32_t h = (lane < n_vars && !((x >> lane) & 1u) && !((forbidden >> lane) & 1u)) ? cnt[lane] : 0u;
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
            if (lane == 0) {
                if (h) mh.R = x | (1u << k);
                else mh.n_kept = 1;  // every clause is hit
            }
        }
        __syncthreads();
        if (mh.n_kept) break;
    }
    uint32_t x = mh.R;
    for (int k = (int)n_vars - 1; k >= 0; --k) {
        if (!((x >> k) & 1u) || ((forced >> k) & 1u)) continue;
        const uint32_t y = x & ~(1u << k);
        bool ok = true;
        for (uint32_t i = tid; i < n_cl && ok; i += nt) ok = (cl[i] & y) != 0;
        if (__syncthreads_and(ok)) x = y;
    }
    if (tid == 0) {
        uint32_t wt = 0;
        for (uint32_t t = x; t; t &= t - 1u) wt += w[__ffs(t) - 1u];
        sm.sol_found = 1;
        sm.sol_mask = x;
        sm.sol_weight = wt;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Loop steps (Algorithm 1)
// ---------------------------------------------------------------------------

// Insert clause c into the clause set; a clause already there is not listed
// again.  Linear probing over a table at least twice the largest clause count
// (2 x 25 x 26 / 2 = 650 witness pairs), so every probe sequence meets an
// empty entry; kNoClause, itself a clause (all 32 slots), is tracked apart.
__device__ __forceinline__ void add_clause(Smem &sm, MhsSmem &mh, uint32_t c) {
    bool fresh = true;
    if (c == kNoClause) {
        fresh = atomicExch(&mh.full_seen, 1u) == 0u;
    } else {
        uint32_t h = (c * 0x9E3779B1u) >> (32u - kClauseSetLog2);  // Fibonacci hashing
        for (uint32_t q = 0; q < kClauseSet; ++q) {
            const uint32_t prev = atomicCAS(&mh.set[h], kNoClause, c);
            if (prev == kNoClause) break;
            if (prev == c) {
                fresh = false;
                break;
            }
            h = (h + 1u) & (kClauseSet - 1u);
        }
    }
    if (fresh) mh_cl(sm)[atomicAdd(&sm.n_cl, 1u)] = c;
}

// Clause list from the accumulated witnesses: same-block (i, j) -> the slots
// whose barriers run in gaps i..j-1 (slots i..j-1 without loops); cross-block
// (i, j) -> the grid slots among them (GenerateClause).  The list holds each
// distinct clause once: the clauses form a set, so the greedy strategy's hit
// counts count distinct clauses.
__device__ void build_clauses(Smem &sm) {
    const DevProg &P = sm.prog;
    const uint32_t S = P.n_stmts;
    MhsSmem &mh = *reinterpret_cast<MhsSmem *>(reinterpret_cast<uint8_t *>(&sm) + kFixedSmem);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kClauseSet; i += blockDim.x) mh.set[i] = kNoClause;
    if (threadIdx.x == 0) {
        sm.n_cl = 0;
        mh.full_seen = 0;
    }
    __syncthreads();
    for (uint32_t idx = threadIdx.x; idx < S * S; idx += blockDim.x) {
        const uint32_t i = idx / S, j = idx - i * S;
        if (j < i) continue;
        const uint32_t rg = slots_of_gaps(P, range_mask(i, j));
        if ((sm.acc_intra[i] >> j) & 1u) add_clause(sm, mh, rg);
        if ((sm.acc_inter[i] >> j) & 1u) add_clause(sm, mh, rg & P.grid_mask);
    }
    __syncthreads();
}

// Initial state: remove mode probes E; repair mode starts at MHS(empty) = E.
__device__ void loop_init(Smem &sm, const gr_options &opts) {
    const DevProg &P = sm.prog;
    if (threadIdx.x == 0) {
        sm.forced = P.mode == GR_MODE_REPAIR ? P.existing : 0u;
        sm.forbidden = opts.grid_enabled ? 0u : P.grid_mask;
        sm.max_iters = opts.max_iters == 0 ? GR_MAX_ITERS : min(opts.max_iters, (uint32_t)GR_MAX_ITERS);
        sm.iters = 0;
        sm.done = 0;
        sm.status = GR_REPAIRED;
        sm.access_pairs = 0;
        sm.n_cl = 0;
        sm.t_start = globaltimer();
        sm.deadline_ns = opts.deadline_us * 1000ull;
        sm.probe = P.mode == GR_MODE_REMOVE ? 1u : 0u;
        sm.greedy = opts.strategy == GR_STRATEGY_MHS ? 1u : 0u;
        sm.mask = P.existing;
    }
    if (threadIdx.x < 32) {
        sm.acc_intra[threadIdx.x] = 0;
        sm.acc_inter[threadIdx.x] = 0;
    }
    __syncthreads();
    if (P.mode != GR_MODE_REMOVE && threadIdx.x == 0) {
        // Solve over no positive clause: every admissible mask contains the
        // forced set, so the forced set itself is the lowest key, unless it
        // meets a forbidden slot or holds all slots of a negative clause (then
        // so does every mask containing it)
        bool ok = (sm.forced & sm.forbidden) == 0u;
        for (uint32_t c = 0; c < P.n_neg && ok; ++c)
            if ((sm.forced & P.neg[c]) == P.neg[c]) ok = false;
        if (ok) {
            sm.mask = sm.forced;
        } else {
            sm.status = GR_UNREPAIRABLE;
            sm.done = 1;
        }
    }
    if (threadIdx.x == 0 && !sm.done && sm.iters >= sm.max_iters) {
        sm.status = GR_ITER_CAP;
        sm.done = 1;
    }
    __syncthreads();
}

// After a check (witnesses in rows_*, diverge, pairs): record it, stop if the
// proposed mask is clean, else add the clauses and solve for the next mask.
__device__ void loop_step(Smem &sm, MhsSmem &mh) {
    const DevProg &P = sm.prog;
    __syncthreads();
    if (threadIdx.x < 32) {  // lane i: witness row i (rows past the instances are zero)
        const uint32_t i = threadIdx.x;
        const uint32_t ra = sm.rows_intra[i], re = sm.rows_inter[i];
        const bool clean = !__any_sync(0xFFFFFFFFu, (ra | re) != 0u) && !sm.diverge && !sm.probe;
        if (!clean) {
            sm.acc_intra[i] |= ra;
            sm.acc_inter[i] |= re;
        }
        __syncwarp();  // every lane has read probe before lane 0 clears it
        if (i == 0) {
            sm.traj[sm.iters] = sm.mask;
            sm.iters += 1;
            sm.access_pairs += sm.pairs;
            sm.step = 0;  // a new proposal is needed
            if (clean) {
                if (sm.greedy) {  // a clean greedy proposal: one exact query decides
                    sm.greedy = 0;
                    sm.step = 1;
                } else {
                    sm.status = GR_REPAIRED;
                    sm.done = 1;
                    sm.step = 2;
                }
            } else {
                sm.probe = 0;
                sm.forbidden |= sm.diverge;
            }
        }
    }
    __syncthreads();
    const uint32_t step = sm.step;
    if (step == 2) return;
    build_clauses(sm);
    bool solved = false;
    if (step == 0 && sm.greedy) {
        mhs_greedy(sm, mh, P.n_slots, P.weights, sm.n_cl, sm.forced, sm.forbidden);
        // a greedy set that breaks a negative clause falls back to the MaxSAT solve
        bool ok = sm.sol_found != 0;
        for (uint32_t c = 0; c < P.n_neg && ok; ++c)
            if ((sm.sol_mask & P.neg[c]) == P.neg[c]) ok = false;
        solved = ok;
    }
    if (!solved) mhs_solve(sm, mh, P.n_slots, P.weights, sm.n_cl, P.neg, P.n_neg, sm.forced, sm.forbidden);
    if (threadIdx.x == 0) {
        if (step == 1 && (!sm.sol_found || sm.sol_mask == sm.mask)) {
            sm.status = GR_REPAIRED;  // the greedy proposal is the minimum
            sm.done = 1;
        } else if (!sm.sol_found) {
            sm.status = GR_UNREPAIRABLE;
            sm.done = 1;
        } else {
            sm.mask = sm.sol_mask;
            if (sm.iters >= sm.max_iters) {
                sm.status = GR_ITER_CAP;
                sm.done = 1;
            } else if (sm.deadline_ns && globaltimer() - sm.t_start >= sm.deadline_ns) {
                sm.status = GR_TIMEOUT;
                sm.done = 1;
            }
        }
    }
    __syncthreads();
}

// The program's result: status, mask, weight, the sorted unique clause list,
// the trajectory and the counters.
__device__ void write_result(Smem &sm, gr_repair_result *out) {
    const DevProg &P = sm.prog;
    build_clauses(sm);
    // the listed clauses are distinct: each goes straight to its rank
    const uint32_t n_unique = sm.n_cl;
    const uint32_t *cl = mh_cl(sm);
    for (uint32_t i = threadIdx.x; i < n_unique; i += blockDim.x) {
        const uint32_t c = cl[i];
        uint32_t pos = 0;
        for (uint32_t j = 0; j < n_unique; ++j) pos += cl[j] < c ? 1u : 0u;
        out->clauses[pos] = c;
    }
    for (uint32_t i = threadIdx.x + n_unique; i < GR_MAX_CLAUSES; i += blockDim.x) out->clauses[i] = 0;
    for (uint32_t i = threadIdx.x; i < GR_MAX_ITERS; i += blockDim.x) out->traj[i] = i < sm.iters ? sm.traj[i] : 0u;
    if (threadIdx.x == 0) {
        const bool ok = sm.status == GR_REPAIRED;
        const uint32_t m = ok ? sm.mask : 0u;
        uint32_t wt = 0;
        for (uint32_t t = m; t; t &= t - 1u) wt += P.weights[__ffs(t) - 1u];
        out->status = (int32_t)sm.status;
        out->mask = m;
        out->weight = wt;
        out->added = m & ~P.existing;
        out->removed = ok ? (P.existing & ~m) : 0u;
        out->iters = sm.iters;
        out->n_clauses = n_unique;
        out->forbidden = sm.forbidden;
        out->_pad = 0;
        out->access_pairs = sm.access_pairs;
        out->t_start_ns = sm.t_start;
        out->t_end_ns = globaltimer();
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// K0: CTAs take work items (runs of up to kItemSegs (statement, block)
// segments of one program, largest programs first, so that a few large
// programs spread over many CTAs and many small ones share them; or block 0
// of a program's shared-array statements when its blocks are alike); one
// warp per segment of t_pad threads.  Writes the u16 address trace, and per
// segment the mask of 1,024-word chunks and the [min, max] address of its
// active accesses (min > max when none is active).
__global__ void __launch_bounds__(256) k_expand(const uint8_t *__restrict__ arena, uint8_t *__restrict__ scratch,
                                                uint64_t scratch_bytes, uint32_t general_only) {
    const ArenaView V = view(arena);
    if (V.h->magic != kArenaMagic || scratch_bytes < V.h->scratch_bytes) {
        if (threadIdx.x == 0) atomicOr(reinterpret_cast<uint32_t *>(scratch) + 1, kErrArgs);
        return;
    }
    // the general programs' items come first: the relation kernel computes
    // the other programs' addresses itself
    const uint64_t n_items = general_only ? V.h->n_items_gen : V.h->n_items;
    const uint4 *items = reinterpret_cast<const uint4 *>(arena + V.h->items_off);
    uint16_t *traces = reinterpret_cast<uint16_t *>(scratch + V.h->scratch_trace_off);
    uint64_t *segmask = reinterpret_cast<uint64_t *>(scratch + V.h->scratch_segmask_off);
    uint32_t *segrange = reinterpret_cast<uint32_t *>(scratch + V.h->scratch_segrange_off);
    __shared__ __align__(16) DevStmt st_sh[GR_MAX_STMTS];  // filled by 16-byte stores
    __shared__ uint32_t mag_sh[GR_MAX_STMTS];               // floor((2^32 - 1) / M) of each statement
    __shared__ uint32_t hdr[4];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (uint64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const uint4 it = items[item];
        const DevProg &P = V.progs[it.x];
        __syncthreads();
        if (threadIdx.x < GR_MAX_STMTS * sizeof(DevStmt) / 16)
            reinterpret_cast<uint4 *>(st_sh)[threadIdx.x] = reinterpret_cast<const uint4 *>(P.stmts)[threadIdx.x];
        if (threadIdx.x == 0) {
            hdr[0] = P.blocks;
            hdr[1] = P.threads;
            hdr[2] = P.t_pad;
        }
        __syncthreads();
        if (threadIdx.x < GR_MAX_STMTS) mag_sh[threadIdx.x] = st_sh[threadIdx.x].m ? 0xFFFFFFFFu / st_sh[threadIdx.x].m : 0u;
        __syncthreads();
        const uint32_t B = hdr[0], T = hdr[1], tpad = hdr[2];
        // kind 0: segments it.y..it.z-1; kind 1: block 0 of the shared-array
        // statements it.y..it.z-1 (blocks alike: no other block is read)
        for (uint32_t u = it.y + warp; u < it.z; u += nwarps) {
            if (it.w == 1u && st_sh[u].space != GR_SHARED) continue;
            const uint32_t seg = it.w == 1u ? u * B : u;
            const uint32_t s = seg / B, blk = seg - s * B;
            const DevStmt &st = st_sh[s];
            const uint32_t M = st.m, mag = mag_sh[s];
            // cm, blk < 2^16: cm blk < 2^32; then + bm < 2^17
            const uint32_t base = mod_u32(mod_u32(st.cm * blk, M, mag) + st.bm, M, mag);
            const bool perm = st.kind == GR_PERM;
            const uint32_t step = perm ? 1u : st.am;
            uint16_t *out = traces + P.trace_off + (size_t)seg * tpad;
            uint64_t chunks = 0;
            uint32_t amin = 0xFFFFu, amax = 0;
            const uint32_t nv = tpad >> 3;
            // 32-bit arithmetic: step, base < M <= 65,536 and t < 1,024
            const uint32_t gk = st.gk, gr = st.gr, dx32 = mod_u32(step * 32u, M, mag), dg = mod_u32(step * 256u, M, mag);
            uint32_t xg = mod_u32(step * lane + base, M, mag);  // the address at t = lane of group 0
            // An unguarded affine or strided segment whose addresses do not
            // wrap (base + step (T - 1) < M) and step at most a chunk apart
            // touches every chunk from base's to its last address's: its mask
            // and range in closed form, and only the trace per unit.
            if (!perm && gk == 0 && step <= kChunkWords && base + step * (T - 1u) < M) {
                for (uint32_t v = lane; v < nv; v += 32) {
                    const uint32_t g = v >> 5, U = min(32u, nv - 32u * g), t0 = 256u * g + lane;
                    uint32_t x = xg;
                    const uint32_t dx = U == 32u ? dx32 : mod_u32(step * U, M, mag);
                    uint32_t w4[4] = {0, 0, 0, 0};
#pragma unroll
                    for (uint32_t e = 0; e < 8; ++e) {
                        const uint32_t a = t0 + U * e < T ? x : 0u;
                        w4[e >> 1] |= a << ((e & 1u) * 16u);
                        x += dx;
                        if (x >= M) x -= M;
                    }
                    xg += dg;
                    if (xg >= M) xg -= M;
                    reinterpret_cast<uint4 *>(out)[v] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
                }
                if (lane == 0) {
                    const uint32_t hi = base + step * (T - 1u), c0 = base >> kChunkShift, c1 = hi >> kChunkShift;
                    segmask[P.segmask_off + seg] = (c1 == 63u ? ~0ull : ((1ull << (c1 + 1u)) - 1ull)) & ~((1ull << c0) - 1ull);
                    segrange[P.segmask_off + seg] = base | (hi << 16);
                }
                continue;
            }
            for (uint32_t v = lane; v < nv; v += 32) {
                // unit v of group g holds threads 256 g + (v mod 32) + U e, e = 0..7
                // (U = the group's units), so that a warp's 32 units read 32
                // consecutive threads at each e
                const uint32_t g = v >> 5, U = min(32u, nv - 32u * g), t0 = 256u * g + lane;
                // x = (step * t + base) mod M and t mod gk, advanced by U threads at a time
                uint32_t x = xg;
                const uint32_t dx = U == 32u ? dx32 : mod_u32(step * U, M, mag);
                uint32_t m = gk ? t0 % gk : 0u;
                const uint32_t dm = gk ? U % gk : 0u;
                // the 8 indices first, so that a permutation's 8 table loads
                // (every index is below M, padding threads included) are in
                // flight together
                uint32_t av[8];
                uint8_t on = 0;
#pragma unroll
                for (uint32_t e = 0; e < 8; ++e) {
                    av[e] = x;
                    if (t0 + U * e < T && (gk == 0 || m == gr)) on |= (uint8_t)(1u << e);
                    x += dx;
                    if (x >= M) x -= M;
                    m += dm;
                    if (m >= gk) m -= gk;
                }
                if (perm) {
#pragma unroll
                    for (uint32_t e = 0; e < 8; ++e) av[e] = V.perm[st.perm_off + av[e]];
                }
                uint32_t w4[4] = {0, 0, 0, 0};
#pragma unroll
                for (uint32_t e = 0; e < 8; ++e) {
                    const uint32_t a = t0 + U * e < T ? av[e] : 0u;
                    if ((on >> e) & 1u) {
                        chunks |= 1ull << (a >> kChunkShift);
                        amin = min(amin, a);
                        amax = max(amax, a);
                    }
                    w4[e >> 1] |= (a & 0xFFFFu) << ((e & 1u) * 16u);
                }
                xg += dg;
                if (xg >= M) xg -= M;
                reinterpret_cast<uint4 *>(out)[v] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
            }
            const uint32_t lo32 = __reduce_or_sync(0xFFFFFFFFu, (uint32_t)chunks);
            const uint32_t hi32 = __reduce_or_sync(0xFFFFFFFFu, (uint32_t)(chunks >> 32));
            amin = __reduce_min_sync(0xFFFFFFFFu, amin);
            amax = __reduce_max_sync(0xFFFFFFFFu, amax);
            if (lane == 0) {
                segmask[P.segmask_off + seg] = ((uint64_t)hi32 << 32) | lo32;
                segrange[P.segmask_off + seg] = amin | (amax << 16);
            }
        }
    }
}

// Permutation windows of a packed batch: the leading pneed entries of each
// window a permutation statement reads must be distinct (the host checked
// that they are below M while converting them to u16).  CTAs take programs;
// per window a 65,536-bit map in shared memory marks the entries and the
// marks are counted.  The lowest failing program, plus `base`, is kept as
// its complement in *bad (atomicMax; 0 = none).
__global__ void __launch_bounds__(256) k_perm_check(const uint8_t *__restrict__ arena, uint32_t base,
                                                    uint32_t *__restrict__ bad) {
    const ArenaView V = view(arena);
    const uint32_t n = V.h->n_progs, tid = threadIdx.x;
    __shared__ uint32_t bits[GR_MAX_WORDS / 32];
    __shared__ uint32_t total, n_stmts;
    __shared__ __align__(16) DevStmt st_sh[GR_MAX_STMTS];  // filled by 16-byte stores
    for (uint32_t p = blockIdx.x; p < n; p += gridDim.x) {
        const DevProg &P = V.progs[p];
        __syncthreads();  // the previous program's statements are no longer read
        if (tid < GR_MAX_STMTS * sizeof(DevStmt) / 16)
            reinterpret_cast<uint4 *>(st_sh)[tid] = reinterpret_cast<const uint4 *>(P.stmts)[tid];
        if (tid == 0) n_stmts = P.n_stmts;
        __syncthreads();
        for (uint32_t s = 0; s < n_stmts; ++s) {
            const DevStmt &st = st_sh[s];
            if (st.kind != GR_PERM) continue;
            // equal instances share their window
            bool again = false;
            for (uint32_t q = 0; q < s && !again; ++q) again = st_sh[q].kind == GR_PERM && st_sh[q].perm_off == st.perm_off;
            if (again) continue;
            const uint32_t M = st.m, need = st.pneed, words = (M + 31u) >> 5;
            for (uint32_t i = tid; i < words; i += blockDim.x) bits[i] = 0;
            if (tid == 0) total = 0;
            __syncthreads();
            const uint16_t *tbl = V.perm + st.perm_off;
            for (uint32_t i = tid; i < need; i += blockDim.x) {
                const uint32_t v = tbl[i];
                if (v < M) atomicOr(&bits[v >> 5], 1u << (v & 31u));  // an entry past M marks nothing
            }
            __syncthreads();
            uint32_t c = 0;
            for (uint32_t i = tid; i < words; i += blockDim.x) c += __popc(bits[i]);
            c = __reduce_add_sync(0xFFFFFFFFu, c);
            if ((tid & 31u) == 0 && c) atomicAdd(&total, c);
            __syncthreads();
            if (tid == 0 && total != need) atomicMax(bad, ~(base + p));  // need distinct marks
            __syncthreads();  // the map and the count, before the next window clears them
        }
    }
}

struct Dyn {
    Smem *sm;
    uint16_t *tab;
    MhsSmem *mh;
};

__device__ __forceinline__ Dyn dyn_smem() {
    extern __shared__ uint4 dyn_raw[];
    Dyn d;
    d.sm = reinterpret_cast<Smem *>(dyn_raw);
    d.tab = reinterpret_cast<uint16_t *>(reinterpret_cast<uint8_t *>(dyn_raw) + kFixedSmem);
    d.mh = reinterpret_cast<MhsSmem *>(d.tab);
    return d;
}

// The checks of the batch's general part (a global array, or blocks that
// differ), one per work item of the arena's check list: a program, or a
// range of a program's blocks when its blocks differ (then its items OR
// their witness rows into the program's entry, which k_split_zero cleared,
// and each item first reads the pairs the others found, to skip them).  The
// item holding block 0 (primary) also takes the divergence, the pair count
// and the cross-block pass.  Under masks[p], or under the empty mask when
// masks is NULL: then the witness rows are the program's conflict relation,
// written to the scratch's relation area for the loop kernel (out == NULL)
// or to out.  Persistent: CTAs take items from a queue, largest first.
// Instantiated for several CTA shapes (threads x CTAs per SM); the host
// picks one per batch.
template <uint32_t NT, uint32_t MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_check(const uint8_t *__restrict__ arena, uint32_t n, const uint32_t *__restrict__ masks,
            uint8_t *__restrict__ scratch, uint64_t scratch_bytes, gr_witnesses *__restrict__ out,
            uint32_t table_bytes) {
    Dyn d = dyn_smem();
    Smem &sm = *d.sm;
    const ArenaView V = view(arena);
    uint32_t *ctrl = reinterpret_cast<uint32_t *>(scratch);
    if (!launch_matches(V, n, scratch_bytes)) {
        if (threadIdx.x == 0) atomicOr(&ctrl[1], kErrArgs);
        return;
    }
    const uint16_t *traces = reinterpret_cast<const uint16_t *>(scratch + V.h->scratch_trace_off);
    const uint64_t *segmask = reinterpret_cast<const uint64_t *>(scratch + V.h->scratch_segmask_off);
    const uint32_t *segrange = reinterpret_cast<const uint32_t *>(scratch + V.h->scratch_segrange_off);
    gr_witnesses *dst = out ? out : reinterpret_cast<gr_witnesses *>(scratch + V.h->scratch_rel_off);
    const uint4 *citems = reinterpret_cast<const uint4 *>(arena + V.h->citems_off);
    const uint32_t n_citems = V.h->n_citems;
    if (threadIdx.x == 0) sm.err = &ctrl[1];
    for (;;) {
        if (threadIdx.x == 0) sm.item = atomicAdd(&ctrl[0], 1u);
        __syncthreads();
        const uint32_t item = sm.item;
        if (item >= n_citems) break;
        const uint4 ci = citems[item];
        const uint32_t p = ci.x;
        const bool primary = (ci.w & kItemPrimary) != 0, split = (ci.w & kItemSplit) != 0;
        load_program(sm, &V.progs[p]);
        const uint32_t mask = masks ? masks[p] : 0u;
        prepare_check(sm, mask);
        if (primary) check_misc(sm, mask);
        if (split && threadIdx.x < 32) {
            sm.rows_intra[threadIdx.x] = *(volatile uint32_t *)&dst[p].race_intra[threadIdx.x];
            sm.rows_inter[threadIdx.x] = *(volatile uint32_t *)&dst[p].race_inter[threadIdx.x];
        }
        __syncthreads();
        check_blocks(sm, d.tab, table_bytes, traces + sm.prog.trace_off, segmask + sm.prog.segmask_off,
                     segrange + sm.prog.segmask_off, ci.y, ci.z, primary);
        if (threadIdx.x < 32) {
            const uint32_t ri = sm.rows_intra[threadIdx.x], rx = sm.rows_inter[threadIdx.x];
            if (!split) {
                dst[p].race_intra[threadIdx.x] = ri;
                dst[p].race_inter[threadIdx.x] = rx;
            } else {
                if (ri) atomicOr(&dst[p].race_intra[threadIdx.x], ri);
                if (rx) atomicOr(&dst[p].race_inter[threadIdx.x], rx);
            }
        }
        if (primary && threadIdx.x == 0) {
            dst[p].diverge = sm.diverge;
            dst[p].n_stmts = sm.prog.n_stmts;
            dst[p].access_pairs = sm.pairs;
        }
        __syncthreads();
    }
}

// Clears the witness entries of the programs split over several check items
// (their items OR into them).  Runs before the check kernel on its stream.
__global__ void __launch_bounds__(128) k_split_zero(const uint8_t *__restrict__ arena, uint32_t n,
                                                    uint8_t *__restrict__ scratch, uint64_t scratch_bytes,
                                                    gr_witnesses *__restrict__ out) {
    const ArenaView V = view(arena);
    if (!launch_matches(V, n, scratch_bytes)) return;  // the check kernel reports it
    gr_witnesses *dst = out ? out : reinterpret_cast<gr_witnesses *>(scratch + V.h->scratch_rel_off);
    const uint4 *citems = reinterpret_cast<const uint4 *>(arena + V.h->citems_off);
    for (uint32_t i = blockIdx.x; i < V.h->n_citems; i += gridDim.x) {
        const uint4 ci = citems[i];
        if ((ci.w & (kItemPrimary | kItemSplit)) != (kItemPrimary | kItemSplit)) continue;
        uint32_t *w = reinterpret_cast<uint32_t *>(&dst[ci.x]);
        for (uint32_t j = threadIdx.x; j < sizeof(gr_witnesses) / 4; j += blockDim.x) w[j] = 0u;
    }
}

// ---- plain path: one launch per stage ------------------------------------

__device__ void state_to_smem(Smem &sm, const LoopState *st) {
    if (threadIdx.x == 0) {
        sm.mask = st->mask;
        sm.probe = st->probe;
        sm.done = st->done;
        sm.status = st->status;
        sm.iters = st->iters;
        sm.forced = st->forced;
        sm.forbidden = st->forbidden;
        sm.max_iters = st->max_iters;
        sm.deadline_ns = st->deadline_ns;
        sm.access_pairs = st->access_pairs;
        sm.t_start = st->t_start;
        sm.greedy = st->greedy;
    }
    if (threadIdx.x < 32) {
        sm.acc_intra[threadIdx.x] = st->acc_intra[threadIdx.x];
        sm.acc_inter[threadIdx.x] = st->acc_inter[threadIdx.x];
    }
    for (uint32_t i = threadIdx.x; i < GR_MAX_ITERS; i += blockDim.x) sm.traj[i] = st->traj[i];
    __syncthreads();
}

__device__ void state_from_smem(const Smem &sm, LoopState *st) {
    __syncthreads();
    if (threadIdx.x == 0) {
        st->mask = sm.mask;
        st->probe = sm.probe;
        st->done = sm.done;
        st->status = sm.status;
        st->iters = sm.iters;
        st->forced = sm.forced;
        st->forbidden = sm.forbidden;
        st->max_iters = sm.max_iters;
        st->deadline_ns = sm.deadline_ns;
        st->access_pairs = sm.access_pairs;
        st->t_start = sm.t_start;
        st->greedy = sm.greedy;
    }
    if (threadIdx.x < 32) {
        st->acc_intra[threadIdx.x] = sm.acc_intra[threadIdx.x];
        st->acc_inter[threadIdx.x] = sm.acc_inter[threadIdx.x];
    }
    for (uint32_t i = threadIdx.x; i < GR_MAX_ITERS; i += blockDim.x) st->traj[i] = sm.traj[i];
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 1)
    k_plain_init(const uint8_t *__restrict__ arena, uint32_t p, gr_options opts, LoopState *st) {
    Dyn d = dyn_smem();
    Smem &sm = *d.sm;
    const ArenaView V = view(arena);
    load_program(sm, &V.progs[p]);
    loop_init(sm, opts);
    state_from_smem(sm, st);
}

// CTA b < B: same-block passes of block b; CTA B: cross-block pass, divergence
// and the pair count.  Witness bits are OR-ed into wit (zeroed by the host).
__global__ void __launch_bounds__(kThreads, 1)
    k_plain_check(const uint8_t *__restrict__ arena, uint32_t p, const uint8_t *__restrict__ scratch,
                  const LoopState *__restrict__ st, gr_witnesses *wit, uint32_t table_bytes) {
    Dyn d = dyn_smem();
    Smem &sm = *d.sm;
    const ArenaView V = view(arena);
    const uint16_t *traces = reinterpret_cast<const uint16_t *>(scratch + V.h->scratch_trace_off);
    const uint64_t *segmask = reinterpret_cast<const uint64_t *>(scratch + V.h->scratch_segmask_off);
    const uint32_t *segrange = reinterpret_cast<const uint32_t *>(scratch + V.h->scratch_segrange_off);
    if (threadIdx.x == 0) sm.err = const_cast<uint32_t *>(reinterpret_cast<const uint32_t *>(scratch)) + 1;
    load_program(sm, &V.progs[p]);
    const uint32_t mask = st->mask;
    prepare_check(sm, mask);
    const uint32_t B = sm.prog.blocks;
    const uint32_t b = blockIdx.x;
    if (b < B) {
        check_blocks(sm, d.tab, table_bytes, traces + sm.prog.trace_off, segmask + sm.prog.segmask_off,
                     segrange + sm.prog.segmask_off, b, b + 1, false);
    } else {
        check_misc(sm, mask);
        check_blocks(sm, d.tab, table_bytes, traces + sm.prog.trace_off, segmask + sm.prog.segmask_off,
                     segrange + sm.prog.segmask_off, 0, 0, true);
        if (threadIdx.x == 0) {
            wit->diverge = sm.diverge;
            wit->access_pairs = sm.pairs;
            wit->n_stmts = sm.prog.n_stmts;
        }
    }
    if (threadIdx.x < 32) {
        if (sm.rows_intra[threadIdx.x]) atomicOr(&wit->race_intra[threadIdx.x], sm.rows_intra[threadIdx.x]);
        if (sm.rows_inter[threadIdx.x]) atomicOr(&wit->race_inter[threadIdx.x], sm.rows_inter[threadIdx.x]);
    }
}

__global__ void __launch_bounds__(kThreads, 1)
    k_plain_solve(const uint8_t *__restrict__ arena, uint32_t p, LoopState *st, const gr_witnesses *__restrict__ wit,
                  gr_repair_result *out) {
    Dyn d = dyn_smem();
    Smem &sm = *d.sm;
    const ArenaView V = view(arena);
    load_program(sm, &V.progs[p]);
    state_to_smem(sm, st);
    if (!sm.done) {
        if (threadIdx.x < 32) {
            sm.rows_intra[threadIdx.x] = wit->race_intra[threadIdx.x];
            sm.rows_inter[threadIdx.x] = wit->race_inter[threadIdx.x];
        }
        if (threadIdx.x == 0) {
            sm.diverge = wit->diverge;
            sm.pairs = wit->access_pairs;
        }
        __syncthreads();
        loop_step(sm, *d.mh);
    }
    state_from_smem(sm, st);
    if (sm.done) write_result(sm, out);
}

// ---- wide lane: one CTA per (program, block), the loop on the device -------

struct WideView {
    LoopState *st;
    gr_witnesses *wit;
    WideCtl *ctl;
};

__device__ __forceinline__ WideView wide_view(uint8_t *scratch, uint64_t wide_off, uint32_t n) {
    WideView v;
    v.st = reinterpret_cast<LoopState *>(scratch + wide_off);
    const size_t st_bytes = ((size_t)n * sizeof(LoopState) + 255) & ~(size_t)255;
    v.wit = reinterpret_cast<gr_witnesses *>(scratch + wide_off + st_bytes);
    const size_t wit_bytes = ((size_t)n * sizeof(gr_witnesses) + 255) & ~(size_t)255;
    v.ctl = reinterpret_cast<WideCtl *>(scratch + wide_off + st_bytes + wit_bytes);
    return v;
}

__device__ void zero_witness(gr_witnesses *w) {
    uint32_t *u = reinterpret_cast<uint32_t *>(w);
    for (uint32_t i = threadIdx.x; i < sizeof(gr_witnesses) / 4; i += blockDim.x) u[i] = 0;
}

// CTA p: the initial proposal of program p (Algorithm 1's first Solve, or the
// removal-mode probe); a program already decided writes its result.
__global__ void __launch_bounds__(kWideThreads, 2)
    k_wide_init(const uint8_t *__restrict__ arena, uint32_t n, gr_options opts, uint8_t *scratch, uint64_t wide_off,
                gr_repair_result *out) {
    Dyn d = dyn_smem();
    Smem &sm = *d.sm;
    const ArenaView V = view(arena);
    const WideView W = wide_view(scratch, wide_off, n);
    const uint32_t p = blockIdx.x;
    if (p == 0 && threadIdx.x == 0) *W.ctl = WideCtl{0u, 0u, 0u, 0u};
    load_program(sm, &V.progs[p]);
    loop_init(sm, opts);
    state_from_smem(sm, &W.st[p]);
    zero_witness(&W.wit[p]);
    if (sm.done) write_result(sm, &out[p]);
}

// CTA (b, p): b < B_p the same-block passes of block b of program p; b == B_p
// the cross-block pass, divergence and pair count.  Programs already done and
// CTAs beyond their program's blocks return at once.
__global__ void __launch_bounds__(kWideThreads, 2)
    k_wide_check(const uint8_t *__restrict__ arena, uint32_t n, uint8_t *scratch, uint64_t wide_off,
                 uint32_t table_bytes) {
    const ArenaView V = view(arena);
    const WideView W = wide_view(scratch, wide_off, n);
    const uint32_t p = blockIdx.y, b = blockIdx.x;
    if (W.st[p].done || b > V.progs[p].blocks) return;  // uniform over the CTA
    Dyn d = dyn_smem();
    Smem &sm = *d.sm;
    const uint16_t *traces = reinterpret_cast<const uint16_t *>(scratch + V.h->scratch_trace_off);
    const uint64_t *segmask = reinterpret_cast<const uint64_t *>(scratch + V.h->scratch_segmask_off);
    const uint32_t *segrange = reinterpret_cast<const uint32_t *>(scratch + V.h->scratch_segrange_off);
    if (threadIdx.x == 0) sm.err = reinterpret_cast<uint32_t *>(scratch) + 1;
    load_program(sm, &V.progs[p]);
    const uint32_t mask = W.st[p].mask;
    prepare_check(sm, mask);
    const uint32_t B = sm.prog.blocks;
    gr_witnesses *wit = &W.wit[p];
    if (b < B) {
        check_blocks(sm, d.tab, table_bytes, traces + sm.prog.trace_off, segmask + sm.prog.segmask_off,
                     segrange + sm.prog.segmask_off, b, b + 1, false);
    } else {
        check_misc(sm, mask);
        check_blocks(sm, d.tab, table_bytes, traces + sm.prog.trace_off, segmask + sm.prog.segmask_off,
                     segrange + sm.prog.segmask_off, 0, 0, true);
        if (threadIdx.x == 0) {
            wit->diverge = sm.diverge;
            wit->access_pairs = sm.pairs;
            wit->n_stmts = sm.prog.n_stmts;
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        if (sm.rows_intra[threadIdx.x]) atomicOr(&wit->race_intra[threadIdx.x], sm.rows_intra[threadIdx.x]);
        if (sm.rows_inter[threadIdx.x]) atomicOr(&wit->race_inter[threadIdx.x], sm.rows_inter[threadIdx.x]);
    }
}

// CTA p: clauses from the check's witnesses, the next proposal (one loop step
// of Algorithm 1), the result once decided, the witness buffer cleared for the
// next round.  The last CTA of the round to finish sets the while-node's
// condition: another round while some program runs and the bound is not hit.
__global__ void __launch_bounds__(kWideThreads, 2)
    k_wide_solve(const uint8_t *__restrict__ arena, uint32_t n, uint8_t *scratch, uint64_t wide_off,
                 gr_repair_result *out, cudaGraphConditionalHandle cond) {
    Dyn d = dyn_smem();
    Smem &sm = *d.sm;
    const ArenaView V = view(arena);
    const WideView W = wide_view(scratch, wide_off, n);
    const uint32_t p = blockIdx.x;
    __shared__ uint32_t was_done;
    if (threadIdx.x == 0) was_done = W.st[p].done;
    __syncthreads();
    if (!was_done) {
        load_program(sm, &V.progs[p]);
        state_to_smem(sm, &W.st[p]);
        const gr_witnesses *wit = &W.wit[p];
        if (threadIdx.x < 32) {
            sm.rows_intra[threadIdx.x] = wit->race_intra[threadIdx.x];
            sm.rows_inter[threadIdx.x] = wit->race_inter[threadIdx.x];
        }
        if (threadIdx.x == 0) {
            sm.diverge = wit->diverge;
            sm.pairs = wit->access_pairs;
        }
        __syncthreads();
        loop_step(sm, *d.mh);
        state_from_smem(sm, &W.st[p]);
        if (sm.done) write_result(sm, &out[p]);
        zero_witness(&W.wit[p]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t running = was_done ? 0u : (sm.done ? 0u : 1u);
        if (running) atomicAdd(&W.ctl->active, 1u);
        __threadfence();
        if (atomicAdd(&W.ctl->arrived, 1u) == n - 1u) {  // the last CTA of this round
            __threadfence();
            const uint32_t active = atomicAdd(&W.ctl->active, 0u);
            const uint32_t rounds = W.ctl->rounds + 1u;
            W.ctl->rounds = rounds;
            W.ctl->arrived = 0u;
            W.ctl->active = 0u;
            const bool bound = rounds >= kWideRounds;
            if (active && bound) atomicOr(reinterpret_cast<uint32_t *>(scratch) + 1, kErrWideRounds);
            cudaGraphSetConditional(cond, (active && !bound) ? 1u : 0u);
        }
    }
}

// gr_solve: in = [n_vars, n_pos, n_neg, forced, forbidden, w[24], pos..., neg...];
// out = [found, mask, weight].
__global__ void __launch_bounds__(kThreads, 1) k_solve(const uint32_t *__restrict__ in, uint32_t *__restrict__ out) {
    Dyn d = dyn_smem();
    Smem &sm = *d.sm;
    MhsSmem &mh = *d.mh;
    const uint32_t n_vars = in[0], n_pos = in[1], n_neg = in[2], forced = in[3], forbidden = in[4];
    const uint32_t *w = in + 5;
    for (uint32_t i = threadIdx.x; i < n_pos; i += blockDim.x) mh_cl(sm)[i] = in[5 + GR_MAX_SLOTS + i];
    // negative clauses live after the positive ones in the mhs scratch
    uint32_t *neg = mh.nlo;  // staging; mhs_solve reads neg[] before it writes nlo
    for (uint32_t i = threadIdx.x; i < n_neg; i += blockDim.x) neg[i] = in[5 + GR_MAX_SLOTS + n_pos + i];
    __shared__ uint32_t wsh[GR_MAX_SLOTS];
    if (threadIdx.x < GR_MAX_SLOTS) wsh[threadIdx.x] = threadIdx.x < n_vars ? w[threadIdx.x] : 0u;
    __syncthreads();
    mhs_solve(sm, mh, n_vars, wsh, n_pos, neg, n_neg, forced, forbidden);
    if (threadIdx.x == 0) {
        out[0] = sm.sol_found;
        out[1] = sm.sol_found ? sm.sol_mask : 0u;
        out[2] = sm.sol_found ? sm.sol_weight : 0u;
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------

size_t dyn_bytes(uint32_t table_bytes) {
    const size_t region = table_bytes > sizeof(MhsSmem) ? table_bytes : sizeof(MhsSmem);
    return kFixedSmem + align_up(region, 16);
}

// The CTA shapes of the persistent kernels: {threads, CTAs per SM}.
const LaunchShape kShapes[kNumShapes] = {{512, 2}, {256, 3}, {256, 4}, {1024, 1}, {384, 3}};

template <typename F>
static cudaError_t set_smem(F *f, uint32_t max_dynamic_smem) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, (const void *)f);
    if (e != cudaSuccess) return e;
    const size_t cap = max_dynamic_smem > a.sharedSizeBytes ? max_dynamic_smem - a.sharedSizeBytes : 0;
    return cudaFuncSetAttribute((const void *)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
}

cudaError_t configure_kernels(uint32_t max_dynamic_smem) {
    cudaError_t e;
    const void *fns[] = {(const void *)k_plain_init, (const void *)k_plain_check, (const void *)k_plain_solve,
                         (const void *)k_solve, (const void *)k_wide_init, (const void *)k_wide_check,
                         (const void *)k_wide_solve};
    for (const void *f : fns) {
        cudaFuncAttributes a;
        e = cudaFuncGetAttributes(&a, f);
        if (e != cudaSuccess) return e;
        const size_t cap = max_dynamic_smem > a.sharedSizeBytes ? max_dynamic_smem - a.sharedSizeBytes : 0;
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
        if (e != cudaSuccess) return e;
    }
    if ((e = set_smem(k_check<512, 2>, max_dynamic_smem)) != cudaSuccess) return e;
    if ((e = set_smem(k_check<256, 3>, max_dynamic_smem)) != cudaSuccess) return e;
    if ((e = set_smem(k_check<256, 4>, max_dynamic_smem)) != cudaSuccess) return e;
    if ((e = set_smem(k_check<1024, 1>, max_dynamic_smem)) != cudaSuccess) return e;
    if ((e = set_smem(k_check<384, 3>, max_dynamic_smem)) != cudaSuccess) return e;
    if ((e = configure_relation(max_dynamic_smem)) != cudaSuccess) return e;
    if ((e = configure_loop(max_dynamic_smem)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t launch_perm_check(const void *d_arena, uint32_t n, uint32_t base, uint32_t *d_bad, uint32_t sms,
                              cudaStream_t st) {
    const uint32_t grid = n < 4u * sms ? (n ? n : 1u) : 4u * sms;
    k_perm_check<<<grid, 256, 0, st>>>(static_cast<const uint8_t *>(d_arena), base, d_bad);
    return cudaGetLastError();
}

cudaError_t launch_expand(const void *d_arena, void *d_scratch, uint64_t scratch_bytes, bool general_only,
                          uint32_t grid, cudaStream_t st) {
    k_expand<<<grid, 256, 0, st>>>(static_cast<const uint8_t *>(d_arena), static_cast<uint8_t *>(d_scratch),
                                   scratch_bytes, general_only ? 1u : 0u);
    return cudaGetLastError();
}

cudaError_t launch_split_zero(const void *d_arena, uint32_t n, void *d_scratch, uint64_t scratch_bytes,
                              gr_witnesses *d_out, cudaStream_t st) {
    k_split_zero<<<64, 128, 0, st>>>(static_cast<const uint8_t *>(d_arena), n, static_cast<uint8_t *>(d_scratch),
                                     scratch_bytes, d_out);
    return cudaGetLastError();
}

cudaError_t launch_check(const void *d_arena, uint32_t n, const uint32_t *d_masks, void *d_scratch,
                         uint64_t scratch_bytes, gr_witnesses *d_out, LaunchCfg cfg, cudaStream_t st) {
    const uint8_t *a = static_cast<const uint8_t *>(d_arena);
    uint8_t *sc = static_cast<uint8_t *>(d_scratch);
    const size_t smem = dyn_bytes(cfg.table_bytes);
    switch (cfg.shape & kShapeMask) {
        case 1: k_check<256, 3><<<cfg.grid, 256, smem, st>>>(a, n, d_masks, sc, scratch_bytes, d_out, cfg.table_bytes); break;
        case 2: k_check<256, 4><<<cfg.grid, 256, smem, st>>>(a, n, d_masks, sc, scratch_bytes, d_out, cfg.table_bytes); break;
        case 3: k_check<1024, 1><<<cfg.grid, 1024, smem, st>>>(a, n, d_masks, sc, scratch_bytes, d_out, cfg.table_bytes); break;
        case 4: k_check<384, 3><<<cfg.grid, 384, smem, st>>>(a, n, d_masks, sc, scratch_bytes, d_out, cfg.table_bytes); break;
        default: k_check<512, 2><<<cfg.grid, 512, smem, st>>>(a, n, d_masks, sc, scratch_bytes, d_out, cfg.table_bytes); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_plain_init(const void *d_arena, uint32_t p, const gr_options &opts, LoopState *d_state,
                              cudaStream_t st) {
    k_plain_init<<<1, kThreads, dyn_bytes(kMinTableBytes), st>>>(static_cast<const uint8_t *>(d_arena), p, opts,
                                                                  d_state);
    return cudaGetLastError();
}

cudaError_t launch_plain_check(const void *d_arena, uint32_t p, void *d_scratch, LoopState *d_state,
                               gr_witnesses *d_wit, uint32_t n_blocks, uint32_t table_bytes, cudaStream_t st) {
    k_plain_check<<<n_blocks + 1, kThreads, dyn_bytes(table_bytes), st>>>(
        static_cast<const uint8_t *>(d_arena), p, static_cast<const uint8_t *>(d_scratch), d_state, d_wit,
        table_bytes);
    return cudaGetLastError();
}

cudaError_t launch_plain_solve(const void *d_arena, uint32_t p, LoopState *d_state, const gr_witnesses *d_wit,
                               gr_repair_result *out, cudaStream_t st) {
    k_plain_solve<<<1, kThreads, dyn_bytes(kMinTableBytes), st>>>(static_cast<const uint8_t *>(d_arena), p,
                                                                   d_state, d_wit, out);
    return cudaGetLastError();
}

// Work-queue counters (scratch control words 0, 2, 3) and, when clear_error,
// the device error word (word 1).
static cudaError_t clear_ctrl(void *d_scratch, bool clear_error, cudaStream_t st) {
    if (clear_error) return cudaMemsetAsync(d_scratch, 0, 256, st);
    cudaError_t e = cudaMemsetAsync(d_scratch, 0, 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(static_cast<uint32_t *>(d_scratch) + 2, 0, 8, st);
    return e;
}

cudaError_t enqueue_relation(const void *d_arena, uint32_t n, void *d_scratch, uint64_t scratch_bytes,
                             const LaunchCfg &cfg, uint32_t expand_grid, bool expand, bool clear_error, cudaStream_t st) {
    const bool general = !(cfg.skip & kSkipGeneral), fast = !(cfg.skip & kSkipFast);
    cudaError_t e = clear_ctrl(d_scratch, clear_error, st);
    if (e == cudaSuccess && general && expand)
        e = launch_expand(d_arena, d_scratch, scratch_bytes, true, expand_grid, st);
    if (e == cudaSuccess && general && !(cfg.skip & kSkipSplit))
        e = launch_split_zero(d_arena, n, d_scratch, scratch_bytes, nullptr, st);
    if (e == cudaSuccess && fast)
        e = launch_relation(d_arena, n, nullptr, d_scratch, scratch_bytes, nullptr, cfg.rel, st);
    if (e == cudaSuccess && general)
        e = launch_check(d_arena, n, nullptr, d_scratch, scratch_bytes, nullptr, cfg, st);
    return e;
}

cudaError_t enqueue_loop(const void *d_arena, uint32_t n, const gr_options &opts, void *d_scratch,
                         uint64_t scratch_bytes, gr_repair_result *d_out, const LaunchCfg &cfg, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(static_cast<uint32_t *>(d_scratch) + 3, 0, 4, st);  // its queue counter
    if (e == cudaSuccess) e = launch_loop(d_arena, n, opts, d_scratch, scratch_bytes, d_out, cfg.loop_grid, cfg.simple != 0, st);
    return e;
}

cudaError_t enqueue_repair(const void *d_arena, uint32_t n, const gr_options &opts, void *d_scratch,
                           uint64_t scratch_bytes, gr_repair_result *d_out, const LaunchCfg &cfg, uint32_t expand_grid,
                           bool expand, bool clear_error, cudaStream_t st) {
    if (cfg.flags_off && cfg.flags_off + (uint64_t)n * 4u <= scratch_bytes) {
        // one launch: the relations, then each CTA runs the loop of programs
        // whose relation is out (their done flags start cleared)
        cudaError_t e = clear_ctrl(d_scratch, clear_error, st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(static_cast<uint8_t *>(d_scratch) + cfg.flags_off, 0, (size_t)n * 4u, st);
        if (e == cudaSuccess) e = launch_relation_loop(d_arena, n, d_scratch, scratch_bytes, opts, d_out, cfg.fused, st);
        return e;
    }
    cudaError_t e = enqueue_relation(d_arena, n, d_scratch, scratch_bytes, cfg, expand_grid, expand, clear_error, st);
    if (e == cudaSuccess) e = launch_loop(d_arena, n, opts, d_scratch, scratch_bytes, d_out, cfg.loop_grid, cfg.simple != 0, st);
    return e;
}

cudaError_t enqueue_check(const void *d_arena, uint32_t n, const uint32_t *d_masks, void *d_scratch,
                          uint64_t scratch_bytes, gr_witnesses *d_out, const LaunchCfg &cfg, uint32_t expand_grid,
                          bool expand, cudaStream_t st) {
    const bool general = !(cfg.skip & kSkipGeneral), fast = !(cfg.skip & kSkipFast);
    cudaError_t e = clear_ctrl(d_scratch, true, st);
    if (e == cudaSuccess && general && expand)
        e = launch_expand(d_arena, d_scratch, scratch_bytes, true, expand_grid, st);
    if (e == cudaSuccess && general && !(cfg.skip & kSkipSplit))
        e = launch_split_zero(d_arena, n, d_scratch, scratch_bytes, d_out, st);
    if (e == cudaSuccess && fast)
        e = launch_relation(d_arena, n, d_masks, d_scratch, scratch_bytes, d_out, cfg.rel, st);
    if (e == cudaSuccess && general) e = launch_check(d_arena, n, d_masks, d_scratch, scratch_bytes, d_out, cfg, st);
    return e;
}

size_t wide_bytes(uint32_t n) {
    const size_t a = ((size_t)n * sizeof(LoopState) + 255) & ~(size_t)255;
    const size_t b = ((size_t)n * sizeof(gr_witnesses) + 255) & ~(size_t)255;
    return a + b + 256;
}

cudaError_t launch_wide(const void *d_arena, uint32_t n, uint32_t max_blocks, const gr_options &opts,
                        void *d_scratch, uint64_t wide_off, gr_repair_result *d_out, uint32_t table_bytes,
                        cudaStream_t st) {
    const uint8_t *a = static_cast<const uint8_t *>(d_arena);
    uint8_t *sc = static_cast<uint8_t *>(d_scratch);
    const size_t small = dyn_bytes(kMinTableBytes);
    k_wide_init<<<n, kWideThreads, small, st>>>(a, n, opts, sc, wide_off, d_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the loop: a graph whose while-node runs [check, solve] until the solve
    // kernel clears the condition
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    cudaStream_t cap = nullptr;
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return e;
    cudaGraphConditionalHandle cond;
    e = cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            k_wide_check<<<dim3(max_blocks + 1, n), kWideThreads, dyn_bytes(table_bytes), cap>>>(a, n, sc, wide_off,
                                                                                               table_bytes);
            cudaError_t e1 = cudaGetLastError();
            k_wide_solve<<<n, kWideThreads, small, cap>>>(a, n, sc, wide_off, d_out, cond);
            cudaError_t e2 = cudaGetLastError();
            e = cudaStreamEndCapture(cap, &body);
            if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(x, st);
    // released once the launch completes
    if (x) cudaGraphExecDestroy(x);
    if (cap) cudaStreamDestroy(cap);
    cudaGraphDestroy(g);
    return e;
}

cudaError_t launch_solve(const uint32_t *d_in, uint32_t *d_out, cudaStream_t st) {
    k_solve<<<1, kThreads, dyn_bytes(kMinTableBytes), st>>>(d_in, d_out);
    return cudaGetLastError();
}

}  // namespace gr
