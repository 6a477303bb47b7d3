// engine.cuh — packed device layout shared by the host packer (capi.cu) and
// the kernels (kernels.cu).  Internal to libgpurepair; not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "gpurepair.h"

namespace gr {

constexpr uint32_t kArenaMagic = 0x47525031u;  // "GRP1"
constexpr uint32_t kThreads = 512;             // threads per CTA of the repair kernels
constexpr uint32_t kWideThreads = 512;         // threads per CTA of the wide lane (two CTAs per SM)
constexpr uint32_t kChunkShift = 10;           // address chunk = 1,024 words
constexpr uint32_t kChunkWords = 1u << kChunkShift;
constexpr uint32_t kMaxTileChunks = 8;           // address chunks per owner-table tile
constexpr uint32_t kSegCap = 512;                // (statement, block) segments listed per batch
constexpr uint32_t kItemSegs = 64;               // segments per trace-expansion work item
constexpr uint16_t kEmpty = 0xFFFFu;           // owner-table sentinels
constexpr uint16_t kMulti = 0xFFFEu;
constexpr uint32_t kClauseCap = 1024;          // clause buffer (>= 2 * 25 * 26 / 2)
constexpr uint32_t kClauseSetLog2 = 11;
constexpr uint32_t kClauseSet = 1u << kClauseSetLog2;  // clause hash set (>= 2 x 650 entries)
constexpr uint32_t kNoClause = 0xFFFFFFFFu;            // its empty marker
constexpr uint32_t kMinTableBytes = 25u * 2u * kChunkWords;  // one chunk for 25 rows
constexpr uint32_t kErrTableTooSmall = 1u;  // bits of the device error word (scratch control word 1)
constexpr uint32_t kErrArgs = 4u;           // the launch's n or scratch size does not match the arena
constexpr uint32_t kErrStall = 8u;          // a bounded wait for another CTA's result ran out
constexpr uint8_t kStmtInjective = 1u;      // DevStmt::flags: no two threads of a block share an address
constexpr uint32_t kArenaSimple = 1u;       // ArenaHeader::flags: every program is straight-line (no loops or
                                            // explicit slot places) on the shared array alone
constexpr uint32_t kMaxCheckSplit = 16u;    // most check items of one program (its blocks in ranges)
constexpr uint32_t kItemPrimary = 1u;       // check item flags: the item with block 0, the divergence, the
constexpr uint32_t kItemSplit = 2u;         //   pair count and the cross-block pass; one of several items

// One statement, with map coefficients reduced modulo its array's size.
struct DevStmt {
    uint8_t op, space, kind, flags;  // flags: kStmtInjective
    uint32_t am, bm, cm;   // a, b, c mod M
    uint32_t perm_off;     // GR_PERM: absolute index of its window (its table from b on; bm is then 0)
    uint16_t gk, gr;       // guard: active iff gk == 0 || tid % gk == gr
    uint32_t m;            // words of its array
    uint32_t pneed;        // GR_PERM: leading entries of its window that must be distinct (see the packer)
};
static_assert(sizeof(DevStmt) == 32, "DevStmt layout");

// One program: header + executed statement instances + slots.  n_stmts counts
// the instances (a loop body once per iteration); n_slots the program's slots.
// Instances k and k+1 are separated by the barriers of the slots gapslots[k] (slot k without
// loops and explicit places).  16-byte aligned, fixed size.
struct DevProg {
    uint32_t n_stmts, n_slots, blocks, threads;
    uint32_t t_pad;        // threads rounded up to a multiple of 8
    uint32_t m_shared, m_global;
    int32_t mode;          // GR_MODE_*
    uint32_t existing, grid_mask, write_mask, shared_rows;
    uint32_t global_rows, guarded_slots;
    uint32_t blk_invariant;  // 1: every block has the same same-block witnesses (see the packer)
    uint32_t general;      // 1: counted loops or explicit slot places (gaps differ from slots)
    uint64_t trace_off;    // u16 elements from the scratch trace base; layout [S][B][t_pad], unit order
    uint64_t segmask_off;  // element index of the program's [S][B] segment masks and ranges
    uint32_t weights[GR_MAX_SLOTS];
    uint16_t slot_gk[GR_MAX_SLOTS];
    uint16_t slot_gr[GR_MAX_SLOTS];
    uint8_t rep[32];       // lowest instance with the same array, map and guard
    uint32_t gapslots[32]; // slots whose barriers run between instances k and k+1
    uint32_t n_neg;
    uint32_t fast;         // 1: checked by the relation kernel (shared array only, blocks alike)
    uint32_t _r3[2];
    uint32_t neg[GR_MAX_NEG];  // negative clauses given with the program
    DevStmt stmts[GR_MAX_STMTS];  // one per executed statement instance
};
static_assert(sizeof(DevProg) % 16 == 0, "DevProg alignment");

// Arena = ArenaHeader | DevProg[n] | order[n] | seg_base[n+1] | items[] | perm[]
//   order: the n_fast programs the relation kernel checks, then the others,
//   each part largest first; items: the expansion work items of the other
//   programs (n_items_gen of them), then those of the n_fast programs.
// Scratch = ctrl (256 B) | segmask u64[] | segrange u32[] | trace u16[] | wide | rel gr_witnesses[n]
struct ArenaHeader {
    uint32_t magic, n_progs, s_max, b_max;  // most statement instances / blocks of any program
    uint64_t progs_off, order_off, segbase_off, perm_off;  // bytes from the arena start
    uint64_t n_segments;                                   // sum over programs of S*B
    uint64_t scratch_segmask_off, scratch_trace_off;       // bytes from the scratch start
    uint64_t scratch_bytes;
    uint64_t scratch_segrange_off;
    uint64_t scratch_wide_off;  // wide lane: LoopState[n] | gr_witnesses[n] | WideCtl
    uint64_t items_off;       // expansion work items (uint4: program, first, end segment)
    uint32_t n_items;
    uint32_t flags;           // kArena* bits
    uint64_t scratch_rel_off;     // each program's conflict relation (gr_witnesses rows)
    uint32_t n_fast;              // programs checked by the relation kernel (first in order)
    uint32_t n_items_gen;         // expansion items of the other programs (first in items)
    // the general check kernel's work items (uint4: program, first block,
    // end block, kItem* flags), largest first: one per program, or, for a
    // program whose blocks differ, one per range of its blocks
    uint64_t citems_off;
    uint32_t n_citems;
    uint32_t n_split;             // programs with more than one check item
    uint32_t _r[12];
};
static_assert(sizeof(ArenaHeader) == 192, "ArenaHeader layout");

// Loop state of one program between iterations (plain path keeps it in
// device memory between launches).
struct LoopState {
    uint32_t mask, probe, done, status, iters, forced, forbidden, max_iters;
    uint32_t greedy, _pad0;
    uint64_t access_pairs, t_start;
    uint64_t deadline_ns;  // 0: none
    uint32_t traj[GR_MAX_ITERS];
    uint32_t acc_intra[32], acc_inter[32];
};

// Round bookkeeping of the wide lane's device-side loop (a graph while-node).
struct WideCtl {
    uint32_t arrived;  // solve CTAs finished in this round
    uint32_t active;   // of them, programs still running
    uint32_t rounds;   // rounds so far (bounded)
    uint32_t _pad;
};

// Launch of the relation kernel (relation.cu).
struct RelCfg {
    uint32_t grid;         // CTAs (persistent)
    uint32_t table_bytes;  // owner-table budget per CTA
    uint32_t shape;        // index into kRelShapes
};

// Launch of a repair: the general check kernel (k_check, one CTA per program
// of the batch's general part), the relation kernel and the loop kernel.
struct LaunchCfg {
    uint32_t grid;         // CTAs of k_check
    uint32_t table_bytes;  // its owner-table budget per CTA
    uint32_t shape;        // index into kShapes
    RelCfg rel;
    uint32_t loop_grid;    // CTAs of the loop kernel
    uint32_t skip;         // kSkip* bits: parts of the batch known to be empty
    uint32_t simple;       // 1: the loop kernel's small build (a batch the packer marked kArenaSimple)
    RelCfg fused;          // the relation kernel that also runs the loop (table_bytes 0: not used)
    uint64_t flags_off;    // scratch bytes to its per-program done flags (see rel_flags_off)
};

// Scratch offset of the per-program done flags (u32[n]) after the relations.
__host__ __device__ inline uint64_t rel_flags_off(uint64_t scratch_rel_off, uint32_t n) {
    return (scratch_rel_off + (uint64_t)n * sizeof(gr_witnesses) + 255u) & ~(uint64_t)255u;
}
constexpr uint32_t kSkipGeneral = 1u;  // no general program: no expansion, no k_check
constexpr uint32_t kSkipFast = 2u;     // no program for the relation kernel
constexpr uint32_t kSkipSplit = 4u;    // no program with several check items (nothing to zero first)

// The kSkip* bits of a packed batch.
inline uint32_t skip_bits(const ArenaHeader &h) {
    return (h.n_fast == 0 ? kSkipFast : 0u) | (h.n_fast == h.n_progs ? kSkipGeneral : 0u) |
           (h.n_split == 0 ? kSkipSplit : 0u);
}

// CTA shapes the persistent kernels are instantiated for.
struct LaunchShape {
    uint32_t threads, ctas_per_sm;
};
constexpr uint32_t kNumShapes = 5;
constexpr uint32_t kShapeMask = 15u;      // LaunchCfg::shape: index into kShapes ...
constexpr uint32_t kShapeBalanced = 16u;  // ... plus: grid cut so every CTA gets the same number of programs
extern const LaunchShape kShapes[kNumShapes];
size_t dyn_bytes(uint32_t table_bytes);
size_t mhs_smem_bytes();
constexpr uint32_t kNumRelShapes = 6;
extern const LaunchShape kRelShapes[kNumRelShapes];
size_t rel_fixed_bytes();   // the relation kernel's shared memory besides its table
size_t loop_smem_bytes(bool simple);  // the loop kernel's shared memory per CTA
uint32_t loop_threads(bool simple);    // its threads per CTA (a warp per program)
constexpr uint32_t kLoopThreads = 128;  // the general build's CTA: four warps

// Host-side helpers (capi.cu).
struct Layout {
    size_t progs_off, order_off, segbase_off, items_off, citems_off, perm_off, arena_bytes;
    uint64_t n_items, n_citems;
    size_t segmask_off, segrange_off, trace_off, wide_off, rel_off, scratch_bytes;
    uint64_t n_segments, perm_elems;
    std::vector<uint64_t> trace_elem, segmask_elem, perm_base;
};
gr_status fail(gr_status code, const char *fmt, ...);
// Check items of a program in the general check kernel's queue (see
// ArenaHeader::citems_off): 0 for a program the relation kernel checks.
uint32_t check_items_of(const gr_program &p, const gr_launch &l);
// u16 entries of the permutation windows the packer reserves for a program:
// one per permutation instance, the instance's table from its offset b on
// (the block's threads' entries, padded, or the whole table).
uint64_t perm_window_elems(const gr_program &p, const gr_launch &l);
gr_status validate_one(const gr_program *p, gr_launch l, uint32_t idx, bool tables = true);
// Statement instances in execution order (st: statement, ctr: counter of its
// innermost loop); returns how many run, storing at most cap (counting stops
// past cap).
uint32_t exec_order(const gr_program &p, uint8_t *st, uint8_t *ctr, uint32_t cap);
inline uint32_t slots_of(const gr_program &p) { return p.n_slots ? p.n_slots : p.n_stmts - 1; }
// Every block of the launch has the same same-block witnesses (a validated program).
bool blocks_alike(const gr_program &p);
inline uint32_t exec_count(const gr_program &p) {
    if (p.n_loops == 0) return p.n_stmts;
    uint8_t st[GR_MAX_STMTS], ctr[GR_MAX_STMTS];
    return exec_order(p, st, ctr, GR_MAX_STMTS);
}
size_t align_to(size_t x, size_t a);
Layout layout_of(const gr_program *progs, const gr_launch *ls, uint32_t n);
// table_bad (may be NULL): per program, the lowest statement whose permutation
// table is not one (left as is when every table is).  range_only: only entries
// at or above M count as bad (repeats are left to the device check,
// launch_perm_check).
void pack_into(const gr_program *progs, const gr_launch *ls, const int32_t *modes, uint32_t n, const Layout &L,
               uint8_t *arena, uint32_t *table_bad = nullptr, bool range_only = false);
// The launch of a repair of n packed programs at d_arena on the current
// device: the shapes gr_tune_packed recorded for (d_arena, n), else the
// defaults, plus the kSkip* bits `skip`; `simple`: the arena header's
// kArenaSimple flag (the loop kernel's small build).
LaunchCfg packed_launch_cfg(const void *d_arena, uint32_t n, uint32_t skip, bool simple, uint64_t rel_off,
                            gr_status *status);
// Options: GR_EINVAL for an unknown strategy or values out of range; the
// defaults filled in (NULL: grid enabled, 64 iterations, no deadline).
gr_status validate_opts(const gr_options *o);
gr_options opts_or_default(const gr_options *o);
void set_last_error(const char *msg);

// Host-callable launchers (kernels.cu).
// general_only: only the general programs' traces (the relation kernel
// computes the other programs' addresses itself).
cudaError_t launch_expand(const void *d_arena, void *d_scratch, uint64_t scratch_bytes, bool general_only,
                          uint32_t grid, cudaStream_t st);
// Device check that the batch's permutation tables are permutations (the
// lowest failing program + base, complemented, into *d_bad by atomicMax).
cudaError_t launch_perm_check(const void *d_arena, uint32_t n, uint32_t base, uint32_t *d_bad, uint32_t sms,
                              cudaStream_t st);
// One check per general program (d_masks NULL: the empty mask, rows into the
// scratch's relation area when d_out is NULL).
// Clears the witness entries of programs split over several check items.
cudaError_t launch_split_zero(const void *d_arena, uint32_t n, void *d_scratch, uint64_t scratch_bytes,
                              gr_witnesses *d_out, cudaStream_t st);
cudaError_t launch_check(const void *d_arena, uint32_t n, const uint32_t *d_masks, void *d_scratch,
                         uint64_t scratch_bytes, gr_witnesses *d_out, LaunchCfg cfg, cudaStream_t st);
// The same for the programs the relation kernel takes.
// The relation kernel that, once the relation queue is empty, runs the loop
// of every program (one warp each) in the same launch (batches the packer
// marked simple with no general program; cfg.fused the CTA shape).
cudaError_t launch_relation_loop(const void *d_arena, uint32_t n, void *d_scratch, uint64_t scratch_bytes,
                                 const gr_options &opts, gr_repair_result *d_out, RelCfg cfg, cudaStream_t st);
// Whether the fused kernel's loop records fit a CTA's table of table_bytes.
bool relation_loop_fits(uint32_t table_bytes);
cudaError_t launch_relation(const void *d_arena, uint32_t n, const uint32_t *d_masks, void *d_scratch,
                            uint64_t scratch_bytes, gr_witnesses *d_out, RelCfg cfg, cudaStream_t st);
// Algorithm 1 per program over the relations in the scratch.
cudaError_t launch_loop(const void *d_arena, uint32_t n, const gr_options &opts, void *d_scratch,
                        uint64_t scratch_bytes, gr_repair_result *d_out, uint32_t grid, bool simple, cudaStream_t st);
// The whole repair of a packed batch on the device: the general programs'
// traces (when `expand`), the relations, the loop.  Clears the work-queue
// counters first, and the device error word too when clear_error.
cudaError_t enqueue_repair(const void *d_arena, uint32_t n, const gr_options &opts, void *d_scratch,
                           uint64_t scratch_bytes, gr_repair_result *d_out, const LaunchCfg &cfg, uint32_t expand_grid,
                           bool expand, bool clear_error, cudaStream_t st);
// The two halves of enqueue_repair: the relations (the queue counters, and
// the error word when clear_error, cleared first), then the loop (its queue
// counter cleared first).
cudaError_t enqueue_relation(const void *d_arena, uint32_t n, void *d_scratch, uint64_t scratch_bytes,
                             const LaunchCfg &cfg, uint32_t expand_grid, bool expand, bool clear_error, cudaStream_t st);
cudaError_t enqueue_loop(const void *d_arena, uint32_t n, const gr_options &opts, void *d_scratch,
                         uint64_t scratch_bytes, gr_repair_result *d_out, const LaunchCfg &cfg, cudaStream_t st);
// One check per program of a packed batch under d_masks.
cudaError_t enqueue_check(const void *d_arena, uint32_t n, const uint32_t *d_masks, void *d_scratch,
                          uint64_t scratch_bytes, gr_witnesses *d_out, const LaunchCfg &cfg, uint32_t expand_grid,
                          bool expand, cudaStream_t st);
cudaError_t launch_plain_init(const void *d_arena, uint32_t p, const gr_options &opts,
                              LoopState *d_state, cudaStream_t st);
cudaError_t launch_plain_check(const void *d_arena, uint32_t p, void *d_scratch, LoopState *d_state,
                               gr_witnesses *d_wit, uint32_t n_blocks, uint32_t table_bytes,
                               cudaStream_t st);
cudaError_t launch_plain_solve(const void *d_arena, uint32_t p, LoopState *d_state,
                               const gr_witnesses *d_wit, gr_repair_result *d_out, cudaStream_t st);
cudaError_t launch_solve(const uint32_t *d_in, uint32_t *d_out, cudaStream_t st);
// Wide lane: initial solve of every program, then a graph whose while-node
// repeats [check: one CTA per (program, block) + one per program for the
// cross-block pass; solve: one CTA per program] until every program is done
// (at most kWideRounds rounds).  Builds, launches and releases the graph.
constexpr uint32_t kWideRounds = GR_MAX_ITERS + 4;
constexpr uint32_t kErrWideRounds = 2u;  // device error word bit: the round bound was hit
cudaError_t launch_wide(const void *d_arena, uint32_t n, uint32_t max_blocks, const gr_options &opts,
                        void *d_scratch, uint64_t wide_off, gr_repair_result *d_out, uint32_t table_bytes,
                        cudaStream_t st);
size_t wide_bytes(uint32_t n);
LaunchCfg wide_launch_cfg(uint32_t n, uint32_t s_max, gr_status *status);
size_t fixed_smem_bytes();
cudaError_t configure_kernels(uint32_t max_dynamic_smem);
cudaError_t configure_relation(uint32_t max_dynamic_smem);
cudaError_t configure_loop(uint32_t max_dynamic_smem);

}  // namespace gr
