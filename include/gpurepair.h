/*
 * gpurepair.h — C ABI of the GB300 engine for GPURepair's repair loop
 * (Joshi and Muduganti, "GPURepair: Automated Repair of GPU Kernels",
 * arXiv 2011.08373).
 *
 * The engine restates the paper's instrumented kernel (Section 2.2) over a
 * concrete launch and runs Algorithm 1 (Section 2.4) on the GPU:
 *   check  — every race witness (i, j) and every divergent enabled barrier of
 *            a program under a barrier mask (the paper's Verify);
 *   clause — each race witness becomes "some slot that can order it is on",
 *            each divergent slot a negative unit clause (GenerateClause);
 *   solve  — the exact minimum-weight hitting set of the clauses, ties broken
 *            by the lowest mask (Solve, in its weighted MaxSAT form);
 *   repair — the loop of the three to a fixed point.
 *
 * Model.  A program has S (1..25) straight-line statements.  Statement s is a
 * read (GR_R) or write (GR_W) of one 32-bit word of the SHARED array (one
 * private copy per block, m_shared words) or of the GLOBAL array (one copy
 * for the grid, m_global words) at an address given by a per-thread map:
 *   GR_AFFINE, GR_STRIDED: (a*tid + c*blk + b) mod M
 *   GR_PERM:               perm[perm_off + ((tid + c*blk + b) mod M)]
 * (64-bit intermediates; tid = threadIdx.x, blk = blockIdx.x).  Statement s
 * runs for thread tid iff guard_k == 0 or tid % guard_k == guard_r.
 * A GR_PERM statement's table entries must be distinct indices below M
 * where it reads them: when its address does not depend on the block
 * (c mod M == 0, or one block) the min(T, M) entries from b on, cyclically
 * (entries (b + tid) mod M, tid < T); else the whole table (a permutation
 * of 0..M-1).  Entries it never reads are neither checked nor copied.
 * Slot k (0..S-2) is a candidate barrier between statements k and k+1 with a
 * level (GR_BLOCK orders threads of one block, GR_GRID orders all threads;
 * Section 2.2), a guard (same meaning; the barrier is executed by the threads
 * whose guard holds) and a weight (Section 2.4: (gw*gb) + lw^ld).  A mask has
 * bit k set when slot k is enabled.
 *
 * Ownership and errors (every entry point).  The caller owns every input and
 * output buffer.  Host-pointer entry points copy their inputs during the call
 * and return after the result is in the caller's memory.  Inputs are
 * validated before any device work (one exception: gr_repair_batch checks
 * that the permutation entries each statement reads are distinct on the
 * device, next to the repair, and reads that back before it copies any
 * result); a rejected
 * call returns GR_EINVAL and leaves the outputs untouched (gr_last_error()
 * says why).  CUDA failures
 * return GR_ECUDA; a failed allocation returns GR_ENOMEM.  The library keeps
 * one device workspace per device, grown on demand and guarded by a mutex:
 * host-pointer calls from several threads are serialised.
 */
#ifndef GPUREPAIR_H
#define GPUREPAIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GR_MAX_STMTS 25
#define GR_MAX_SLOTS 32
#define GR_MAX_THREADS 1024
#define GR_MAX_BLOCKS 65533
#define GR_MAX_WORDS 65536
#define GR_MAX_WEIGHT (1u << 24)
#define GR_MAX_CLAUSES 656
#define GR_MAX_ITERS 64
#define GR_MAX_LOOPS 4
#define GR_MAX_NEG 32
#define GR_MAX_DEADLINE_US (1ull << 40) /* about 12.7 days */

typedef int32_t gr_status;
enum {
    GR_OK = 0,
    GR_UNSAT = 1,      /* gr_solve only: no mask satisfies the clauses */
    GR_EINVAL = -1,    /* invalid argument; outputs untouched */
    GR_ENOMEM = -2,    /* device or host allocation failed */
    GR_ECUDA = -4,     /* a CUDA call failed (gr_last_error has the text) */
    GR_EBUSY = -5,     /* gr_server_poll / gr_server_drain: not finished yet */
    GR_ECAPACITY = -6  /* a buffer the caller passed is too small */
};

enum { GR_R = 0, GR_W = 1 };
enum { GR_SHARED = 0, GR_GLOBAL = 1 };
enum { GR_AFFINE = 0, GR_STRIDED = 1, GR_PERM = 2 };
enum { GR_BLOCK = 0, GR_GRID = 1 };

/* Repair modes (Section 5, Table 3 configurations).
 * GR_MODE_REPAIR  (--disable-inspect): existing barriers stay on; only new
 *                 ones are added.
 * GR_MODE_REMOVE  (default inspection): existing barriers are variables too;
 *                 the existing mask is checked first as a probe and the loop
 *                 may drop barriers that no witness needs. */
enum { GR_MODE_REPAIR = 0, GR_MODE_REMOVE = 1 };

/* Per-program outcome (Algorithm 1's exits).  GR_ITER_CAP and GR_TIMEOUT are
 * the two ways the loop gives up: more checks than gr_options.max_iters, or
 * longer than gr_options.deadline_us (Section 5 runs every kernel under a
 * time limit); both leave mask 0 and keep the trajectory so far. */
enum { GR_REPAIRED = 0, GR_UNREPAIRABLE = 1, GR_ITER_CAP = 2, GR_TIMEOUT = 3 };

typedef struct {
    uint8_t op;        /* GR_R / GR_W */
    uint8_t space;     /* GR_SHARED / GR_GLOBAL */
    uint8_t kind;      /* GR_AFFINE / GR_STRIDED / GR_PERM */
    uint8_t _pad;
    uint32_t a, b, c;  /* map coefficients (a unused for GR_PERM) */
    uint32_t perm_off; /* GR_PERM: offset of this statement's table in perm */
    uint16_t guard_k;  /* 0: unguarded; else tid % guard_k == guard_r */
    uint16_t guard_r;
} gr_stmt;

/* A counted loop (Section 2.2 places candidate barriers at loop heads;
 * Section 2.4 weighs a barrier by the depth of its loop, lw^ld).  Statements
 * lo..hi run `trips` times.  The barrier of slot k stands just before
 * statement k+1 and runs every time control reaches statement k+1, so slot
 * lo-1 is the loop head: it runs before every iteration; slot hi runs once
 * after the last.  Requirements: 1 <= lo <= hi < n_stmts, trips >= 1; two
 * loops are disjoint or nested with the inner one starting after the outer
 * one's first statement; the statement instances executed in all (a loop
 * body once per iteration, recursively) number at most GR_MAX_STMTS. */
typedef struct {
    uint32_t lo, hi, trips;
} gr_loop;

typedef struct {
    uint32_t n_stmts;             /* 1..GR_MAX_STMTS */
    const gr_stmt *stmts;         /* n_stmts entries */
    const uint8_t *slot_level;    /* one per slot (n_slots, or n_stmts-1 if n_slots is 0):
                                     GR_BLOCK / GR_GRID */
    const uint16_t *slot_guard;   /* two per slot: (k, r); NULL = unguarded */
    const uint32_t *slot_weight;  /* one per slot, in 1..GR_MAX_WEIGHT; NULL = paper
                                     defaults gw=12, ld=0: block 1, grid 13 */
    uint32_t m_shared, m_global;  /* words (1..GR_MAX_WORDS) of each array a statement uses */
    const uint32_t *perm;         /* concatenated permutation tables (may be NULL if unused) */
    uint32_t perm_len;
    uint32_t existing_mask;       /* barriers the programmer wrote (E) */
    uint32_t n_loops;             /* 0..GR_MAX_LOOPS counted loops */
    const gr_loop *loops;         /* n_loops entries (may be NULL if n_loops == 0) */
    const uint32_t *iter_coef;    /* n_stmts entries or NULL (= 0): statement s's address
                                     adds iter_coef[s] * t, t in 0..trips-1 the counter of
                                     the innermost loop holding s (0 outside loops) */
    uint32_t n_slots;             /* 0: one slot per place, slot k after statement k (n_stmts-1
                                     slots); else 1..GR_MAX_SLOTS slots placed by slot_pos */
    const uint8_t *slot_pos;      /* n_slots entries or NULL: the statement (0..n_stmts-2) each
                                     slot follows; several slots may share a place, e.g. a block
                                     and a grid candidate at every site (Section 2.2 instruments
                                     both variables per site).  slot_level, slot_guard,
                                     slot_weight, existing_mask and neg index slots. */
    uint32_t n_neg;               /* 0..GR_MAX_NEG negative clauses given with the program */
    const uint32_t *neg;          /* n_neg nonzero slot masks: no repair enables every slot of
                                     one (Section 2.4's negative monotone clauses, supplied from
                                     outside the model, e.g. barrier pairs the programmer rules
                                     out); they join every Solve of the loop, and a greedy (mhs)
                                     proposal that breaks one is replaced by the MaxSAT solve */
} gr_program;

typedef struct {
    uint32_t blocks;   /* 1..GR_MAX_BLOCKS */
    uint32_t threads;  /* 1..GR_MAX_THREADS */
} gr_launch;

/* Witness rows index the executed statement instances in execution order
 * (the statements themselves when the program has no loop). */
typedef struct {
    uint32_t race_intra[32]; /* row i, bit j (j >= i): same-block race witness (i, j) */
    uint32_t race_inter[32]; /* row i, bit j (j >= i): cross-block race witness (i, j) */
    uint32_t diverge;        /* bit k: enabled slot k is divergent */
    uint32_t n_stmts;        /* executed statement instances (rows in use) */
    uint64_t access_pairs;   /* thread pairs a pairwise checker would examine under the
                                mask: instance pairs (i <= j) of one space with a write;
                                ordered pairs for i < j, unordered for i == j; same-block
                                pairs unless an enabled barrier runs between i and j (slots
                                i..j-1 without loops), cross-block pairs (global only)
                                unless an enabled grid barrier does */
} gr_witnesses;

/* Proposal strategies of Algorithm 1's Solve step (Section 2.4). */
enum {
    GR_STRATEGY_MAXSAT = 0, /* every proposal is the minimum-weight hitting set (--maxsat) */
    GR_STRATEGY_MHS = 1     /* greedy minimal hitting sets (Johnson), the MaxSAT solve as the
                               fallback when a clause cannot be hit, and one exact query once a
                               proposal is clean (the paper's default) */
};

typedef struct {
    uint8_t grid_enabled; /* 0 = --disable-grid: every grid slot is forbidden */
    uint8_t strategy;     /* GR_STRATEGY_*; both end at the same minimum mask */
    uint8_t _pad[2];
    uint32_t max_iters;   /* checks allowed per program, 1..GR_MAX_ITERS; 0 = 64 */
    uint64_t deadline_us; /* 0: none.  Else the time limit of each program's loop (Section 5
                             runs the tool under a per-kernel timeout), on the device clock
                             from the moment the program's loop starts: after a Solve, a
                             program whose loop has run at least this long stops with
                             GR_TIMEOUT instead of checking the next proposal.  At most
                             GR_MAX_DEADLINE_US. */
} gr_options;

typedef struct {
    int32_t status;               /* GR_REPAIRED / GR_UNREPAIRABLE / GR_ITER_CAP / GR_TIMEOUT */
    uint32_t mask;                /* final mask (0 unless repaired) */
    uint32_t weight;              /* sum of the weights of mask's slots */
    uint32_t added, removed;      /* mask & ~E, E & ~mask (removed is 0 unless repaired) */
    uint32_t iters;               /* checks performed (the paper's verifier calls) */
    uint32_t traj[GR_MAX_ITERS];  /* the masks checked, in order */
    uint32_t n_clauses;
    uint32_t clauses[GR_MAX_CLAUSES]; /* final positive clauses, sorted, unique */
    uint32_t forbidden;           /* final negative unit clauses (divergent or disabled slots) */
    uint32_t _pad;
    uint64_t access_pairs;        /* summed over this program's checks */
    uint64_t t_start_ns, t_end_ns;/* device clock when the program's loop began / ended */
} gr_repair_result;

/* ---------------------------------------------------------------------- */
/* Library                                                                 */
/* ---------------------------------------------------------------------- */

/* Version string of the engine. */
const char *gr_version(void);
/* Text of the last error raised on the calling thread ("" if none). */
const char *gr_last_error(void);
/* Validate one program and launch without touching the device. */
gr_status gr_validate(const gr_program *prog, gr_launch launch);

/* ---------------------------------------------------------------------- */
/* Host-pointer entry points (synchronous; library-owned device workspace) */
/* ---------------------------------------------------------------------- */

/* Verify(P_sol) of Algorithm 1 (Section 2.4) as an exact concrete check:
 * every race witness and divergent slot of prog under mask.  mask must only
 * use bits < n_stmts-1. */
gr_status gr_check(const gr_program *prog, gr_launch launch, uint32_t mask, gr_witnesses *out);

/* Algorithm 1 (Section 2.4) on one program, in one persistent launch.
 * mode: GR_MODE_REPAIR / GR_MODE_REMOVE.  opts may be NULL (grid enabled,
 * 64 iterations). */
gr_status gr_repair(const gr_program *prog, gr_launch launch, int32_t mode,
                    const gr_options *opts, gr_repair_result *out);

/* The same loop driven from the host with one check launch and one solve
 * launch per iteration (the plain comparison path). Same result as gr_repair. */
gr_status gr_repair_plain(const gr_program *prog, gr_launch launch, int32_t mode,
                          const gr_options *opts, gr_repair_result *out);

/* gr_repair_plain, also writing to *loop_ms (when not NULL) the time, by CUDA
 * events on the call's stream, from the first launch of the loop to its last:
 * the per-iteration launches and the host's reads of the done flag, without
 * validation, packing or the upload.  On an error *loop_ms is unchanged. */
gr_status gr_repair_plain_timed(const gr_program *prog, gr_launch launch, int32_t mode,
                                const gr_options *opts, gr_repair_result *out, float *loop_ms);

/* Minimum-weight hitting set (Section 2.3 definitions, Section 2.4 weighted
 * MaxSAT form) on the GPU: the least (weight, mask) over masks x of n_vars
 * (1..32) bits with forced <= x, x & forbidden == 0, x & pos[i] != 0 for
 * every positive clause and (x & neg[i]) != neg[i] for every negative clause.
 * w: n_vars weights in 1..GR_MAX_WEIGHT.  n_pos + n_neg <= GR_MAX_CLAUSES.
 * Returns GR_OK (outputs set) or GR_UNSAT (outputs set to 0). */
gr_status gr_solve(uint32_t n_vars, const uint32_t *w, const uint32_t *pos, uint32_t n_pos,
                   const uint32_t *neg, uint32_t n_neg, uint32_t forced, uint32_t forbidden,
                   uint32_t *mask_out, uint32_t *weight_out);

/* Algorithm 1 (Section 2.4) on each of many independent programs (uneven
 * sizes), batched on the device: each program's conflict relation (Verify of
 * Section 2.4 under the empty mask) in one check launch, then the loop of
 * every program in one loop launch, on `stream` (a cudaStream_t, NULL =
 * legacy default stream); returns once out holds every result.  Each result
 * equals gr_repair's on the program alone.  modes: one GR_MODE_* per
 * program (Section 5's configurations). */
gr_status gr_repair_batch(const gr_program *progs, const gr_launch *launches,
                          const int32_t *modes, uint32_t n, const gr_options *opts,
                          gr_repair_result *out, void *stream);

/* Verify (Algorithm 1, Section 2.4) of each (program, masks[i]) pair, all in
 * one batched launch: out[i] equals gr_check(progs[i], launches[i], masks[i]). */
gr_status gr_check_batch(const gr_program *progs, const gr_launch *launches,
                         const uint32_t *masks, uint32_t n, gr_witnesses *out, void *stream);

/* ---------------------------------------------------------------------- */
/* Device-resident entry points (asynchronous on `stream`, no allocation)  */
/* ---------------------------------------------------------------------- */

/* Bytes of the packed program arena and of the device scratch (address
 * traces and tile masks) that n programs need. */
gr_status gr_pack_size(const gr_program *progs, const gr_launch *launches, uint32_t n,
                       uint64_t *arena_bytes, uint64_t *scratch_bytes);

/* Validate and pack n programs into a host buffer of arena_bytes (16-byte
 * aligned).  The caller copies it to device memory; it stays valid for any
 * number of launches. */
gr_status gr_pack(const gr_program *progs, const gr_launch *launches, const int32_t *modes,
                  uint32_t n, void *host_arena, uint64_t arena_bytes);

/* Algorithm 1 on every program of a packed arena already in device memory.
 * Programs on the shared array whose blocks see one access pattern (no
 * address depends on the block, or every map shifts by the same offset per
 * block) get their conflict relation from the relation kernel, which
 * computes addresses from the maps; the others (a global array, or blocks
 * that differ) have their address traces expanded into d_scratch and checked
 * by the general check kernel; then the loop kernel runs Algorithm 1 per
 * program on the relations.  d_out: n results in device memory.  Enqueued on
 * stream; nothing is allocated and nothing synchronises.  d_arena and
 * d_scratch must be 256-byte aligned; n must be the arena's program count and
 * scratch_bytes at least gr_pack_size's figure.  The kernels compare both
 * with the arena header: on a mismatch they do nothing (d_out untouched) and
 * set bit 2 (value 4) of the device error word, the 32-bit word at byte 4 of
 * d_scratch, which the host-pointer calls report as GR_ECUDA. */
gr_status gr_repair_packed(const void *d_arena, uint32_t n, const gr_options *opts,
                           void *d_scratch, uint64_t scratch_bytes, gr_repair_result *d_out,
                           void *stream);

/* The same repair as gr_repair_packed, spread wide for programs with many
 * blocks: every check runs one CTA per (program, block) for the same-block
 * passes plus one CTA per program for the cross-block pass, divergence and the
 * pair count, and one CTA per program takes each loop step (Algorithm 1's
 * clause building and Solve).  The loop itself runs on the device as a CUDA
 * graph whose while-node repeats [check, step] until every program is decided
 * (bounded: GR_MAX_ITERS + 4 rounds; running past the bound sets the device
 * error word).  Results equal gr_repair_packed's.  Reads the 192-byte arena
 * header back to the host (a synchronising copy on stream), then enqueues the
 * expansion and the graph on stream.  n <= 65,535. */
gr_status gr_repair_packed_wide(const void *d_arena, uint32_t n, const gr_options *opts,
                                void *d_scratch, uint64_t scratch_bytes, gr_repair_result *d_out,
                                void *stream);

/* The two halves of gr_repair_packed, for callers that time or overlap them:
 * gr_expand_packed writes the address traces and chunk masks of the programs
 * the general check kernel reads (a global array, or blocks that differ) into
 * d_scratch; gr_repair_expanded runs the relation, check and loop kernels on
 * traces a previous gr_expand_packed of the same arena wrote. */
gr_status gr_expand_packed(const void *d_arena, void *d_scratch, uint64_t scratch_bytes, void *stream);
gr_status gr_repair_expanded(const void *d_arena, uint32_t n, const gr_options *opts, void *d_scratch,
                             uint64_t scratch_bytes, gr_repair_result *d_out, void *stream);

/* The two stages of gr_repair_expanded, for callers that time them apart.
 * gr_relation_packed: Verify (Algorithm 1, Section 2.4) of every program
 * under the empty mask, i.e. each program's conflict relation (every
 * instance pair with a write that conflicts on some word, same-block and
 * cross-block), written into d_scratch: the relation kernel for programs on
 * the shared array with alike blocks, the general check kernel on the traces
 * a previous gr_expand_packed wrote for the others.  gr_loop_packed: the
 * loop of Algorithm 1 for every program on the relations a previous
 * gr_relation_packed of the same arena wrote (Verify of a proposal is the
 * relation restricted to the proposal's phases, exact because a witness's
 * clause is exactly the slots that order it), results into d_out.  The two
 * calls in order on one stream equal gr_repair_expanded. */
gr_status gr_relation_packed(const void *d_arena, uint32_t n, void *d_scratch, uint64_t scratch_bytes,
                             void *stream);
gr_status gr_loop_packed(const void *d_arena, uint32_t n, const gr_options *opts, void *d_scratch,
                         uint64_t scratch_bytes, gr_repair_result *d_out, void *stream);

/* The repair of gr_repair_packed as one launch, whatever the autotuner
 * picked: the relation kernel computes each program's relation, then its
 * warps run the loop of Algorithm 1 (Section 2.4) on the relations, each
 * program's loop waiting for a flag its relation sets (a bounded wait:
 * when it runs out, that program's result is not written, the warp takes
 * no further program and bit 3, value 8, of the device error word at byte 4
 * of d_scratch is set).  Only for a batch of straight-line
 * programs on the shared array with no general program (the packer's simple
 * flag, no program needing expanded traces); any other batch returns
 * GR_EINVAL with nothing launched.  Reads the arena header back and
 * synchronises on it (not capturable), then enqueues the launch on stream.
 * Results into d_out as gr_repair_packed writes them. */
gr_status gr_relation_loop_packed(const void *d_arena, uint32_t n, const gr_options *opts, void *d_scratch,
                                  uint64_t scratch_bytes, gr_repair_result *d_out, void *stream);

/* Autotuner: time every CTA shape the check kernels are built for (threads
 * per CTA x CTAs per SM, with the owner-table budget that shape leaves) on
 * this arena, remember the fastest for later gr_repair_packed /
 * gr_repair_expanded / gr_check_packed calls (and gr_repair_packed_noalloc)
 * on the same (d_arena, n), and return them in shape_out (may be NULL): bits
 * 0-7 index the relation kernel's shape, bits 8-11 the general check
 * kernel's, bit 12 is set when that kernel's grid is cut so that every CTA
 * gets the same number of programs (fewer CTAs than fit, no partly filled
 * last round); bit 16 (the relation kernel running the loop too, in one
 * launch) is never set here: it is set through gr_set_shape_packed, and
 * gr_relation_loop_packed runs that launch directly.  Runs the kernels
 * several times, then one repair with the choices picked into d_out, and
 * synchronises the stream.  The
 * host-pointer batch calls tune the same way by themselves, once per batch
 * size class. */
gr_status gr_tune_packed(const void *d_arena, uint32_t n, const gr_options *opts, void *d_scratch,
                         uint64_t scratch_bytes, gr_repair_result *d_out, void *stream, uint32_t *shape_out);

/* Record a shape word for later calls on (d_arena, n) without timing
 * anything, as if gr_tune_packed had picked it: a word gr_tune_packed
 * returned earlier (for this batch or one like it, in this process or
 * another), so a caller can tune once and reuse the choice.  The word's
 * fields are gr_tune_packed's.  GR_EINVAL, with nothing recorded, for a
 * field that names no built shape, a bit above 16, or bit 16 on a batch
 * that cannot run in one launch.  Reads the arena header back on stream
 * (synchronises); launches no kernel and writes no device memory. */
gr_status gr_set_shape_packed(const void *d_arena, uint32_t n, uint32_t shape, void *stream);

/* One check per program of a device-resident packed arena under d_masks[p]. */
gr_status gr_check_packed(const void *d_arena, uint32_t n, const uint32_t *d_masks,
                          void *d_scratch, uint64_t scratch_bytes, gr_witnesses *d_out,
                          void *stream);
/* gr_check_packed without the expansion: the checks alone, on traces a
 * previous gr_expand_packed (or gr_check_packed / gr_repair_packed) of the same
 * arena wrote into d_scratch.  For callers that time the check kernel. */
gr_status gr_check_expanded(const void *d_arena, uint32_t n, const uint32_t *d_masks,
                            void *d_scratch, uint64_t scratch_bytes, gr_witnesses *d_out,
                            void *stream);

/* ---------------------------------------------------------------------- */
/* Repair server: continuous batching over a device-memory budget          */
/* ---------------------------------------------------------------------- */

/* A server repairs single programs submitted at any time (the repair loop of
 * Algorithm 1, Section 2.4, per request; each result equals gr_repair's).
 * It owns n_slots (1..16) launch slots, each with its own stream and
 * device buffers; together they take mem_budget_bytes of
 * device memory, allocated here, and nothing more is allocated while
 * serving.  A dispatcher thread admits queued requests in arrival order into
 * whichever slot is idle, as many as fit the slot's share of the budget and
 * the max_inflight cap, and runs them as one persistent repair launch;
 * requests that arrive while other launches run are admitted by the next
 * free slot and overlap with them on the device.  Each request's traces,
 * clauses and masks stay on the device for its whole loop.  opts may be
 * NULL.  The server binds to the device current at creation. */
typedef struct gr_server gr_server;
gr_status gr_server_create(uint64_t mem_budget_bytes, uint32_t n_slots, uint32_t max_inflight,
                           const gr_options *opts, gr_server **out);
/* Copy one program (the caller may free it on return) and queue it.  Returns
 * a ticket.  GR_ECAPACITY if the program alone exceeds one slot's memory. */
gr_status gr_server_submit(gr_server *s, const gr_program *prog, gr_launch launch, int32_t mode,
                           uint64_t *ticket);
/* GR_OK and the result (and, if latency_ns is not NULL, the time from submit
 * to completion seen by the server) once the request is done, after which the
 * ticket is forgotten; GR_EBUSY while it is queued or running. */
gr_status gr_server_poll(gr_server *s, uint64_t ticket, gr_repair_result *out, uint64_t *latency_ns);
/* Wait until nothing is queued or running (GR_OK) or timeout_ms passed (GR_EBUSY). */
gr_status gr_server_drain(gr_server *s, uint32_t timeout_ms);
/* Queued requests, requests on the device, launches issued so far. */
gr_status gr_server_stats(gr_server *s, uint64_t *pending, uint64_t *inflight, uint64_t *launches);
/* Stop the dispatcher, wait for the device, free everything. */
gr_status gr_server_destroy(gr_server *s);

/* gr_repair_packed without a scratch buffer, for callers that cannot
 * allocate device memory where they run the repair (inside a host callback or
 * another allocation-free path, a plug-in whose host forbids allocation after
 * start-up, a real-time loop that must not pay cudaMalloc's implicit device
 * synchronisation).  The paper has no counterpart: this is a deployment
 * variant of the same launch.
 * The scratch is a fixed 64 MiB device array inside the library, held by
 * every GPU that loads the library until the process exits; a batch whose
 * gr_pack_size scratch figure exceeds it is rejected with GR_ECAPACITY.  The
 * first call on a device sets that device up (it looks up the array's
 * device address, with the device current), so that first call should come
 * before any stream capture; a cudaDeviceReset of the device discards the
 * array, and the entry point must not be called on that device again in
 * the same process.  Each call reads the 192-byte arena header back to the
 * host (a synchronising copy on stream); it allocates nothing, validates
 * opts as gr_repair_packed does and launches what
 * gr_repair_packed launches (with the shapes gr_tune_packed recorded for
 * (d_arena, n), else the defaults).  Device-side errors (the device error
 * word) are not reported on this path: the word stays in the fixed array.
 * All calls share the array: calls whose GPU work overlaps (other streams,
 * other threads) race and must not be issued.
 * d_arena: a gr_pack arena in device memory, 256-byte aligned; d_out: n
 * results in device memory.  Enqueued on stream. */
gr_status gr_repair_packed_noalloc(const void *d_arena, uint32_t n, const gr_options *opts,
                                   gr_repair_result *d_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GPUREPAIR_H */
