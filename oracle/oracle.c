/*
 * CPU oracle for the barrier-repair loop of GPURepair (arXiv 2011.08373).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, literal C: every function below
 * writes out a definition or the steps of Algorithm 1 with no blocking,
 * fusion or reordering.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library; the product path never
 * does.  It shares no code, header or table with the CUDA engine.
 *
 * Model (the paper's instrumented kernel, Section 2.2, restated over a
 * concrete launch of B blocks x T threads):
 *   statement s: op (0 read / 1 write), space (0 shared: one private array per
 *   block / 1 global: one array for the grid), address map
 *     affine, strided : (a*tid + c*blk + b) mod M
 *     permutation     : perm[perm_off + ((tid + c*blk + b) mod M)]
 *   and guard (k, r): statement s runs for thread tid iff k == 0 or tid%k == r.
 *   slot k (between statements k and k+1): level (0 block / 1 grid),
 *   guard (k, r) with the same meaning, weight w_k.  With explicit slot
 *   positions several slots may share one place: slot k then sits after
 *   statement slot_pos[k] (two slots per place, one block and one grid, give
 *   the paper's two barrier variables per candidate site).
 *   counted loops (lo, hi, trips): statements lo..hi run trips times; a
 *   statement's address adds d*t, t the counter (0..trips-1) of its innermost
 *   loop.  The barrier of slot k stands just before statement k+1, so it runs
 *   every time control reaches statement k+1: the loop-head slot lo-1 runs
 *   before every iteration, the exit slot hi once after the last one.
 *
 * Parity-pinned functions (see tests/test_oracle_pins.py):
 *   orc_check  -- pinned by the paper's listings (Section 1, Appendix A.4),
 *                 an independent flag-reset race detector (Section 2.2),
 *                 a number-theoretic closed form for affine maps, invariants.
 *   orc_clauses-- pinned by the exact-filter invariant against orc_check.
 *   orc_solve  -- pinned by the mhs counterexample of Section 2.4, interval
 *                 stabbing by dynamic programming, and scipy's MILP solver.
 *   orc_repair -- pinned by the listings and by the path-independence lemma
 *                 (final mask = lowest-key witness-free mask over all masks).
 *   orc_check_words, orc_repair_words -- the same definitions grouped by
 *                 word (for full-size launches), pinned by equality with
 *                 orc_check / orc_repair on random programs.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_STMTS 25
#define ORC_MAX_CLAUSES 656
#define ORC_MAX_TRAJ 64

typedef struct {
    uint32_t n_stmts;
    const uint8_t *op, *space, *kind;
    const uint32_t *a, *b, *c, *perm_off;
    const uint32_t *guard_k, *guard_r;         /* per statement */
    const uint8_t *slot_level;                 /* per slot */
    const uint32_t *slot_guard_k, *slot_guard_r;
    const uint32_t *slot_weight;
    uint32_t m_shared, m_global;
    const uint32_t *perm;
    uint32_t perm_len;
    uint32_t existing_mask;
    uint32_t blocks, threads;
    uint32_t n_loops;
    const uint32_t *loop_lo, *loop_hi, *loop_trips; /* per loop */
    const uint32_t *iter_coef;                      /* per statement; NULL = 0 */
    uint32_t n_neg;                                 /* negative clauses given with the program */
    const uint32_t *neg;                            /* each: not all of these slots together */
    uint32_t n_slots;                               /* 0: n_stmts - 1, one slot per place */
    const uint32_t *slot_pos;                       /* per slot: the statement it follows; NULL: k */
} orc_prog;

typedef struct {
    uint32_t intra[32]; /* row i: bit j set <=> same-block witness (i, j), j >= i */
    uint32_t inter[32]; /* row i: bit j set <=> cross-block witness (i, j)        */
    uint32_t diverge;   /* bit k set <=> enabled slot k is divergent               */
    uint64_t access_pairs;
} orc_witness;

typedef struct {
    int32_t status; /* 0 repaired, 1 unrepairable, 2 iteration cap reached */
    uint32_t mask, weight, added, removed, iters;
    uint32_t traj[ORC_MAX_TRAJ];
    uint32_t n_clauses;
    uint32_t clauses[ORC_MAX_CLAUSES];
    uint32_t forbidden;
    uint64_t access_pairs;
} orc_result;

/* --- the model's primitive definitions ----------------------------------- */

static int orc_active(uint32_t k, uint32_t r, uint32_t tid) {
    return k == 0 || tid % k == r;
}

/* Address of statement s for thread tid of block blk in iteration it of the
 * statement's innermost loop (it = 0 outside loops). */
static uint32_t orc_addr(const orc_prog *p, uint32_t s, uint32_t blk, uint32_t tid, uint32_t it) {
    uint64_t M = p->space[s] == 0 ? p->m_shared : p->m_global;
    const uint64_t d = p->iter_coef ? (uint64_t)p->iter_coef[s] * it : 0;
    if (p->kind[s] == 2) {
        uint64_t idx = ((uint64_t)tid + (uint64_t)p->c[s] * blk + p->b[s] + d) % M;
        return p->perm[p->perm_off[s] + idx];
    }
    return (uint32_t)(((uint64_t)p->a[s] * tid + (uint64_t)p->c[s] * blk + p->b[s] + d) % M);
}

/* The statements in execution order (each statement of a loop body once per
 * iteration): st[x] is the statement of the x-th executed instance, it[x] the
 * counter of its innermost loop.  Statements lo..hi of the range, which is
 * the body of loop `in` (-1: the whole program) in its iteration t. */
static void orc_emit(const orc_prog *p, uint32_t lo, uint32_t hi, int in, uint32_t t, uint32_t *st,
                     uint32_t *it, uint32_t *n) {
    uint32_t s = lo;
    while (s <= hi) {
        int l = -1;
        for (uint32_t q = 0; q < p->n_loops; q++)
            if ((int)q != in && p->loop_lo[q] == s) l = (int)q;
        if (l < 0) {
            if (*n < ORC_MAX_STMTS) {
                st[*n] = s;
                it[*n] = t;
            }
            (*n)++;
            s++;
            continue;
        }
        for (uint32_t t2 = 0; t2 < p->loop_trips[l]; t2++)
            orc_emit(p, p->loop_lo[l], p->loop_hi[l], l, t2, st, it, n);
        s = p->loop_hi[l] + 1;
    }
}

/* Number of executed statement instances (at most ORC_MAX_STMTS are stored). */
uint32_t orc_unroll(const orc_prog *p, uint32_t *st, uint32_t *it) {
    uint32_t n = 0;
    orc_emit(p, 0, p->n_stmts - 1, -1, 0, st, it, &n);
    return n;
}

static uint32_t orc_nslots(const orc_prog *p) { return p->n_slots ? p->n_slots : p->n_stmts - 1; }

static uint32_t orc_pos(const orc_prog *p, uint32_t k) { return p->slot_pos ? p->slot_pos[k] : k; }

/* Is there an enabled barrier (any level / grid level) among those that run
 * between instances x < y?  The barrier of a slot after statement q runs each
 * time control reaches statement q+1.  A block barrier orders the accesses of threads in the same
 * block, a grid barrier those of every pair of threads (Section 2.2, flag
 * reset). */
static int orc_separated(const orc_prog *p, const uint32_t *st, uint32_t mask, uint32_t x, uint32_t y,
                         int grid_only) {
    for (uint32_t z = x + 1; z <= y; z++) {
        const uint32_t q = st[z] - 1;
        for (uint32_t k = 0; k < orc_nslots(p); k++)
            if (orc_pos(p, k) == q && ((mask >> k) & 1u))
                if (!grid_only || p->slot_level[k] == 1) return 1;
    }
    return 0;
}

/* Check P under barrier mask m: every race witness (x, y) and every
 * divergent enabled slot.  Definition by enumeration of all thread pairs over
 * the executed statement instances x <= y (orc_unroll; without loops
 * instance x is statement x).
 *   (x, y), same space, at least one write: a witness exists iff there are
 *   distinct threads g1 (running x) and g2 (running y) with the same address
 *   in the same array instance (same block for shared arrays), and no enabled
 *   barrier runs between x and y.  Same-block pairs go to intra[x], cross
 *   block pairs to inter[x].  Values are not modelled: equal-value writes race
 *   (Appendix A.4, write-write race).
 *   Slot k diverges iff it is enabled and its guard is true for some thread
 *   of a block and false for another (Section 1, barrier divergence).
 * access_pairs counts the thread pairs examined: for x < y ordered pairs
 * (g1 at x, g2 at y), for x == y unordered pairs, each only while its scope
 * (same block / cross block) is not separated under m. */
void orc_check(const orc_prog *p, uint32_t mask, orc_witness *out) {
    memset(out, 0, sizeof(*out));
    uint32_t st[ORC_MAX_STMTS], it[ORC_MAX_STMTS];
    const uint32_t X = orc_unroll(p, st, it);
    if (X > ORC_MAX_STMTS) return;
    const uint32_t B = p->blocks, T = p->threads;
    const uint64_t G = (uint64_t)B * T;
    /* each instance's address and guard, evaluated once per thread */
    uint32_t *addr = (uint32_t *)malloc(sizeof(uint32_t) * X * G);
    uint8_t *act = (uint8_t *)malloc(X * (size_t)T);
    for (uint32_t x = 0; x < X; x++) {
        const uint32_t s = st[x];
        for (uint32_t t = 0; t < T; t++) act[(size_t)x * T + t] = (uint8_t)orc_active(p->guard_k[s], p->guard_r[s], t);
        for (uint32_t b = 0; b < B; b++)
            for (uint32_t t = 0; t < T; t++) addr[x * G + (uint64_t)b * T + t] = orc_addr(p, s, b, t, it[x]);
    }
    for (uint32_t x = 0; x < X; x++) {
        for (uint32_t y = x; y < X; y++) {
            const uint32_t i = st[x], j = st[y];
            if (p->space[i] != p->space[j]) continue;
            if (p->op[i] != 1 && p->op[j] != 1) continue;
            const int shared = p->space[i] == 0;
            const int open_same = !orc_separated(p, st, mask, x, y, 0);
            const int open_cross = !shared && !orc_separated(p, st, mask, x, y, 1);
            if (!open_same && !open_cross) continue;
            for (uint32_t b1 = 0; b1 < B; b1++) {
                for (uint32_t t1 = 0; t1 < T; t1++) {
                    if (!act[(size_t)x * T + t1]) continue;
                    const uint32_t a1 = addr[x * G + (uint64_t)b1 * T + t1];
                    for (uint32_t b2 = 0; b2 < B; b2++) {
                        const int same = b1 == b2;
                        if (same && !open_same) continue;
                        if (!same && !open_cross) continue;
                        for (uint32_t t2 = 0; t2 < T; t2++) {
                            if (same && t1 == t2) continue;
                            /* one instance: count each unordered pair once */
                            if (x == y && (uint64_t)b2 * T + t2 < (uint64_t)b1 * T + t1) continue;
                            if (!act[(size_t)y * T + t2]) continue;
                            out->access_pairs++;
                            if (addr[y * G + (uint64_t)b2 * T + t2] != a1) continue;
                            if (same) out->intra[x] |= 1u << y;
                            else out->inter[x] |= 1u << y;
                        }
                    }
                }
            }
        }
    }
    free(addr);
    free(act);
    for (uint32_t k = 0; k < orc_nslots(p); k++) {
        if (!((mask >> k) & 1u) || p->slot_guard_k[k] == 0) continue;
        int seen_true = 0, seen_false = 0;
        for (uint32_t t = 0; t < T; t++) {
            if (orc_active(p->slot_guard_k[k], p->slot_guard_r[k], t)) seen_true = 1;
            else seen_false = 1;
        }
        if (seen_true && seen_false) out->diverge |= 1u << k;
    }
}

/* The same definition for one instance pair (x <= y): whether a same-block
 * and a cross-block witness (x, y) exist under mask m, and the thread pairs
 * examined.  Used to sample full-size launches whose whole check is too slow
 * to enumerate. */
void orc_check_pair(const orc_prog *p, uint32_t mask, uint32_t x, uint32_t y, int32_t *intra, int32_t *inter,
                    uint64_t *pairs) {
    *intra = 0;
    *inter = 0;
    *pairs = 0;
    uint32_t st[ORC_MAX_STMTS], it[ORC_MAX_STMTS];
    const uint32_t X = orc_unroll(p, st, it);
    const uint32_t B = p->blocks, T = p->threads;
    if (X > ORC_MAX_STMTS || x > y || y >= X) return;
    const uint32_t i = st[x], j = st[y];
    if (p->space[i] != p->space[j]) return;
    if (p->op[i] != 1 && p->op[j] != 1) return;
    const int shared = p->space[i] == 0;
    const int open_same = !orc_separated(p, st, mask, x, y, 0);
    const int open_cross = !shared && !orc_separated(p, st, mask, x, y, 1);
    if (!open_same && !open_cross) return;
    const uint64_t G = (uint64_t)B * T;
    uint32_t *ai = (uint32_t *)malloc(sizeof(uint32_t) * G);
    uint32_t *aj = (uint32_t *)malloc(sizeof(uint32_t) * G);
    for (uint32_t b = 0; b < B; b++)
        for (uint32_t t = 0; t < T; t++) {
            ai[(uint64_t)b * T + t] = orc_addr(p, i, b, t, it[x]);
            aj[(uint64_t)b * T + t] = orc_addr(p, j, b, t, it[y]);
        }
    for (uint32_t b1 = 0; b1 < B; b1++) {
        for (uint32_t t1 = 0; t1 < T; t1++) {
            if (!orc_active(p->guard_k[i], p->guard_r[i], t1)) continue;
            const uint32_t a1 = ai[(uint64_t)b1 * T + t1];
            for (uint32_t b2 = 0; b2 < B; b2++) {
                const int same = b1 == b2;
                if (same && !open_same) continue;
                if (!same && !open_cross) continue;
                for (uint32_t t2 = 0; t2 < T; t2++) {
                    if (same && t1 == t2) continue;
                    if (x == y && (uint64_t)b2 * T + t2 < (uint64_t)b1 * T + t1) continue;
                    if (!orc_active(p->guard_k[j], p->guard_r[j], t2)) continue;
                    (*pairs)++;
                    if (aj[(uint64_t)b2 * T + t2] != a1) continue;
                    if (same) *intra = 1;
                    else *inter = 1;
                }
            }
        }
    }
    free(ai);
    free(aj);
}

/* orc_check's definition grouped by word, for full-size launches whose
 * thread-pair enumeration is too slow.  Two accesses can only race at a word
 * both touch, so each instance's active accesses are sorted by (word, block,
 * thread) and, for an instance pair, only the accesses of each word the two
 * share are paired; a pair races under the same conditions as in orc_check
 * (distinct threads; same block for the same-block scope, different blocks
 * for the cross-block one, the latter only on the global array; the scope
 * not separated under m).  The thread pairs orc_check examines do not depend
 * on the addresses, so their number is counted rather than enumerated: for
 * x < y, B (n_x n_y - n_xy) same-block pairs (t1 != t2; n_xy threads run
 * both) and B (B - 1) n_x n_y cross-block pairs; for x == y, each unordered
 * pair once, B n_x (n_x - 1) / 2 and B (B - 1) / 2 n_x^2 (n_x: the threads of
 * a block that run x).  Pinned against orc_check on random programs
 * (tests/test_oracle_pins.py). */
typedef struct {
    uint32_t word, blk, tid;
} orc_acc;

static int orc_cmp_acc(const void *u, const void *v) {
    const orc_acc *a = (const orc_acc *)u, *b = (const orc_acc *)v;
    if (a->word != b->word) return a->word < b->word ? -1 : 1;
    if (a->blk != b->blk) return a->blk < b->blk ? -1 : 1;
    if (a->tid != b->tid) return a->tid < b->tid ? -1 : 1;
    return 0;
}

void orc_check_words(const orc_prog *p, uint32_t mask, orc_witness *out) {
    memset(out, 0, sizeof(*out));
    uint32_t st[ORC_MAX_STMTS], it[ORC_MAX_STMTS];
    const uint32_t X = orc_unroll(p, st, it);
    if (X > ORC_MAX_STMTS) return;
    const uint32_t B = p->blocks, T = p->threads;
    const uint64_t G = (uint64_t)B * T;
    orc_acc *acc = (orc_acc *)malloc(sizeof(orc_acc) * X * G);
    uint8_t *act = (uint8_t *)malloc(X * (size_t)T);
    uint64_t cnt[ORC_MAX_STMTS], nact[ORC_MAX_STMTS];
    for (uint32_t x = 0; x < X; x++) {
        const uint32_t s = st[x];
        nact[x] = 0;
        for (uint32_t t = 0; t < T; t++) {
            act[(size_t)x * T + t] = (uint8_t)orc_active(p->guard_k[s], p->guard_r[s], t);
            nact[x] += act[(size_t)x * T + t];
        }
        uint64_t n = 0;
        for (uint32_t b = 0; b < B; b++)
            for (uint32_t t = 0; t < T; t++)
                if (act[(size_t)x * T + t]) acc[x * G + n++] = (orc_acc){orc_addr(p, s, b, t, it[x]), b, t};
        cnt[x] = n;
        qsort(acc + x * G, n, sizeof(orc_acc), orc_cmp_acc);
    }
    for (uint32_t x = 0; x < X; x++) {
        for (uint32_t y = x; y < X; y++) {
            const uint32_t i = st[x], j = st[y];
            if (p->space[i] != p->space[j]) continue;
            if (p->op[i] != 1 && p->op[j] != 1) continue;
            const int shared = p->space[i] == 0;
            const int open_same = !orc_separated(p, st, mask, x, y, 0);
            const int open_cross = !shared && !orc_separated(p, st, mask, x, y, 1);
            if (!open_same && !open_cross) continue;
            const uint64_t nx = nact[x], ny = nact[y], bb = B;
            if (x < y) {
                uint64_t nxy = 0;
                for (uint32_t t = 0; t < T; t++) nxy += act[(size_t)x * T + t] && act[(size_t)y * T + t];
                if (open_same) out->access_pairs += bb * (nx * ny - nxy);
                if (open_cross) out->access_pairs += bb * (bb - 1) * nx * ny;
            } else {
                if (open_same) out->access_pairs += bb * (nx * (nx - 1) / 2);
                if (open_cross) out->access_pairs += bb * (bb - 1) / 2 * nx * nx;
            }
            /* the words both instances touch, in order */
            const orc_acc *ax = acc + x * G, *ay = acc + y * G;
            int found_same = 0, found_cross = 0;
            uint64_t u = 0, v = 0;
            while (u < cnt[x] && v < cnt[y] && (open_same > found_same || open_cross > found_cross)) {
                if (ax[u].word < ay[v].word) {
                    u++;
                } else if (ax[u].word > ay[v].word) {
                    v++;
                } else {
                    const uint32_t w = ax[u].word;
                    uint64_t u1 = u, v1 = v;
                    while (u1 < cnt[x] && ax[u1].word == w) u1++;
                    while (v1 < cnt[y] && ay[v1].word == w) v1++;
                    for (uint64_t a = u; a < u1; a++)
                        for (uint64_t c = v; c < v1; c++) {
                            const int same = ax[a].blk == ay[c].blk;
                            if (same && ax[a].tid == ay[c].tid) continue; /* one thread */
                            if (same && open_same) found_same = 1;
                            if (!same && open_cross) found_cross = 1;
                        }
                    u = u1;
                    v = v1;
                }
            }
            if (found_same) out->intra[x] |= 1u << y;
            if (found_cross) out->inter[x] |= 1u << y;
        }
    }
    free(acc);
    free(act);
    for (uint32_t k = 0; k < orc_nslots(p); k++) {
        if (!((mask >> k) & 1u) || p->slot_guard_k[k] == 0) continue;
        int seen_true = 0, seen_false = 0;
        for (uint32_t t = 0; t < T; t++) {
            if (orc_active(p->slot_guard_k[k], p->slot_guard_r[k], t)) seen_true = 1;
            else seen_false = 1;
        }
        if (seen_true && seen_false) out->diverge |= 1u << k;
    }
}

/* GenerateClause (Section 2.4): a race witness (x, y) is avoided exactly when
 * some barrier able to order it is on: any slot whose barrier runs between
 * instances x and y for a same-block witness, such a grid slot for a
 * cross-block one.  Without loops that is slots x .. y-1; (x, x) gives the
 * empty clause.  Result: the set of clauses as sorted unique masks. */
static int orc_cmp_u32(const void *x, const void *y) {
    uint32_t a = *(const uint32_t *)x, b = *(const uint32_t *)y;
    return a < b ? -1 : a > b;
}

static uint32_t orc_slots_between(const orc_prog *p, const uint32_t *st, uint32_t x, uint32_t y) {
    uint32_t m = 0;
    for (uint32_t z = x + 1; z <= y; z++)
        for (uint32_t k = 0; k < orc_nslots(p); k++)
            if (orc_pos(p, k) == st[z] - 1u) m |= 1u << k;
    return m;
}

uint32_t orc_clauses(const orc_prog *p, const orc_witness *w, uint32_t *clauses, uint32_t n_in) {
    uint32_t grid = 0, n = n_in;
    for (uint32_t k = 0; k < orc_nslots(p); k++)
        if (p->slot_level[k] == 1) grid |= 1u << k;
    uint32_t st[ORC_MAX_STMTS], it[ORC_MAX_STMTS];
    const uint32_t X = orc_unroll(p, st, it);
    if (X > ORC_MAX_STMTS) return n_in;
    for (uint32_t x = 0; x < X; x++) {
        for (uint32_t y = x; y < X; y++) {
            if ((w->intra[x] >> y) & 1u) clauses[n++] = orc_slots_between(p, st, x, y);
            if ((w->inter[x] >> y) & 1u) clauses[n++] = orc_slots_between(p, st, x, y) & grid;
        }
    }
    qsort(clauses, n, sizeof(uint32_t), orc_cmp_u32);
    uint32_t u = 0;
    for (uint32_t t = 0; t < n; t++)
        if (u == 0 || clauses[u - 1] != clauses[t]) clauses[u++] = clauses[t];
    return u;
}

/* Minimum-weight hitting set (Section 2.3 definitions; weighted form of
 * Section 2.4): among masks x with forced <= x, x & forbidden == 0, x hitting
 * every positive clause and not containing any negative clause, the least
 * (weight(x), x) in lexicographic order.  Brute force over all 2^n masks.
 * Returns 0 and fills mask/weight, or 1 if no such mask exists. */
int orc_solve(uint32_t n, const uint32_t *w, const uint32_t *pos, uint32_t n_pos,
              const uint32_t *neg, uint32_t n_neg, uint32_t forced, uint32_t forbidden,
              uint32_t *mask_out, uint64_t *weight_out) {
    int found = 0;
    uint64_t best_w = 0;
    uint32_t best_x = 0;
    const uint64_t total = 1ull << n;
    for (uint64_t xx = 0; xx < total; xx++) {
        const uint32_t x = (uint32_t)xx;
        if ((x & forced) != forced) continue;
        if (x & forbidden) continue;
        int ok = 1;
        for (uint32_t c = 0; c < n_pos && ok; c++)
            if ((x & pos[c]) == 0) ok = 0;
        for (uint32_t c = 0; c < n_neg && ok; c++)
            if ((x & neg[c]) == neg[c]) ok = 0;
        if (!ok) continue;
        uint64_t wt = 0;
        for (uint32_t k = 0; k < n; k++)
            if ((x >> k) & 1u) wt += w[k];
        if (!found || wt < best_w || (wt == best_w && x < best_x)) {
            found = 1;
            best_w = wt;
            best_x = x;
        }
    }
    if (!found) return 1;
    *mask_out = best_x;
    *weight_out = best_w;
    return 0;
}

/* The mhs strategy's hitting set (Section 2.4: a polynomial greedy algorithm
 * after Johnson, 1974, giving a minimal hitting set).  Starting from the forced
 * variables, repeatedly take the allowed (not forbidden) variable that hits the
 * most clauses not yet hit per unit of weight — ratios compared by cross
 * multiplication, ties to the lower index — until every clause is hit; then
 * make the set minimal by dropping, from the highest index down, each
 * non-forced variable whose removal leaves every clause hit.
 * Returns 0 and the mask, or 1 if some clause has no allowed variable. */
int orc_greedy(uint32_t n, const uint32_t *w, const uint32_t *pos, uint32_t n_pos, uint32_t forced,
               uint32_t forbidden, uint32_t *mask_out) {
    uint32_t x = forced;
    if (forced & forbidden) return 1;
    for (uint32_t c = 0; c < n_pos; c++)
        if (!(pos[c] & x) && !(pos[c] & ~forbidden)) return 1;
    for (;;) {
        int best = -1;
        uint32_t best_hits = 0;
        for (uint32_t k = 0; k < n; k++) {
            if (((x >> k) & 1u) || ((forbidden >> k) & 1u)) continue;
            uint32_t hits = 0;
            for (uint32_t c = 0; c < n_pos; c++)
                if (!(pos[c] & x) && ((pos[c] >> k) & 1u)) hits++;
            if (hits == 0) continue;
            if (best < 0 || (uint64_t)hits * w[best] > (uint64_t)best_hits * w[k]) {
                best = (int)k;
                best_hits = hits;
            }
        }
        if (best < 0) break;
        x |= 1u << best;
    }
    for (int k = (int)n - 1; k >= 0; k--) {
        if (!((x >> k) & 1u) || ((forced >> k) & 1u)) continue;
        const uint32_t y = x & ~(1u << k);
        int ok = 1;
        for (uint32_t c = 0; c < n_pos && ok; c++)
            if (!(pos[c] & y)) ok = 0;
        if (ok) x = y;
    }
    *mask_out = x;
    return 0;
}

/* Algorithm 1, with the exact clause of each witness.
 *   strategy 0 (the paper's MaxSAT strategy): every proposal is the minimum
 *     hitting set of the clauses so far.
 *   strategy 1 (the paper's mhs strategy, its default): proposals are greedy
 *     minimal hitting sets; when a clause has no allowed variable the MaxSAT
 *     solve is used instead; once a greedy proposal is clean, one exact solve
 *     decides: the same mask ends the loop, a lighter one is checked next and
 *     the loop continues with exact proposals.
 *   mode 0 (repair, inspection off): existing barriers are forced on.
 *   mode 1 (remove, inspection on): no slot is forced; the existing mask is
 *     checked first as a probe whose witnesses seed the clause set, and is not
 *     itself returned.
 *   grid_enabled == 0 forbids every grid slot.
 *   Negative clauses given with the program (p->neg) hold throughout: no
 *   proposal contains all slots of one; a greedy proposal that does is
 *   replaced by the MaxSAT solve (the fallback of Section 2.4).
 * Loop: propose the minimum hitting set of the clauses so far; stop when a
 * proposed mask has no witness (repaired) or the clauses are unsatisfiable
 * (unrepairable); each race witness adds its clause, each divergent slot a
 * negative unit clause.  More than max_iters checks ends with status 2. */
typedef void (*orc_check_fn)(const orc_prog *, uint32_t, orc_witness *);

static void orc_repair_by(const orc_prog *p, int mode, int grid_enabled, uint32_t max_iters, int strategy,
                          orc_check_fn check, orc_result *r) {
    memset(r, 0, sizeof(*r));
    const uint32_t n = orc_nslots(p);
    uint32_t grid = 0;
    for (uint32_t k = 0; k < n; k++)
        if (p->slot_level[k] == 1) grid |= 1u << k;
    const uint32_t forced = mode == 0 ? p->existing_mask : 0;
    uint32_t forbidden = grid_enabled ? 0 : grid;
    uint32_t clauses[ORC_MAX_CLAUSES + 2 * ORC_MAX_STMTS * ORC_MAX_STMTS];
    uint32_t n_cl = 0;
    uint32_t m = 0;
    int probe = 0;
    int status = 0;
    int greedy = strategy == 1;
    if (mode == 1) {
        m = p->existing_mask;
        probe = 1;
    } else {
        uint64_t wt;
        if (orc_solve(n, p->slot_weight, NULL, 0, p->neg, p->n_neg, forced, forbidden, &m, &wt)) {
            status = 1;
            goto done;
        }
    }
    for (;;) {
        if (r->iters == max_iters) {
            status = 2;
            break;
        }
        orc_witness w;
        check(p, m, &w);
        if (r->iters < ORC_MAX_TRAJ) r->traj[r->iters] = m;
        r->iters++;
        r->access_pairs += w.access_pairs;
        /* any witness row: one per executed instance (rows past the last
           instance are zero) */
        int any = w.diverge != 0;
        for (uint32_t i = 0; i < 32; i++)
            if (w.intra[i] | w.inter[i]) any = 1;
        if (!any && !probe) {
            if (greedy) {
                /* one exact query: is the clean greedy proposal also the minimum? */
                uint32_t xs;
                uint64_t wt;
                greedy = 0;
                if (!orc_solve(n, p->slot_weight, clauses, n_cl, p->neg, p->n_neg, forced, forbidden, &xs, &wt) &&
                    xs != m) {
                    m = xs;
                    continue;
                }
            }
            status = 0;
            r->mask = m;
            break;
        }
        probe = 0;
        n_cl = orc_clauses(p, &w, clauses, n_cl);
        forbidden |= w.diverge;
        uint64_t wt;
        if (greedy && !orc_greedy(n, p->slot_weight, clauses, n_cl, forced, forbidden, &m)) {
            int ok = 1;
            for (uint32_t c = 0; c < p->n_neg; c++)
                if ((m & p->neg[c]) == p->neg[c]) ok = 0;
            if (ok) continue;
        }
        if (orc_solve(n, p->slot_weight, clauses, n_cl, p->neg, p->n_neg, forced, forbidden, &m, &wt)) {
            status = 1;
            break;
        }
    }
done:
    r->status = status;
    if (status != 0) r->mask = 0;
    for (uint32_t k = 0; k < n; k++)
        if ((r->mask >> k) & 1u) r->weight += p->slot_weight[k];
    r->added = r->mask & ~p->existing_mask;
    r->removed = status == 0 ? (p->existing_mask & ~r->mask) : 0;
    r->n_clauses = n_cl;
    memcpy(r->clauses, clauses, n_cl * sizeof(uint32_t));
    r->forbidden = forbidden;
}

/* Algorithm 1 with Verify by the thread-pair enumeration (orc_check), or by
 * its word-grouped form (orc_check_words) for full-size launches. */
void orc_repair(const orc_prog *p, int mode, int grid_enabled, uint32_t max_iters, int strategy, orc_result *r) {
    orc_repair_by(p, mode, grid_enabled, max_iters, strategy, orc_check, r);
}

void orc_repair_words(const orc_prog *p, int mode, int grid_enabled, uint32_t max_iters, int strategy,
                      orc_result *r) {
    orc_repair_by(p, mode, grid_enabled, max_iters, strategy, orc_check_words, r);
}

/* Many independent programs on worker threads (programs are independent). */
typedef struct {
    const orc_prog *progs;
    const int32_t *modes;
    int grid_enabled, strategy;
    uint32_t max_iters;
    orc_check_fn check;
    orc_result *out;
    uint32_t n, stride, first;
} orc_job;

static void *orc_worker(void *arg) {
    orc_job *j = (orc_job *)arg;
    for (uint32_t i = j->first; i < j->n; i += j->stride)
        orc_repair_by(&j->progs[i], j->modes[i], j->grid_enabled, j->max_iters, j->strategy, j->check, &j->out[i]);
    return NULL;
}

static void orc_repair_batch_by(const orc_prog *progs, const int32_t *modes, uint32_t n, int grid_enabled,
                                uint32_t max_iters, int strategy, orc_check_fn check, orc_result *out,
                                uint32_t n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    orc_job jobs[256];
    for (uint32_t t = 0; t < n_threads; t++) {
        jobs[t] = (orc_job){progs, modes, grid_enabled, strategy, max_iters, check, out, n, n_threads, t};
        pthread_create(&th[t], NULL, orc_worker, &jobs[t]);
    }
    for (uint32_t t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
}

void orc_repair_batch(const orc_prog *progs, const int32_t *modes, uint32_t n, int grid_enabled,
                      uint32_t max_iters, int strategy, orc_result *out, uint32_t n_threads) {
    orc_repair_batch_by(progs, modes, n, grid_enabled, max_iters, strategy, orc_check, out, n_threads);
}

void orc_repair_batch_words(const orc_prog *progs, const int32_t *modes, uint32_t n, int grid_enabled,
                            uint32_t max_iters, int strategy, orc_result *out, uint32_t n_threads) {
    orc_repair_batch_by(progs, modes, n, grid_enabled, max_iters, strategy, orc_check_words, out, n_threads);
}

uint32_t orc_sizeof_result(void) { return (uint32_t)sizeof(orc_result); }
uint32_t orc_sizeof_prog(void) { return (uint32_t)sizeof(orc_prog); }
uint32_t orc_sizeof_witness(void) { return (uint32_t)sizeof(orc_witness); }
