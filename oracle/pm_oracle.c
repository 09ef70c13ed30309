/*
 * CPU oracle for the p-median genetic algorithm of AlBdaiwi & AboElFotoh,
 * "A GPU-Based Genetic Algorithm for the P-Median Problem" (arXiv:1610.10061).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into a separate shared
 * library that only the test-suite, the smoke check and the benchmark's CPU
 * baseline load.  It shares no code, header or table with the CUDA library
 * and neither one includes the other.  Everything here is plain, slow,
 * single-threaded C written so that each step can be checked against the
 * paper by eye.
 *
 * Conventions: facility ids are 0-based (the paper's Section 1 is 1-based,
 * Section 4.1 is 0-based); a chromosome is a bitset of m bits stored in
 * W = ceil(m/32) uint32 words, facility j open iff bit (j&31) of word (j>>5)
 * is set (Section 4.1: true = open).
 *
 * Functions and the passages they follow:
 *   oracle_tables        Section 2.1, Eq. 4 and the truncation argument
 *                        after Eq. 6 (Pi, Delta -> Pi', Delta').
 *   oracle_eval_direct   Section 1, Eqs. 1-3 (cost of an open set = sum over
 *                        clients of the nearest open facility).  O1.
 *   oracle_eval_scan     Section 4.2, the Fitness function (scan Delta' in
 *                        Pi' order up to the first open facility).  O3.
 *   oracle_brute_force   Section 1, Eqs. 1-3 minimised over every p-subset
 *                        (lexicographic enumeration, O1's cost per subset).
 *   oracle_philox4x32_10 Philox4x32-10 from its published definition
 *                        (Salmon, Moraes, Dror, Shaw, SC'11); stands in for
 *                        the paper's cuRAND generator (Section 3.2.1).
 *   oracle_floyd_*       Random p-subset (Floyd's sampling, Bentley & Floyd,
 *                        CACM 1987), the default chromosome generation (a
 *                        64-bit rank cannot index C(m,p)); the paper's own
 *                        combinadic generation of Section 4.1 is written with
 *                        exact integers in combinadic.py and reaches the GA
 *                        through oracle_ga_run's init_fn.
 *   oracle_crossover     Section 4.3.
 *   oracle_shift         Section 4.4 (circular and block shift).
 *   oracle_ga_run        Sections 3.1 and 3.2.2 (host steps 7-15, Evolve
 *                        steps 1-7) and Section 4.5 (migration variants (i)
 *                        and (ii)).
 *   oracle_swap_stats    Swap statistics of the learned proposal (no
 *                        counterpart in the paper): per facility, the exact
 *                        cost change of opening or closing it alone, from the
 *                        same Pi'/Delta' scan as Section 4.2.
 *
 * Parity status: tables, O1 and O3 are pinned by the paper's Example 1 and by
 * brute force; Philox by its published known-answer vectors; Floyd sampling
 * by exhaustive enumeration; the GA operators by invariants and hand-worked
 * cases from the prose of Sections 4.3-4.4; swap statistics by the exact
 * single-swap identities against O1.  oracle_ga_run: parity unpinned by the
 * paper -- its Figures 1-3 are missing, so the GA trajectory is pinned only by
 * those invariants and the migration-variant checks (its exact random-draw
 * discipline is this library's own reading, not the paper's).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_NO_OPEN 2
#define OR_ERR_OOM 3

/* ------------------------------------------------------------------------ */
/* Bitset helpers                                                           */
/* ------------------------------------------------------------------------ */

static int bit_get(const uint32_t *x, int64_t j) { return (int)((x[j >> 5] >> (j & 31)) & 1u); }

static void bit_set(uint32_t *x, int64_t j, int v)
{
    if (v)
        x[j >> 5] |= (1u << (j & 31));
    else
        x[j >> 5] &= ~(1u << (j & 31));
}

/* ------------------------------------------------------------------------ */
/* Section 2.1, Eq. 4: per client i, an ordering pi_i of the facilities with  */
/* d_{i,pi_i1} <= d_{i,pi_i2} <= ..., delta_i1 = d_{i,pi_i1} and              */
/* delta_ir = d_{i,pi_ir} - d_{i,pi_i(r-1)}.  Equal distances are ordered by */
/* ascending facility index (the paper only asks for <=; Example 1 is         */
/* consistent with this choice).  Only the first L columns are kept; L =     */
/* m - p + 1 gives Pi', Delta' (the last p-1 terms of Eq. 4 vanish because   */
/* any m-p+1 facilities contain an open one), L = m gives the full tables.   */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t d;
    int32_t j;
} oracle_pair;

static int oracle_pair_cmp(const void *a, const void *b)
{
    const oracle_pair *x = (const oracle_pair *)a, *y = (const oracle_pair *)b;
    if (x->d != y->d)
        return x->d < y->d ? -1 : 1;
    return x->j < y->j ? -1 : (x->j > y->j ? 1 : 0);
}

int oracle_tables(const int32_t *d, int64_t n, int64_t m, int64_t L, uint16_t *pi, int32_t *delta)
{
    if (n < 1 || m < 1 || m > 65536 || L < 1 || L > m)
        return OR_ERR_ARG;
    oracle_pair *row = (oracle_pair *)malloc((size_t)m * sizeof(oracle_pair));
    if (!row)
        return OR_ERR_OOM;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < m; ++j) {
            row[j].d = d[i * m + j];
            row[j].j = (int32_t)j;
        }
        qsort(row, (size_t)m, sizeof(oracle_pair), oracle_pair_cmp);
        for (int64_t r = 0; r < L; ++r) {
            pi[i * L + r] = (uint16_t)row[r].j;
            delta[i * L + r] = (r == 0) ? row[0].d : row[r].d - row[r - 1].d;
        }
    }
    free(row);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* O1.  Section 1, Eqs. 1-3: with open set O, client i is served by the      */
/* nearest open facility; the cost is the sum of those distances.            */
/* ------------------------------------------------------------------------ */

int oracle_eval_direct(const int32_t *d, int64_t n, int64_t m, const uint32_t *masks, int64_t W, int64_t P,
                       int64_t *costs)
{
    for (int64_t t = 0; t < P; ++t) {
        const uint32_t *x = masks + t * W;
        int64_t total = 0;
        for (int64_t i = 0; i < n; ++i) {
            int64_t best = -1;
            for (int64_t j = 0; j < m; ++j) {
                if (bit_get(x, j) && (best < 0 || d[i * m + j] < best))
                    best = d[i * m + j];
            }
            if (best < 0)
                return OR_ERR_NO_OPEN;
            total += best;
        }
        costs[t] = total;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Brute force.  Section 1, Eqs. 1-3 minimised by enumeration: every         */
/* p-subset whose smallest facility lies in [lo, hi), visited in             */
/* lexicographic order, costed by O1's definition (each client's nearest     */
/* facility of the subset, summed).  Ties keep the lexicographically first   */
/* subset.  best_set receives the p facility ids of the best subset in       */
/* ascending order.  Splitting [0, m - p + 1) into ranges lets callers run   */
/* ranges on several host threads and keep the smallest (cost, subset).      */
/* ------------------------------------------------------------------------ */

int oracle_brute_force(const int32_t *d, int64_t n, int64_t m, int64_t p, int64_t lo, int64_t hi, int64_t *best_cost,
                       int32_t *best_set)
{
    if (n < 1 || p < 1 || p > m || lo < 0 || hi > m - p + 1 || lo >= hi)
        return OR_ERR_ARG;
    int64_t *s = (int64_t *)malloc((size_t)p * sizeof(int64_t));
    if (!s)
        return OR_ERR_OOM;
    for (int64_t k = 0; k < p; ++k)
        s[k] = lo + k;  /* the first subset whose smallest facility is lo */
    *best_cost = -1;
    while (s[0] < hi) {
        int64_t total = 0;
        for (int64_t i = 0; i < n; ++i) {
            int32_t nearest = d[i * m + s[0]];
            for (int64_t k = 1; k < p; ++k)
                if (d[i * m + s[k]] < nearest)
                    nearest = d[i * m + s[k]];
            total += nearest;
        }
        if (*best_cost < 0 || total < *best_cost) {
            *best_cost = total;
            for (int64_t k = 0; k < p; ++k)
                best_set[k] = (int32_t)s[k];
        }
        /* the next subset in lexicographic order: raise the last element that can still rise, then make the
           elements after it consecutive */
        int64_t k = p - 1;
        while (k >= 0 && s[k] == m - p + k)
            --k;
        if (k < 0)
            break;
        s[k] += 1;
        for (int64_t q = k + 1; q < p; ++q)
            s[q] = s[q - 1] + 1;
    }
    free(s);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* O3.  Section 4.2, function Fitness: for each client, walk the client's    */
/* row of Delta' in the order of Pi', adding each increment, and stop after  */
/* the first rank whose facility is open.  The sum over clients is the       */
/* fitness (the value of Eq. 6).  ksum (optional) receives the total number  */
/* of ranks visited, the work of the scan.                                   */
/* ------------------------------------------------------------------------ */

int oracle_eval_scan(const uint16_t *pi, const int32_t *delta, int64_t n, int64_t L, const uint32_t *masks, int64_t W,
                     int64_t P, int64_t *costs, int64_t *ksum)
{
    int64_t visited = 0;
    for (int64_t t = 0; t < P; ++t) {
        const uint32_t *x = masks + t * W;
        int64_t fitness = 0;
        for (int64_t i = 0; i < n; ++i) {
            int64_t s = 0;
            for (;;) {
                if (s == L)
                    return OR_ERR_NO_OPEN; /* fewer than m-L+1 open facilities */
                fitness += delta[i * L + s];
                if (bit_get(x, pi[i * L + s]))
                    break;
                ++s;
            }
            visited += s + 1;
        }
        costs[t] = fitness;
    }
    if (ksum)
        *ksum = visited;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11).  One round maps counter (c0..c3)    */
/* with key (k0,k1) to (hi(B*c2)^c1^k0, lo(B*c2), hi(A*c0)^c3^k1, lo(A*c0)), */
/* A = 0xD2511F53, B = 0xCD9E8D57; the key is advanced by the Weyl           */
/* constants (0x9E3779B9, 0xBB67AE85) between rounds.  Ten rounds.           */
/* ------------------------------------------------------------------------ */

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prodA = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prodB = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(prodB >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)prodB;
        uint32_t n2 = (uint32_t)(prodA >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)prodA;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/*
 * Random-draw discipline of the GA (this library's reading; the paper uses
 * one cuRAND stream per thread and a separate host generator).  Draw number
 * `slot` of operation `op` for unit `unit` (an individual or a crossover
 * pair) in generation `gen` of the instance with id `inst` is word
 * (slot & 3) of Philox4x32-10 with
 *     counter = (gen, unit, op * 2^16 + slot / 4, inst),  key = (seed lo, seed hi).
 * A uniform integer in [0, N) is floor(u * N / 2^32).
 */
#define OP_INIT 0x001u
#define OP_XOVER 0x100u /* + crossover round */
#define OP_MUT 0x200u   /* + mutation try */

uint32_t oracle_draw(uint64_t seed, uint32_t gen, uint32_t unit, uint32_t op, uint32_t slot, uint32_t inst)
{
    uint32_t ctr[4] = {gen, unit, (op << 16) + (slot >> 2), inst};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[slot & 3];
}

uint32_t oracle_uniform(uint32_t u, uint32_t N) { return (uint32_t)(((uint64_t)u * (uint64_t)N) >> 32); }

/* ------------------------------------------------------------------------ */
/* Floyd's sampling of a uniform p-subset of {0..m-1}: for j = m-p .. m-1,   */
/* draw t uniform in [0, j]; add t if it is not yet chosen, else add j.      */
/* `draws` holds the p values t (already in range), in order.                */
/* ------------------------------------------------------------------------ */

void oracle_floyd_from_values(int64_t m, int64_t p, const uint32_t *draws, uint32_t *x)
{
    int64_t W = (m + 31) / 32;
    memset(x, 0, (size_t)W * sizeof(uint32_t));
    for (int64_t q = 0; q < p; ++q) {
        int64_t j = m - p + q;
        int64_t t = draws[q];
        if (!bit_get(x, t))
            bit_set(x, t, 1);
        else
            bit_set(x, j, 1);
    }
}

static void floyd_philox(int64_t m, int64_t p, uint64_t seed, uint32_t gen, uint32_t unit, uint32_t inst,
                         uint32_t *x, uint32_t *scratch)
{
    for (int64_t q = 0; q < p; ++q) {
        uint32_t N = (uint32_t)(m - p + q + 1);
        scratch[q] = oracle_uniform(oracle_draw(seed, gen, unit, OP_INIT, (uint32_t)q, inst), N);
    }
    oracle_floyd_from_values(m, p, scratch, x);
}

/* ------------------------------------------------------------------------ */
/* Section 4.3, crossover of C with its couple at start r1 exchanging r2 =   */
/* 2i genes.  Walk positions r1, r1+1, ... circularly (at most once around). */
/* Only positions where C and the couple differ count: the first i where C  */
/* is 0 become 1 and the first i where C is 1 become 0, so the child keeps   */
/* exactly p open.  Returns 1 and writes F if both counts reach i, else 0    */
/* (the operation fails and produces no offspring).                          */
/* ------------------------------------------------------------------------ */

int oracle_crossover(const uint32_t *C, const uint32_t *couple, int64_t m, int64_t r1, int64_t i, uint32_t *F)
{
    int64_t W = (m + 31) / 32;
    memcpy(F, C, (size_t)W * sizeof(uint32_t));
    int64_t c01 = 0, c10 = 0;
    for (int64_t step = 0; step < m && (c01 < i || c10 < i); ++step) {
        int64_t pos = (r1 + step) % m;
        int cb = bit_get(C, pos), pb = bit_get(couple, pos);
        if (cb == pb)
            continue;
        if (cb == 0 && c01 < i) {
            bit_set(F, pos, 1);
            ++c01;
        } else if (cb == 1 && c10 < i) {
            bit_set(F, pos, 0);
            ++c10;
        }
    }
    return (c01 == i && c10 == i) ? 1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Section 4.4, shift mutation.  The sub-sequence C[a .. a+len-1] is rotated */
/* (a = 0, len = m for the circular shift; a <= b, len = b-a+1 for a block   */
/* shift).  Left by k: F[a+j] = C[a + (j+k) mod len]; right by k is left by  */
/* len-k.  Positions outside the sub-sequence are copied.                    */
/* ------------------------------------------------------------------------ */

void oracle_shift(const uint32_t *C, int64_t m, int64_t a, int64_t len, int64_t k, int right, uint32_t *F)
{
    int64_t W = (m + 31) / 32;
    memcpy(F, C, (size_t)W * sizeof(uint32_t));
    int64_t kl = right ? (len - k) % len : k % len;
    for (int64_t j = 0; j < len; ++j)
        bit_set(F, a + j, bit_get(C, a + (j + kl) % len));
}

/* Mutation parameters for one try (this library's reading of Section 4.4;
 * the paper leaves the distributions open).  Draws 0..4 of op OP_MUT+q:
 *   draw0 -> kind: 0 circular, 1 block (probability 1/2 each)
 *   draw1 -> direction: 0 left, 1 right (probability 1/2 each)
 *   circular: a = 0, len = m, k = 1 + U[0, m-1) from draw2
 *   block: x = U[0,m) from draw2, y = U[0,m-1) from draw3, y += (y >= x);
 *          a = min(x,y), b = max(x,y), len = b-a+1, k = 1 + U[0, b-a) from draw4
 */
void oracle_mutation_params(uint64_t seed, uint32_t gen, uint32_t unit, uint32_t q, uint32_t inst, int64_t m,
                            int64_t *a, int64_t *len, int64_t *k, int *right)
{
    uint32_t op = OP_MUT + q;
    uint32_t kind = oracle_uniform(oracle_draw(seed, gen, unit, op, 0, inst), 2);
    *right = (int)oracle_uniform(oracle_draw(seed, gen, unit, op, 1, inst), 2);
    if (kind == 0) {
        *a = 0;
        *len = m;
        *k = 1 + oracle_uniform(oracle_draw(seed, gen, unit, op, 2, inst), (uint32_t)(m - 1));
    } else {
        int64_t x = oracle_uniform(oracle_draw(seed, gen, unit, op, 2, inst), (uint32_t)m);
        int64_t y = oracle_uniform(oracle_draw(seed, gen, unit, op, 3, inst), (uint32_t)(m - 1));
        if (y >= x)
            ++y;
        int64_t lo = x < y ? x : y, hi = x < y ? y : x;
        *a = lo;
        *len = hi - lo + 1;
        *k = 1 + oracle_uniform(oracle_draw(seed, gen, unit, op, 4, inst), (uint32_t)(hi - lo));
    }
}

/* Crossover parameters for the pair whose lower member is `pair` in round r
 * (Section 4.3: one member draws and shares): r1 = U[0,m) from draw0,
 * i = 1 + U[0, floor(p/2)) from draw1. */
void oracle_crossover_params(uint64_t seed, uint32_t gen, uint32_t pair, uint32_t r, uint32_t inst, int64_t m,
                             int64_t p, int64_t *r1, int64_t *i)
{
    uint32_t op = OP_XOVER + r;
    *r1 = oracle_uniform(oracle_draw(seed, gen, pair, op, 0, inst), (uint32_t)m);
    *i = 1 + oracle_uniform(oracle_draw(seed, gen, pair, op, 1, inst), (uint32_t)(p / 2));
}

/* ------------------------------------------------------------------------ */
/* The GA, Sections 3.1, 3.2.2, 4.5.  P individuals in demes of D (the       */
/* paper's NB blocks of NT threads).  One generation = one Evolve call:      */
/*   host steps 7/11/15: fresh random population; for g > 0 slot 0 of each   */
/*       deme receives that deme's best of generation g-1 (variant (i));     */
/*   Evolve 1: evaluate every individual;                                    */
/*   Evolve 3: crossover rounds r = 0..R-1 with partner t XOR (D >> (1 +     */
/*       r mod lg D)); round r reads the population as it was at the start  */
/*       of the round; a child replaces its parent iff strictly cheaper;    */
/*   Evolve 5: mutation tries q = 0..Q-1 on individuals not yet enhanced;    */
/*       the first strictly cheaper mutant replaces the individual;         */
/*   Evolve 7-8: deme best = lexicographic min of (cost, index);             */
/*   host steps 13-14: global best (replaced only on strict improvement);   */
/*       stop after `gens` generations or when the best has not improved    */
/*       for S generations (S = 0: no saturation stop).                      */
/* State for resuming lives in the caller's arrays: deme_best (P/D x W),    */
/* deme_cost (P/D), best (W), scalars[0..3] = best_cost, sat, evals, next g. */
/* pop_out (optional, gens x P x W) and cost_out (gens x P) receive the     */
/* population after every generation; trace (optional, gens) the best cost. */
/* ------------------------------------------------------------------------ */

typedef struct {
    const uint16_t *pi;
    const int32_t *delta;
    int64_t n, m, p, L, W;
} ga_inst;

static int64_t ga_fitness(const ga_inst *I, const uint32_t *x, int *err)
{
    int64_t c = 0;
    if (oracle_eval_scan(I->pi, I->delta, I->n, I->L, x, I->W, 1, &c, NULL) != OR_OK)
        *err = OR_ERR_NO_OPEN;
    return c;
}

static int ilog2_exact(int64_t v)
{
    int r = 0;
    while ((1LL << r) < v)
        ++r;
    return ((1LL << r) == v) ? r : -1;
}

/* Chromosome generation supplied by the caller (the combinadic draw of Section 4.1 is written with exact
   big integers in oracle/combinadic.py): writes the W words of individual `unit`'s fresh bitset. */
typedef void (*oracle_init_fn)(uint32_t gen, uint32_t unit, uint32_t *x);

/* An extra try between the crossover cycle and the mutation cycle, supplied by the caller (the learned swap
   proposal, which the paper does not have): it may replace individuals of X (P x W) and their costs c, marks
   the replaced ones in `enhanced` (the mutation cycle then skips them, as it skips those a mutant improved)
   and returns the number of evaluations it made. */
typedef int64_t (*oracle_extra_try_fn)(uint32_t gen, uint32_t *X, int64_t *c, unsigned char *enhanced);

int oracle_ga_run(const uint16_t *pi, const int32_t *delta, int64_t n, int64_t m, int64_t p, uint64_t seed,
                  uint32_t inst, int64_t P, int64_t D, int32_t xover_rounds, int32_t mut_tries, int64_t gens,
                  int64_t S, uint32_t *deme_best, int64_t *deme_cost, uint32_t *best, int64_t *scalars,
                  uint32_t *pop_out, int64_t *cost_out, int64_t *trace, int64_t *gens_run, int32_t team,
                  oracle_init_fn init_fn, oracle_extra_try_fn extra_fn)
{
    int lgD = ilog2_exact(D);
    if (n < 1 || p < 1 || p >= m || D < 2 || lgD < 0 || P < D || P % D != 0 || xover_rounds < 0 || mut_tries < 0)
        return OR_ERR_ARG;
    if (team && P / D > D)
        return OR_ERR_ARG;
    ga_inst I = {pi, delta, n, m, p, m - p + 1, (m + 31) / 32};
    const int64_t W = I.W, NB = P / D;
    uint32_t *X = (uint32_t *)calloc((size_t)(P * W), sizeof(uint32_t));
    uint32_t *Xs = (uint32_t *)calloc((size_t)(P * W), sizeof(uint32_t));
    int64_t *c = (int64_t *)calloc((size_t)P, sizeof(int64_t));
    int64_t *cs = (int64_t *)calloc((size_t)P, sizeof(int64_t));
    uint32_t *F = (uint32_t *)calloc((size_t)W, sizeof(uint32_t));
    uint32_t *tmp = (uint32_t *)calloc((size_t)(p > 1 ? p : 1), sizeof(uint32_t));
    unsigned char *enhanced = (unsigned char *)calloc((size_t)P, 1);
    int err = OR_OK;
    if (!X || !Xs || !c || !cs || !F || !tmp || !enhanced) {
        err = OR_ERR_OOM;
        goto done;
    }
    int64_t best_cost = scalars[0], sat = scalars[1], evals = scalars[2], g0 = scalars[3];
    int64_t ran = 0;
    for (int64_t gi = 0; gi < gens; ++gi) {
        const uint32_t g = (uint32_t)(g0 + gi);
        /* new population and migration (Section 4.5): variant (i) copies deme b's best of the previous
           generation into slot 0 of deme b; variant (ii) (team) copies every deme's best into deme 0,
           deme b's into slot b */
        for (int64_t t = 0; t < P; ++t) {
            if (g > 0 && !team && t % D == 0)
                memcpy(X + t * W, deme_best + (t / D) * W, (size_t)W * sizeof(uint32_t));
            else if (g > 0 && team && t < NB)
                memcpy(X + t * W, deme_best + t * W, (size_t)W * sizeof(uint32_t));
            else if (init_fn)
                init_fn(g, (uint32_t)t, X + t * W);
            else
                floyd_philox(m, p, seed, g, (uint32_t)t, inst, X + t * W, tmp);
        }
        /* Evolve step 1 */
        for (int64_t t = 0; t < P; ++t) {
            c[t] = ga_fitness(&I, X + t * W, &err);
            ++evals;
        }
        /* Evolve step 3: crossover cycle */
        for (int32_t r = 0; r < xover_rounds && p / 2 > 0; ++r) {
            int64_t stride = D >> (1 + (r % lgD));
            memcpy(Xs, X, (size_t)(P * W) * sizeof(uint32_t));
            memcpy(cs, c, (size_t)P * sizeof(int64_t));
            for (int64_t t = 0; t < P; ++t) {
                int64_t partner = t ^ stride;
                int64_t pair = t < partner ? t : partner;
                int64_t r1, ii;
                oracle_crossover_params(seed, g, (uint32_t)pair, (uint32_t)r, inst, m, p, &r1, &ii);
                if (!oracle_crossover(Xs + t * W, Xs + partner * W, m, r1, ii, F))
                    continue;
                int64_t cf = ga_fitness(&I, F, &err);
                ++evals;
                if (cf < cs[t]) {
                    memcpy(X + t * W, F, (size_t)W * sizeof(uint32_t));
                    c[t] = cf;
                }
            }
        }
        /* Evolve step 5: mutation cycle, first strict improvement stops; the caller's extra try comes first */
        memset(enhanced, 0, (size_t)P);
        if (extra_fn)
            evals += extra_fn(g, X, c, enhanced);
        for (int32_t q = 0; q < mut_tries; ++q) {
            for (int64_t t = 0; t < P; ++t) {
                if (enhanced[t])
                    continue;
                int64_t a, len, k;
                int right;
                oracle_mutation_params(seed, g, (uint32_t)t, (uint32_t)q, inst, m, &a, &len, &k, &right);
                oracle_shift(X + t * W, m, a, len, k, right, F);
                int64_t cf = ga_fitness(&I, F, &err);
                ++evals;
                if (cf < c[t]) {
                    memcpy(X + t * W, F, (size_t)W * sizeof(uint32_t));
                    c[t] = cf;
                    enhanced[t] = 1;
                }
            }
        }
        if (err != OR_OK)
            goto done;
        /* Evolve steps 7-8: block best, lowest index wins ties */
        for (int64_t b = 0; b < NB; ++b) {
            int64_t tb = b * D;
            for (int64_t t = b * D + 1; t < (b + 1) * D; ++t)
                if (c[t] < c[tb])
                    tb = t;
            memcpy(deme_best + b * W, X + tb * W, (size_t)W * sizeof(uint32_t));
            deme_cost[b] = c[tb];
        }
        /* host steps 13-14 */
        int64_t gb = 0;
        for (int64_t b = 1; b < NB; ++b)
            if (deme_cost[b] < deme_cost[gb])
                gb = b;
        if (best_cost < 0 || deme_cost[gb] < best_cost) {
            best_cost = deme_cost[gb];
            memcpy(best, deme_best + gb * W, (size_t)W * sizeof(uint32_t));
            sat = 0;
        } else {
            ++sat;
        }
        if (pop_out)
            memcpy(pop_out + gi * P * W, X, (size_t)(P * W) * sizeof(uint32_t));
        if (cost_out)
            memcpy(cost_out + gi * P, c, (size_t)P * sizeof(int64_t));
        if (trace)
            trace[gi] = best_cost;
        ++ran;
        if (S > 0 && sat >= S)
            break;
    }
    scalars[0] = best_cost;
    scalars[1] = sat;
    scalars[2] = evals;
    scalars[3] = g0 + ran;
    if (gens_run)
        *gens_run = ran;
done:
    free(X);
    free(Xs);
    free(c);
    free(cs);
    free(F);
    free(tmp);
    free(enhanced);
    return err;
}

/* ------------------------------------------------------------------------ */
/* Swap statistics of an individual (features of the learned swap proposal;  */
/* no counterpart in the paper).  For client i let r1 be the first rank whose */
/* facility is open (its facility f1, its distance D1 = the running sum of   */
/* Delta up to r1) and r2 the second such rank (distance D2; if no second    */
/* open facility lies within the L columns, D2 = the running sum up to the  */
/* last column).  Then, per facility (arrays of m entries per individual):  */
/*   gain[k]   = sum over clients i and ranks s < r1 with Pi[i][s] = k of   */
/*               D1 - (running sum up to s)   (what opening k alone saves)  */
/*   cap[k]    = number of such (i, s)        (clients k would capture)     */
/*   loss[j]   = sum over clients with f1 = j of D2 - D1                    */
/*               (what closing j alone costs)                               */
/*   assign[j] = number of clients with f1 = j                              */
/* ------------------------------------------------------------------------ */

int oracle_swap_stats(const uint16_t *pi, const int32_t *delta, int64_t n, int64_t L, int64_t m, const uint32_t *masks,
                      int64_t W, int64_t P, int64_t *gain, int32_t *cap, int64_t *loss, int32_t *assign)
{
    for (int64_t t = 0; t < P; ++t) {
        const uint32_t *x = masks + t * W;
        int64_t *g = gain + t * m;
        int32_t *c = cap + t * m;
        int64_t *l = loss + t * m;
        int32_t *a = assign + t * m;
        for (int64_t j = 0; j < m; ++j) {
            g[j] = 0;
            c[j] = 0;
            l[j] = 0;
            a[j] = 0;
        }
        for (int64_t i = 0; i < n; ++i) {
            const uint16_t *prow = pi + i * L;
            const int32_t *drow = delta + i * L;
            int64_t r1 = -1, r2 = -1, run = 0, d1 = 0, d2 = 0;
            for (int64_t s = 0; s < L; ++s) {
                run += drow[s];
                if (bit_get(x, prow[s])) {
                    if (r1 < 0) {
                        r1 = s;
                        d1 = run;
                    } else {
                        r2 = s;
                        d2 = run;
                        break;
                    }
                }
            }
            if (r1 < 0)
                return OR_ERR_NO_OPEN;
            if (r2 < 0)
                d2 = run; /* no second open facility within the table: the last column's distance */
            int64_t run2 = 0;
            for (int64_t s = 0; s < r1; ++s) {
                run2 += drow[s];
                g[prow[s]] += d1 - run2;
                c[prow[s]] += 1;
            }
            l[prow[r1]] += d2 - d1;
            a[prow[r1]] += 1;
        }
    }
    return OR_OK;
}
