/*
 * pm.h -- C ABI of libpmgpu, a GB300 (sm_103a) implementation of the
 * population fitness evaluation and genetic algorithm of AlBdaiwi &
 * AboElFotoh, "A GPU-Based Genetic Algorithm for the P-Median Problem"
 * (arXiv:1610.10061).
 *
 * Problem (Section 1, Eqs. 1-3): n clients, m facilities, an n x m matrix of
 * non-negative distances d_ij and an integer 1 <= p < m; choose exactly p
 * open facilities minimising the sum over clients of the distance to the
 * nearest open facility.
 *
 * Conventions for every call:
 *  - Every call returns a pm_status; nothing is thrown across the ABI.
 *  - Facility ids are 0-based (the paper's Section 1 numbers them from 1).
 *  - A population is `pop` bitsets of W = ceil(m/32) uint32 words each,
 *    row-major (individual t occupies words [t*W, (t+1)*W)); facility j is
 *    open in individual t iff bit (j & 31) of word t*W + (j >> 5) is set.
 *    Bits at positions >= m must be 0.  This is the paper's chromosome of m
 *    bits (Section 4.1), true = open.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device
 *    work is enqueued on it; a call that returns results in host memory
 *    synchronises that stream before returning.
 *  - The library never frees or retains caller buffers.  Objects it returns
 *    (pm_instance, pm_ga) are owned by the caller and released with the
 *    matching destroy call; they must not be used concurrently from two
 *    streams.
 *  - Pointers documented as "host or device" are classified with
 *    cudaPointerGetAttributes: device (or managed) memory is used in place,
 *    anything else is treated as host memory and staged through the
 *    library's own device buffers (the call then synchronises `stream`).
 *  - All device work runs in the library's own CUDA kernels; there is no CPU
 *    fallback.  A failed CUDA call is reported as PM_ERR_CUDA.
 *  - Device memory of the library's objects comes from a memory pool of the
 *    library's own per device.  Releasing an object waits, as cudaFree
 *    does, for the device's launches, then keeps up to 256 MiB of the freed
 *    memory mapped for later allocations (the rest goes back to the driver
 *    at the next synchronisation).  PM_POOL=0 in the environment allocates
 *    with cudaMalloc and cudaFree instead.
 */
#ifndef PM_H
#define PM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PM_API __attribute__((visibility("default")))
#else
#define PM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pm_status {
    PM_OK = 0,
    PM_ERR_INVALID_ARG = 1,   /* a size, pointer or parameter is out of range */
    PM_ERR_NEGATIVE_DIST = 2, /* some d_ij < 0 (the paper assumes d >= 0, Section 1) */
    PM_ERR_UNSUPPORTED = 3,   /* m > 65535 (facility ids are stored as uint16) */
    PM_ERR_MASK = 4,          /* checked evaluation: a bitset without exactly p open or with bits >= m */
    PM_ERR_CUDA = 5,          /* a CUDA runtime call failed */
    PM_ERR_OOM = 6,           /* device or host allocation failed */
    PM_ERR_TIMEOUT = 7        /* a bounded device-side wait gave up */
} pm_status;

/* Human-readable name of a status code (static string, never NULL). */
PM_API const char *pm_strerror(pm_status s);

/* ------------------------------------------------------------------------
 * Instances: the truncated ordering and increment tables.
 * ------------------------------------------------------------------------ */

typedef struct pm_instance pm_instance;

/*
 * pm_instance_create -- Section 2.1, Eq. 4 and the truncation argument after
 * Eq. 6.  Copies d (n x m int32, row-major, host or device memory) to the
 * device, checks d >= 0, and builds for each client i the ordering Pi'_i
 * (facility ids sorted by ascending d_ij, equal distances by ascending id)
 * and the increments Delta'_i (Delta'_i0 = smallest distance, then
 * consecutive differences), both truncated to L = m - p + 1 columns.  The
 * tables stay resident on `device` (Pi' uint16, Delta' int32, rows padded to
 * a stride of round_up(L, 32) elements).
 *   d       distance matrix; not retained.
 *   n, m, p 1 <= n, 1 <= p < m <= 65535.
 *   device  CUDA device ordinal; becomes the current device.
 *   out     receives the new instance.
 * Errors: PM_ERR_INVALID_ARG (sizes, NULL pointers), PM_ERR_UNSUPPORTED
 * (m > 65535), PM_ERR_NEGATIVE_DIST, PM_ERR_OOM, PM_ERR_CUDA.  Synchronises
 * `stream` (the distance check needs the device's answer).
 */
PM_API pm_status pm_instance_create(const int32_t *d, int64_t n, int64_t m, int64_t p, int device, void *stream,
                             pm_instance **out);

/*
 * pm_instance_create_ex -- pm_instance_create with flags.
 * PM_TABLES_CUMULATIVE: the instance keeps D'_i = the running sums of
 * Delta'_i (the sorted distances themselves) in place of Delta'_i.  The
 * scan's result is the same integer (by Eq. 4 the Delta' terms up to the
 * first open rank add up to the distance there); the evaluation reads that
 * value instead of summing, so a 32-rank step needs no warp prefix sum and
 * no carry.  No counterpart in the paper, which sums Delta' (Section 4.2).
 * pm_instance_tables still returns Delta'.  Other flags: PM_ERR_INVALID_ARG.
 */
#define PM_TABLES_CUMULATIVE 1u
PM_API pm_status pm_instance_create_ex(const int32_t *d, int64_t n, int64_t m, int64_t p, int device, void *stream,
                                       uint32_t flags, pm_instance **out);
/* The flags the instance was created with. */
PM_API pm_status pm_instance_flags(const pm_instance *inst, uint32_t *flags);

/* Release an instance and its device tables (NULL is accepted). */
PM_API pm_status pm_instance_destroy(pm_instance *inst);

/* Sizes of an instance: n, m, p, L = m-p+1, W = ceil(m/32) and the padded
 * row stride of the device tables (elements).  Any output may be NULL. */
PM_API pm_status pm_instance_info(const pm_instance *inst, int64_t *n, int64_t *m, int64_t *p, int64_t *L, int64_t *W,
                           int64_t *row_stride);

/*
 * pm_instance_tables -- copy Pi' (uint16) and Delta' (int32) into caller
 * buffers of n x L elements each (dense rows, no padding; host or device
 * memory).  Section 2.1, Example 1 shows both tables for a 5 x 4 instance.
 * Synchronises `stream`.
 */
PM_API pm_status pm_instance_tables(const pm_instance *inst, uint16_t *pi_out, int32_t *delta_out, void *stream);

/* ------------------------------------------------------------------------
 * Population fitness evaluation (the hot path).
 * ------------------------------------------------------------------------ */

/*
 * pm_eval_population -- Section 4.2 (function Fitness) and Eq. 6: for every
 * individual t and client i, walk Delta'_i in the order of Pi'_i, adding each
 * increment, and stop after the first rank whose facility is open in t; the
 * cost of t is the int64 sum over clients.  It equals the p-median objective
 * of Eqs. 1-3 for t's open set (Eq. 4 telescopes).
 *   masks   pop x W bitsets (layout above), host or device memory.
 *   pop     number of individuals, >= 0 (0 is a no-op).
 *   costs   pop int64 results, host or device memory.
 *   checked nonzero: first verify every bitset has exactly p open facilities
 *           and no bits >= m, returning PM_ERR_MASK (costs untouched) if
 *           not; this synchronises `stream`.  zero: bitsets are trusted; a
 *           bitset with fewer than p open facilities may yield a meaningless
 *           cost for that individual (never a fault).
 * Asynchronous when masks and costs are device memory and checked == 0.
 * Errors: PM_ERR_INVALID_ARG, PM_ERR_MASK, PM_ERR_OOM, PM_ERR_CUDA, and
 * PM_ERR_TIMEOUT when a bounded device-side wait of the scan gave up (the
 * costs are then unreliable).  A synchronous call (host costs, or checked)
 * reports it directly; an asynchronous one leaves it for pm_eval_status.
 * After reporting it the instance's scratch is reset, so later evaluations
 * are correct again.
 */
PM_API pm_status pm_eval_population(pm_instance *inst, const uint32_t *masks, int64_t pop, int64_t *costs, int checked,
                             void *stream);

/*
 * pm_eval_population_noalloc -- the same evaluation as pm_eval_population,
 * for callers that cannot allocate device memory.  The paper has no
 * counterpart; this entry point exists for the library's users.
 *
 * Some callers may not call cudaMalloc at the time they evaluate: a serving
 * process whose framework has already reserved nearly all device memory for
 * its own pool, a real-time loop that must not hit the allocator's locks and
 * implicit synchronisation, or a component that owns no memory budget of its
 * own.  This call allocates nothing: its scratch (the facility-major copy of
 * the population and the per-split partial sums) lives in one fixed
 * 8 MiB array compiled into the library, which every GPU that loads the
 * library keeps for the life of the process.
 *   masks, costs  device memory only (PM_ERR_INVALID_ARG for host pointers);
 *                 layouts as for pm_eval_population.
 *   pop           >= 0; the scratch needed is about pop * W * 4 bytes plus
 *                 8 bytes per individual per client split; if it exceeds the
 *                 8 MiB array the call returns PM_ERR_INVALID_ARG and launches
 *                 nothing.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  All
 * calls share the one array and each call overwrites it, so calls whose work
 * overlaps on the GPU (different streams, or different instances at the same
 * time) race and must be serialised by the caller.  Asynchronous on
 * `stream`.  Errors: PM_ERR_INVALID_ARG, PM_ERR_CUDA.  A device-side failure
 * (PM_ERR_TIMEOUT: a bounded wait of the scan gave up, the costs of that
 * call are unreliable) cannot be returned by this asynchronous call: the
 * array keeps it in an error word until pm_eval_status, which reads it
 * (synchronising) and clears it.
 */
PM_API pm_status pm_eval_population_noalloc(pm_instance *inst, const uint32_t *masks, int64_t pop, int64_t *costs,
                                            void *stream);

/*
 * pm_eval_status -- synchronise `stream` and report a device-side failure of
 * the asynchronous evaluations on inst since the last report: PM_ERR_TIMEOUT
 * when a bounded wait of the scan gave up in pm_eval_population,
 * pm_eval_columns or pm_eval_population_noalloc (whose fixed array belongs to
 * inst's device, so a failure there is reported for any instance on that
 * device), else PM_OK.  Reading clears the record and resets the scratch the
 * failed launch left behind.  No counterpart in the paper.  Errors:
 * PM_ERR_INVALID_ARG, PM_ERR_CUDA.
 */
PM_API pm_status pm_eval_status(pm_instance *inst, void *stream);

/*
 * The two launches of a column-kernel evaluation as separate calls (no
 * counterpart in the paper; Section 4.2's Fitness over a population kept in
 * facility-major form, the form the GA's operators write).
 *
 * pm_columns_layout -- the facility-major form the evaluation of `pop`
 * individuals on inst uses: *groups = G (tiles of 32 G individuals) and
 * *words = the uint32 words of the whole copy (both nullable).  Word
 * (tile * 32W + j) * G + g, for j < 32W with W = ceil(m / 32), has bit b set
 * iff individual tile * 32G + 32g + b (< pop) has facility j open; every
 * other bit is 0.  Errors: PM_ERR_INVALID_ARG; PM_ERR_UNSUPPORTED when this
 * size is evaluated by the row kernel (very large m, or a pinned or tuned
 * row shape), which has no such form.
 *
 * pm_population_columns -- writes that form of the bitsets `masks` (device,
 * as pm_eval_population) into `cols` (device, *words words from
 * pm_columns_layout for the same pop; caller-owned).  Asynchronous.
 *
 * pm_eval_columns -- costs (device, pop int64) of the population held in
 * `cols` in that form; the same costs as pm_eval_population of the bitsets.
 * Asynchronous.  Both: PM_ERR_INVALID_ARG for host pointers or bad sizes,
 * PM_ERR_UNSUPPORTED as pm_columns_layout, PM_ERR_OOM, PM_ERR_CUDA.
 */
PM_API pm_status pm_columns_layout(pm_instance *inst, int64_t pop, int32_t *groups, int64_t *words);
PM_API pm_status pm_population_columns(pm_instance *inst, const uint32_t *masks, int64_t pop, uint32_t *cols,
                                       void *stream);
PM_API pm_status pm_eval_columns(pm_instance *inst, const uint32_t *cols, int64_t pop, int64_t *costs, void *stream);

/*
 * pm_tune_eval -- autotune the tile shape of pm_eval_population for `pop`
 * individuals on this instance (no counterpart in the paper, whose Fitness
 * runs one thread per chromosome).  Candidates: facility-major tiles of
 * 32, 64 or 128 individuals per CTA (groups = 1, 2, 4; those whose tile fits
 * in shared memory), 8, 16 or 32 warps per CTA, and client splits around the
 * one-wave default (x1/2, x1, x2); the row kernel with bitsets and with byte
 * masks (one byte per facility, where 8 warps' masks fit in shared memory).  Each
 * candidate evaluates a uniformly random population (Floyd sampling, fixed
 * seed) once untimed, then five times eight back-to-back evaluations timed
 * with CUDA events on `stream` (the GA chains its evaluations the same way);
 * the fastest median is kept for this (instance, pop) and used by every later
 * evaluation of that size (pm_eval_population, pm_eval_population_noalloc
 * and GAs created afterwards).  chosen (nullable, host) receives it.
 * Synchronises `stream`.  Errors: PM_ERR_INVALID_ARG, PM_ERR_OOM, PM_ERR_CUDA.
 */
typedef struct pm_eval_shape {
    int32_t groups;   /* 32-individual groups per CTA tile (1, 2, 4); 0 = row kernel (bitsets in shared memory);
                         -1 = row kernel with byte masks (each bitset expanded to a byte per facility) */
    int32_t warps;    /* warps per CTA */
    int32_t splits;   /* client splits: work items per tile */
    int32_t grid;     /* CTAs launched (persistent over tiles x splits) */
    double ms;        /* median time of one evaluation with this shape */
    int32_t candidates; /* shapes timed */
    int32_t reserved;
} pm_eval_shape;

PM_API pm_status pm_tune_eval(pm_instance *inst, int64_t pop, void *stream, pm_eval_shape *chosen);

/*
 * pm_set_eval_shape -- use `shape` (groups, warps, splits; grid, ms,
 * candidates and reserved are ignored) for evaluations of `pop` individuals on inst
 * and for GAs created afterwards, in place of the heuristic or a tuned
 * shape (no counterpart in the paper: it pins a launch shape for
 * reproducible timing and tests).  groups 0 selects the row kernel, -1 the
 * row kernel with byte masks (PM_ERR_UNSUPPORTED where they do not fit); splits 0
 * the default split count.  The costs do not depend on the shape.  Errors:
 * PM_ERR_INVALID_ARG (bad values), PM_ERR_UNSUPPORTED (the shape does not
 * fit this instance's shared-memory budget).
 */
PM_API pm_status pm_set_eval_shape(pm_instance *inst, int64_t pop, const pm_eval_shape *shape);

/*
 * pm_selftest_bounded_wait -- failure-detection self-test (no counterpart in
 * the paper).  Launches one CTA that waits on an mbarrier nothing will
 * complete, with the bounded-poll exit every wait in this library uses; the
 * call returns the status the kernel recorded, PM_ERR_TIMEOUT when the bound
 * works, and leaves the context usable.  Synchronises `stream`.
 */
PM_API pm_status pm_selftest_bounded_wait(int device, void *stream);

/*
 * pm_debug_fail_alloc -- failure injection for tests (no counterpart in the
 * paper).  After `after` more successful device allocations by this library,
 * the next one fails on the host, without calling CUDA, and the call that
 * made it returns PM_ERR_OOM having launched nothing on that memory and
 * freed what it had obtained (one exception: a GA that cannot get the
 * buffers of the speculative mutation cycle runs the cycle try by try, with
 * the same results, instead of failing); the injection then disarms itself.
 * A negative `after` disarms it (the default).  pending (host, nullable)
 * receives the allocations that were still to succeed before the failure
 * armed until now, or -1 if none was armed or it has happened.
 * Process-wide; not meant for concurrent use.  Always PM_OK.
 */
PM_API pm_status pm_debug_fail_alloc(int64_t after, int64_t *pending);

/*
 * pm_debug_scan_timeout -- failure injection for tests (no counterpart in the
 * paper).  In the next `launches` launches of the column scan (by any call)
 * the odd-numbered CTAs issue no tile copy, so their bounded wait for the
 * tile runs out after a few thousand polls with nothing in flight; each of
 * them records PM_ERR_TIMEOUT in the launch's error word and returns, while
 * the even-numbered CTAs finish their work items and leave their split sums
 * behind, as a real timeout would.  A GA whose generations run in the
 * persistent kernel consumes an armed launch there instead: its CTA 0 leaves
 * at once, so the first grid barrier runs out (after 20 ms) in every other
 * CTA, which records PM_ERR_TIMEOUT and leaves.  No fault, trap or hang: this is the
 * exit every wait in the library takes.  launches <= 0 disarms it (the
 * default).  pending (host, nullable) receives the launches still armed until
 * now.  Process-wide; not meant for concurrent use.  Always PM_OK.
 */
PM_API pm_status pm_debug_scan_timeout(int64_t launches, int64_t *pending);

/* ------------------------------------------------------------------------
 * The Hammer-Beresnev polynomial (Section 2.1, Eq. 6, Example 1): a second
 * evaluator of the same costs, for small instances and for checking.
 * ------------------------------------------------------------------------ */

typedef struct pm_hbp pm_hbp;

/*
 * pm_hbp_create -- the reduced polynomial of inst on the device: client i
 * contributes Delta'_i[k] times the monomial over the facility set
 * {Pi'_i[0], ..., Pi'_i[k-1]} (k = 0 .. L-1; k = 0 is the constant term),
 * in the variables z_j = 1 - x_j; like monomials (equal sets from different
 * clients) are merged by adding coefficients and zero coefficients dropped,
 * as Example 1 reduces its 15 terms to 7.  The merge is exact: terms are
 * grouped by set size and a hash of the set, and a term joins a group only
 * after its set has been compared facility by facility with the group's.
 * Synchronises `stream`.  Errors: PM_ERR_INVALID_ARG, PM_ERR_UNSUPPORTED
 * (n * L above 2^26 terms or more than 8 GiB of monomials), PM_ERR_OOM,
 * PM_ERR_CUDA.
 */
PM_API pm_status pm_hbp_create(pm_instance *inst, void *stream, pm_hbp **out);
PM_API pm_status pm_hbp_destroy(pm_hbp *h);
/* Number of monomials after the merge and W = ceil(m/32) (either nullable). */
PM_API pm_status pm_hbp_info(const pm_hbp *h, int64_t *terms, int64_t *W);
/* The monomials, in no particular order: sets (terms x W uint32 bitsets,
 * facility j in the set iff bit (j & 31) of word j >> 5) and coeffs (terms
 * int64); host or device memory, either nullable.  Synchronises `stream`. */
PM_API pm_status pm_hbp_terms(const pm_hbp *h, uint32_t *sets, int64_t *coeffs, void *stream);
/*
 * pm_hbp_eval -- the polynomial's value for each of `pop` bitsets (masks,
 * device, the layout of pm_eval_population): the sum of the coefficients of
 * the monomials with no open facility.  It equals pm_eval_population's cost
 * (Eq. 4).  costs: device, pop int64.  Asynchronous.  Work: terms x W words
 * per individual.  Errors: PM_ERR_INVALID_ARG, PM_ERR_CUDA.
 */
PM_API pm_status pm_hbp_eval(pm_hbp *h, const uint32_t *masks, int64_t pop, int64_t *costs, void *stream);

/* ------------------------------------------------------------------------
 * The genetic algorithm (Sections 3.1, 3.2.2, 4.3-4.5) on the device.
 * ------------------------------------------------------------------------ */

typedef struct pm_ga_params {
    int64_t deme;         /* D, the paper's NT: a power of two >= 2 dividing pop; 0 = min(pop, 256) */
    int32_t xover_rounds; /* crossover rounds per generation; < 0 = lg D (Section 3.2.2, step 3) */
    int32_t mut_tries;    /* mutation tries per generation; < 0 = lg D (Section 3.2.2, step 5) */
    int64_t saturation;   /* S: stop when the best has not improved for S generations; 0 = off */
    uint32_t stream_id;   /* fourth word of every random-number counter (independent runs) */
    uint32_t flags;       /* PM_GA_TUNE: run pm_tune_eval for this population size at creation;
                             PM_GA_MIGRATE_TEAM: migration variant (ii) of Section 4.5;
                             PM_GA_INIT_COMBINADIC: Section 4.1's chromosome generation */
    struct pm_model *model;  /* learned swap proposal (see pm_model_create; the GA's creation builds the
                                instance's D' copy of pm_swap_stats); NULL = the paper's GA only */
    int32_t candidates;      /* learned try: closed facilities (by gain) paired with every open one; <= 0: 4 */
    int32_t reserved;        /* must be 0 */
} pm_ga_params;

#define PM_GA_TUNE 1u
/* Migration (Section 4.5).  Default, variant (i): from the second generation
 * on, slot 0 of deme b receives deme b's best of the previous generation.
 * PM_GA_MIGRATE_TEAM, variant (ii), where the bests of all demes travel
 * together into one deme: deme 0 receives them, deme b's best into slot b
 * (needs pop/deme <= deme, else PM_ERR_INVALID_ARG); every other individual
 * is drawn afresh. */
#define PM_GA_MIGRATE_TEAM 2u
/* Chromosome generation (Section 4.1).  Default: Floyd's sampling of a
 * uniform p-subset (p Philox draws).  PM_GA_INIT_COMBINADIC: the paper's
 * method -- a random rank below C(m, p), drawn exactly uniformly by
 * rejection on multi-word Philox integers (C(900, 90) is about 2^418, past
 * the 64-bit draw the section describes), then the combination of that rank
 * in lexicographic order.  Needs a device table of the binomials the
 * unranking meets ((p + 1) x (m - p + 1) entries of about log2(C(m, p))/32
 * words, built at creation; PM_ERR_UNSUPPORTED above 4 GiB or C(m, p) above
 * about 2^8100) and a single-instance GA. */
#define PM_GA_INIT_COMBINADIC 4u

typedef struct pm_ga pm_ga;
typedef struct pm_model pm_model;

/*
 * pm_ga_create -- allocate a GA of `pop` individuals (pop/D demes, the
 * paper's NB blocks of NT threads) on `inst`, seeded with `seed`.  No
 * generation runs yet.  params may be NULL (all defaults).
 * Random numbers: draw s of operation op for unit u in generation g is word
 * (s & 3) of Philox4x32-10(counter = (g, u, op*2^16 + s/4, stream_id),
 * key = (seed lo, seed hi)); U[0,N) = floor(u32 * N / 2^32).
 * Mutation (Section 4.4): every try mutates the individual as it stood when
 * the cycle began and an individual stops at its first strict improvement,
 * so for a single-instance GA whose evaluation uses the column kernel all
 * tries are built and evaluated in one pass (Q x pop candidates; falls back
 * to try by try if they do not fit in memory, or with PM_GA_SPEC=0 in the
 * environment).  Results and the evaluation count -- the tries each
 * individual reaches -- are the same either way.  With PM_GA_FUSED=1 in the
 * environment, such a GA with Floyd generation and no model runs all the
 * generations of a pm_ga_step call in one cooperative persistent launch,
 * its phases separated by grid-wide barriers (bounded: PM_ERR_TIMEOUT after
 * 4 s); the populations are the same.
 * Errors: PM_ERR_INVALID_ARG, PM_ERR_OOM, PM_ERR_CUDA; PM_ERR_UNSUPPORTED for
 * PM_GA_INIT_COMBINADIC beyond its limits.
 */
PM_API pm_status pm_ga_create(pm_instance *inst, uint64_t seed, int64_t pop, const pm_ga_params *params, void *stream,
                       pm_ga **out);

/*
 * pm_ga_step -- run up to `gens` more generations on the device (one CUDA
 * graph launch: for gens = 1 a plain graph of the generation's kernels, else
 * a conditional while-node around them, so the host is not involved between
 * generations).  A generation is: a fresh random
 * population (Floyd sampling) whose slot 0 of every deme receives that
 * deme's best of the previous generation (migration, Section 4.5 variant
 * (i)); evaluation; crossover rounds with butterfly partners t XOR
 * (D >> (1 + r mod lg D)), children replacing parents only when strictly
 * cheaper; mutation tries (circular or block shift, Section 4.4) on the
 * individuals not yet improved, the first strictly cheaper mutant replacing
 * the individual; deme best (lowest cost, then lowest index); global best
 * and saturation count.  Stops early when saturation is reached.
 *   trace  nullable; receives one int64 per generation actually run (the
 *          global best cost after it), host or device memory, `gens`
 *          entries of room per instance (a batched GA writes instance k's
 *          trace at [k * gens, (k+1) * gens)).  A host trace synchronises
 *          `stream`.
 * Errors: PM_ERR_INVALID_ARG, PM_ERR_OOM, PM_ERR_CUDA.
 */
PM_API pm_status pm_ga_step(pm_ga *ga, int64_t gens, int64_t *trace, void *stream);

/*
 * pm_ga_result -- synchronise `stream` and report the best solution so far
 * (of instance 0 for a batched GA; see pm_ga_instance_result).
 * Any output may be NULL.  best_mask: W words (host or device memory);
 * gens_run: generations run since creation; evals: fitness evaluations so
 * far (failed crossovers produce no child and are not counted; mutation
 * tries after an individual improved are not run and not counted).
 */
PM_API pm_status pm_ga_result(pm_ga *ga, int64_t *best_cost, uint32_t *best_mask, int64_t *gens_run, int64_t *evals,
                       void *stream);

/* pm_ga_population -- copy the population after the last generation: pop x W
 * masks and pop costs (either may be NULL; host or device memory); instance
 * 0 of a batched GA.  Synchronises `stream`. */
PM_API pm_status pm_ga_population(pm_ga *ga, uint32_t *masks, int64_t *costs, void *stream);

/* pm_ga_instance_result / pm_ga_instance_population -- the same for instance
 * k (0 <= k < number of instances) of a GA made by pm_batch_ga_create
 * (k = 0 for any GA).  Synchronise `stream`. */
PM_API pm_status pm_ga_instance_result(pm_ga *ga, int64_t k, int64_t *best_cost, uint32_t *best_mask,
                                       int64_t *gens_run, int64_t *evals, void *stream);
PM_API pm_status pm_ga_instance_population(pm_ga *ga, int64_t k, uint32_t *masks, int64_t *costs, void *stream);

/*
 * pm_ga_save / pm_ga_load -- checkpoint and resume.  The state between
 * generations is (seed, generation index, deme bests, global best,
 * saturation count, evaluation count); the random numbers are keyed by the
 * generation index, so a loaded GA continues exactly as the saved one would
 * have.  pm_ga_save: if buf is NULL, *len receives the size needed;
 * otherwise *len must be at least that size and receives the bytes written
 * (host memory).  Synchronises `stream`.  pm_ga_load creates a new GA on
 * `inst` (which must have the same n, m, p) from such a buffer.
 */
PM_API pm_status pm_ga_save(pm_ga *ga, void *buf, size_t *len, void *stream);
PM_API pm_status pm_ga_load(pm_instance *inst, const void *buf, size_t len, void *stream, pm_ga **out);

/* Release a GA and its device buffers (NULL is accepted). */
PM_API pm_status pm_ga_destroy(pm_ga *ga);

/*
 * pm_ga_info -- the resolved parameters of a GA (any output may be NULL):
 * pop, deme size D, crossover rounds, mutation tries, and the number of
 * library kernels one generation launches (the graph body), plus the number
 * launched once per pm_ga_step call of one generation (outside the body; a
 * graph-mode call of several generations also launches the loop's gate
 * kernel).  No device work.
 */
PM_API pm_status pm_ga_info(const pm_ga *ga, int64_t *pop, int64_t *deme, int32_t *xover_rounds, int32_t *mut_tries,
                            int64_t *kernels_per_generation, int64_t *kernels_per_step_call);

/*
 * pm_ga_run -- convenience: create, run `gens` generations, report, destroy.
 *   best_cost  receives the best cost; best_mask (W words, nullable, host or
 *   device); gens_run, evals nullable; trace nullable (gens entries).
 * Synchronises `stream`.
 */
PM_API pm_status pm_ga_run(pm_instance *inst, uint64_t seed, int64_t pop, int64_t gens, const pm_ga_params *params,
                    int64_t *best_cost, uint32_t *best_mask, int64_t *gens_run, int64_t *evals, int64_t *trace,
                    void *stream);

/* ------------------------------------------------------------------------
 * The learned swap proposal (no counterpart in the paper).  A small
 * perceptron (16 -> 128 -> 128 -> 1, ReLU; BF16 weights and activations on
 * the tensor cores, FP32 accumulation and master weights) scores swap moves
 * (close open facility j, open closed facility k) from exact first-order
 * statistics of the individual; a GA given a model (pm_ga_params.model)
 * adds one learned mutation try per generation before the shift tries: each
 * individual takes its best-scored swap among `candidates` x p candidates,
 * and the child is evaluated exactly and kept only if strictly cheaper, like
 * every other mutant.  The model never decides a cost.
 * ------------------------------------------------------------------------ */

/* Number of model parameters (FP32): W1 [16][128], b1 [128], W2 [128][128],
 * b2 [128], w3 [128], b3 [1], in that order, row = input unit. */
PM_API int64_t pm_model_num_params(void);

/* Create a model on `device` with a seeded He-style initialisation. */
PM_API pm_status pm_model_create(int device, uint64_t seed, pm_model **out);
PM_API pm_status pm_model_destroy(pm_model *model);

/* Set / get the FP32 master parameters (host or device, pm_model_num_params
 * floats).  Setting resets the Adam moments.  Synchronise `stream`. */
PM_API pm_status pm_model_set_params(pm_model *model, const float *params, void *stream);
PM_API pm_status pm_model_get_params(pm_model *model, float *params, void *stream);

/* Predictions y (rows FP32, device) for inputs x (rows x 16 BF16 bit patterns,
 * device, 16-byte aligned, else PM_ERR_INVALID_ARG).  Asynchronous. */
PM_API pm_status pm_model_forward(pm_model *model, const uint16_t *x, int64_t rows, float *y, void *stream);

/* Mean squared error of the predictions against targets t (rows FP32,
 * device) and its gradients (pm_model_num_params FP32, host or device,
 * nullable).  Synchronises `stream`. */
PM_API pm_status pm_model_grad(pm_model *model, const uint16_t *x, const float *t, int64_t rows, float *grads,
                               float *loss, void *stream);

/* One Adam step (Kingma & Ba 2015: beta1 0.9, beta2 0.999, eps 1e-8) on the
 * batch (x, t) with learning rate lr; *loss (nullable) receives the batch's
 * mean squared error before the step (then the call synchronises). */
PM_API pm_status pm_model_train_step(pm_model *model, const uint16_t *x, const float *t, int64_t rows, float lr,
                                     float *loss, void *stream);

/*
 * pm_model_train -- `epochs` passes of Adam (as pm_model_train_step) over the
 * rows (x: rows x 16 BF16 bit patterns, t: rows FP32 targets; device memory)
 * in mini-batches of `batch` rows (the last one of an epoch may be shorter),
 * the order drawn afresh each epoch on the device: position i of epoch e
 * holds row pi_e(i), pi_e a keyed permutation of [0, rows) -- a four-round
 * Feistel network on the smallest even number of bits b with 2^b >= rows
 * (halves of b/2 bits; round r maps (L, R) to (R, L ^ (f(R ^ K_r) mod
 * 2^(b/2))), f = MurmurHash3's 32-bit finaliser; the result is (L << b/2) | R),
 * applied again while the result is >= rows; the round keys K_0..K_3 are the
 * words of Philox4x32-10(counter (e, 0, 0x300 * 2^16, 0), key (seed lo, seed
 * hi)).  The training kernel reads its rows through the permutation (no copy
 * of the data).  losses (nullable; host or device): one FP32 per step, the
 * batch's mean squared error before its update, epochs * ceil(rows / batch)
 * entries; a host array synchronises `stream`, else the call is
 * asynchronous.  No counterpart in the paper.  Errors: PM_ERR_INVALID_ARG
 * (rows >= 2^31, host x or t, batch < 1, lr <= 0), PM_ERR_OOM, PM_ERR_CUDA.
 */
PM_API pm_status pm_model_train(pm_model *model, const uint16_t *x, const float *t, int64_t rows, int32_t epochs,
                                int64_t batch, float lr, uint64_t seed, float *losses, void *stream);

/*
 * pm_swap_stats -- per individual and facility (pop x m arrays, device):
 * gain[k] = the cost saved by opening closed facility k alone, cap[k] = the
 * clients it would take, loss[j] = the cost added by closing open facility j
 * alone (second-nearest minus nearest over j's clients, second-nearest taken
 * within the truncated table), assign[j] = the clients j serves.  From the
 * same walk over Pi' as the fitness (Section 4.2), continued to the second
 * open rank, reading the sorted distances D' (the running sums of Delta').
 * For an instance with Delta' tables the first call builds that D' copy
 * (n x row_stride int32, kept until pm_instance_destroy) on `stream` and
 * waits for it; PM_ERR_OOM if it cannot be allocated.  Asynchronous after
 * that.
 */
PM_API pm_status pm_swap_stats(pm_instance *inst, const uint32_t *masks, int64_t pop, int64_t *gain, int32_t *cap,
                               int64_t *loss, int32_t *assign, void *stream);

/*
 * pm_move_features -- the model's input rows (16 BF16 each; 8 features then
 * zeros) for given moves: moves[(t*C + c)*2 + 0] = j (open, to close),
 * [.. + 1] = k (closed, to open), C moves per individual; costs[t] the
 * individual's cost.  Features, with Z = max(cost/p, 1): loss_j/Z, gain_k/Z,
 * assign_j/(n/p), cap_k/(n/p), (loss_j-gain_k)/Z, log1p(loss_j/Z),
 * log1p(gain_k/Z), p/m.  All device memory.  Asynchronous.
 */
PM_API pm_status pm_move_features(pm_instance *inst, const int64_t *gain, const int32_t *cap, const int64_t *loss,
                                  const int32_t *assign, const int64_t *costs, const int32_t *moves, int64_t pop,
                                  int64_t C, uint16_t *x, void *stream);

/*
 * pm_log_moves -- training tuples (individual, move, exact cost change) for
 * the `pop` individuals in masks (device; costs[t] their exact costs):
 * `per` moves each, j uniform among the open facilities and k, with
 * probability 3/4, among the 4 closed facilities of largest gain, else
 * uniform among the closed ones (Philox4x32-10 keyed by seed).  Writes the
 * moves (pop x per x 2 int32), their feature rows x (pop x per x 16 BF16)
 * and targets t (pop x per FP32) = (exact cost after the swap - cost) / Z,
 * the swapped bitsets evaluated by the fitness kernels.  All device memory.
 * Allocates stream-ordered scratch; the first call on an instance with
 * Delta' tables also builds its D' copy (see pm_swap_stats).  Asynchronous.
 */
PM_API pm_status pm_log_moves(pm_instance *inst, const uint32_t *masks, const int64_t *costs, int64_t pop, int64_t per,
                              uint64_t seed, uint16_t *x, float *t, int32_t *moves, void *stream);

/* ------------------------------------------------------------------------
 * Batches: many instances of uneven (n, m, p) in one launch (no counterpart
 * in the paper, which solves one instance per run).
 * ------------------------------------------------------------------------ */

typedef struct pm_batch pm_batch;

/*
 * pm_batch_create -- group k instances (same device) for batched
 * evaluation and GAs.  The batch refers to the instances; the caller keeps
 * them alive until pm_batch_destroy.  Every instance's facility-major tile
 * must fit in shared memory (m up to about 56000), else PM_ERR_UNSUPPORTED.
 */
PM_API pm_status pm_batch_create(pm_instance *const *insts, int64_t k, pm_batch **out);
PM_API pm_status pm_batch_destroy(pm_batch *b);

/*
 * pm_batch_eval -- Section 4.2 for every individual of every instance in
 * one persistent launch (plus one transpose launch).  Instance j evaluates
 * pops[j] bitsets of W_j = ceil(m_j/32) words; masks holds the instances'
 * populations back to back (instance 0's pops[0] rows, then instance 1's,
 * ...), costs receives sum(pops) int64 values in the same order.  masks and
 * costs must be device memory; pops is host memory.  Work items (instance,
 * tile of 32G individuals, client split) are sized by an estimate of each
 * instance's scan work so that uneven instances share the GPU evenly.
 * Asynchronous.  Errors: PM_ERR_INVALID_ARG, PM_ERR_OOM, PM_ERR_CUDA.
 */
PM_API pm_status pm_batch_eval(pm_batch *b, const uint32_t *masks, const int64_t *pops, int64_t *costs,
                               void *stream);

/*
 * pm_batch_tune -- autotune the batched launch for these population sizes:
 * groups per tile (1, 2, 4), warps per CTA (16, 32) and work items per
 * resident CTA (2, 4, 8), each timed (median of three, CUDA events) on
 * uniformly random populations.  The fastest is used by later pm_batch_eval
 * calls with the same sizes and by batched GAs.  chosen->splits reports the
 * items per CTA.  Synchronises `stream`.
 */
PM_API pm_status pm_batch_tune(pm_batch *b, const int64_t *pops, void *stream, pm_eval_shape *chosen);

/*
 * pm_batch_ga_create -- one GA per instance of the batch, all with `pop`
 * individuals and the same params, run together: every generation is the
 * same sequence of kernels as pm_ga_create's, each launch covering all
 * instances.  Instance k draws its random numbers with stream id
 * params->stream_id + k, so its trajectory equals that of pm_ga_create on
 * the instance alone with that stream id.  An instance that reaches its
 * saturation limit stops while the others go on.  Use pm_ga_step,
 * pm_ga_instance_result, pm_ga_instance_population, pm_ga_info and
 * pm_ga_destroy on the result.  All instances must have p >= 2, or all
 * p = 1 (PM_ERR_UNSUPPORTED otherwise).  PM_GA_TUNE runs pm_batch_tune.
 * The mutation tries run one by one; with PM_GA_SPEC=1 in the environment
 * they are built and evaluated together for all instances (every
 * instance's Q x pop candidates in one launch and one scan) with the same
 * results.
 */
PM_API pm_status pm_batch_ga_create(pm_batch *b, uint64_t seed, int64_t pop, const pm_ga_params *params, void *stream,
                                    pm_ga **out);

#ifdef __cplusplus
}
#endif

#endif /* PM_H */
