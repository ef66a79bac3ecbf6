/* hisa.h -- C-ABI of the GB300 semi-naive Datalog engine (HISA relations).
 *
 * The engine evaluates Datalog programs over binary relations of uint32
 * values to their least fixpoint by semi-naive evaluation, as described in
 * "Optimizing Datalog for the GPU" (arXiv 2311.02206):
 *   - rules are Horn clauses over EDB (loaded) and IDB (derived) relations,
 *     evaluated until no new fact appears (Section 2);
 *   - every IDB relation keeps the versions new, delta and full; each
 *     iteration joins, populates delta = new \ full, merges delta into full
 *     and clears new (Section 5.1 and its evaluation-workflow figure);
 *   - relations are hash-indexed sorted arrays (Section 4): sorted,
 *     deduplicated tuples with an open-addressing index over the runs of
 *     equal join keys, range-probed by the binary join of Algorithm 3;
 *   - rules with three body atoms run as two binary joins through a
 *     temporarily materialized relation (Section 5.2);
 *   - buffers grow eagerly to full + k * delta (Section 5.3).
 * The library is the paper's "library for parallel relational algebra
 * kernels" (Section 1) in C form: declare relations, load EDB tuples, add
 * rules, run to the fixpoint, read IDB relations and per-iteration delta sizes.
 *
 * Conventions for every call:
 *   - A non-negative return is success (HISA_OK); a negative one is an error
 *     code from hisa_status below; hisa_last_error(ctx) gives a message.
 *   - "device" pointers are CUDA device pointers on the context's device;
 *     "host" pointers are ordinary host memory.  The caller owns every buffer
 *     it passes in; the library owns relation storage, which it allocates
 *     only through hisa_config.alloc/free (or cudaMallocAsync when NULL).
 *   - All GPU work is ordered on hisa_config.cuda_stream.  Calls that return
 *     data to the host synchronise that stream.
 *   - A context is not thread-safe; use one context per host thread.
 *   - No call traps or aborts: device-side failures (a bounded wait that ran
 *     out, an exhausted probe sequence) come back as error codes.
 */
#ifndef HISA_H_
#define HISA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t hisa_status;

#define HISA_OK 0
#define HISA_ERR_INVALID_ARG (-1)    /* null pointer, unknown relation, bad rule */
#define HISA_ERR_ARITY (-2)          /* column count does not match the relation */
#define HISA_ERR_OOM (-3)            /* allocation failed or HBM budget exceeded */
#define HISA_ERR_NOT_CONVERGED (-4)  /* max_iters iterations ran without a fixpoint */
#define HISA_ERR_DEVICE_TIMEOUT (-5) /* a bounded device-side wait expired */
#define HISA_ERR_CUDA (-6)           /* a CUDA runtime call failed (message in last_error) */
#define HISA_ERR_UNSUPPORTED (-7)    /* a rule shape this build does not evaluate */
#define HISA_ERR_STATE (-8)          /* call out of order (e.g. load after run) */
#define HISA_ERR_CAPACITY (-9)       /* a caller-provided output buffer is too small */

/* Allocator hooks: return a device pointer of at least `bytes` bytes usable on
 * `stream`, or NULL on failure; free releases one earlier allocation. */
typedef void* (*hisa_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*hisa_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

#define HISA_FLAG_GRAPH 1u        /* run iterations >= 2 as one CUDA graph with a device-side while loop */
#define HISA_FLAG_PHASE_TIMES 2u  /* record per-phase CUDA-event times (host-driven loop only) */
/* Keep full as two sorted levels where no rule probes it (it is only
 * differenced and merged: REACH, SG; not in batched runs): when new is small
 * against the large level it is differenced against it by sorted probes and
 * its delta merged into the small level; when new is large (|new| > |full|/2)
 * the small level is folded in and new is merged into the large level as
 * with one array.  The small level is merged into the large one when it
 * exceeds 1/8 of it and at the end of the run.  Same results; the per-
 * iteration merge no longer rewrites all of full (Section 5.1's merge, which
 * the paper measures at 42-45% of CSPA time).  Set by hisa_config_default. */
#define HISA_FLAG_LOG_FULL 4u
/* Never use the grouped join with bitmap deduplication.  By default, an IDB
 * relation whose only writer in iterations >= 2 is one binary join of its
 * delta with an EDB relation (REACH's recursive rule) is stored with the
 * column the join keeps first, and that join marks each kept value's results
 * in a shared-memory bitmap over the active domain (b <= 18 bits), writing
 * new already sorted and duplicate-free instead of sorting raw results
 * (Algorithm 3 and Section 4.2's sort + unique in one pass).  Same results;
 * not in batched runs. */
#define HISA_FLAG_NO_DENSE 8u
/* Always index join columns by the hashed run index of Section 4.3.  By
 * default a key domain of at most 2^20 values (domain bits + instance bits)
 * is indexed directly: first position of every key, the run of key k being
 * [first[k], first[k+1]) -- one probe instead of a slot walk. */
#define HISA_FLAG_HASH_INDEX 16u
/* Never gather Tmp grouped by its kept column.  By default, a two-step rule
 * variant H(x, y) <- A(x, a), delta(a, c), B(c, y) whose second step is a
 * grouped bitmap join (SG's recursive rule) builds its Tmp relation by
 * counting, per tuple of A in x order, the delta run it meets, and copying
 * those runs to their offsets: Tmp comes out grouped by x with no join
 * partition pass and no radix sort.  Also never run a one-step variant
 * H(x, y) <- A(x, z), delta(z, y) as an inverted grouped bitmap join (A
 * sorted by x the grouped outer, delta directly indexed by z the probed
 * side; domains of at most 2^14 values), which by default replaces its
 * raw results and their sort (CSPA's ValueFlow and ValueAlias rules).  Same
 * results; domain of at most 2^20 values, not in batched runs. */
#define HISA_FLAG_NO_CHAIN 32u
/* Never work a group of the grouped bitmap join in pull mode.  By default,
 * for an IDB relation written only by a one-step grouped bitmap join of its
 * delta with an EDB relation (REACH's recursive rule; domains of at most 2^16
 * values, not in batched runs), each group chooses per iteration between
 * marking the inner runs of its delta values (Algorithm 3's range probes,
 * "push") and "pull": every value o not yet derived for the group that has
 * inner tuples scans them, in the inner relation sorted by its other column,
 * until one joins a delta value -- the direction-optimizing traversal of
 * Beamer et al. (2012) applied per group.  A group pulls when the inner runs
 * its next delta would mark outnumber, several times over, the values it
 * could still derive.  Same results. */
#define HISA_FLAG_NO_PULL 64u
/* Keep an append-only full as sorted levels.  By default, when the program
 * has one IDB relation and it is written only by the grouped bitmap join
 * (REACH, SG) over a domain of 2^8 .. 2^16 values, its full is a bit matrix of
 * 2^(2b) bits (512 MB at b = 16), row = the kept column: the join's set
 * difference is an AND-NOT of the group's row, each iteration's new tuples
 * are ORed into it, and reads write its rows (transposed first when stored
 * column-swapped) in order.  Same results. */
#define HISA_FLAG_LEVELS 128u
/* Keep the grouped bitmap join for a program of REACH's shape.  By default,
 * when the one IDB relation R is defined by rules R(x, y) <- E(x, y) over
 * EDB relations and one recursive rule R(x, z) <- B(x, y), R(y, z) with B an
 * EDB relation, over a domain of at most 2^16 values (not in batched runs,
 * and none of HISA_FLAG_NO_DENSE, HISA_FLAG_NO_PULL, HISA_FLAG_LEVELS set),
 * R's full and delta are bit matrices over (first column, second column)
 * and an iteration ORs, for each tuple (x, y) of B, delta's row y into a new
 * row x, keeps the bits not in full's row x as delta' and ORs them into full
 * (Algorithm 3 and Section 5.1's difference and merge on 2^b tuples per
 * word operation).  Same results. */
#define HISA_FLAG_NO_BITJOIN 256u

typedef struct {
  hisa_alloc_fn alloc;      /* NULL: cudaMallocAsync from a private pool */
  hisa_free_fn free;
  void* user;               /* passed to alloc/free */
  void* cuda_stream;        /* cudaStream_t for all work; NULL: the legacy default stream */
  uint64_t hbm_budget_bytes;/* cap on library-owned device memory; 0 = no cap */
  float load_factor;        /* hash-index load factor; 0 = 0.8 (Section 6.2) */
  float ebm_k;              /* eager buffer growth factor k of Section 5.3; 0 = 2 */
  uint32_t max_iters;       /* iteration cap; 0 = 1,000,000 */
  uint32_t flags;           /* HISA_FLAG_*; default HISA_FLAG_LOG_FULL */
  int32_t device;           /* CUDA device ordinal; -1 = the current device */
  float pull_ratio;         /* pull mode switch point (HISA_FLAG_NO_PULL): a group pulls when the
                               inner runs its next delta would mark exceed pull_ratio times the
                               values it could still derive (plus the delta's size); 0 = 4 */
  uint32_t radix_items;     /* keys per thread of a radix-sort tile: 0 = 24 (32-bit codes) / 12 (64-bit);
                               16 / 8 take a smaller tile; other values = 0 */
  uint32_t dense_unit;      /* outer tuples per work unit of the grouped bitmap join (the join's work
                               split): 0 = 16 x the bitmap's words, within 256 .. 32768; 64 .. 2^20 */
} hisa_config;

typedef struct hisa_ctx hisa_ctx;

/* Fills `cfg` with the defaults above.  Never fails for a non-null cfg. */
hisa_status hisa_config_default(hisa_config* cfg);

/* Creates a context on cfg->device (the config is copied).  *out receives the
 * handle.  Errors: INVALID_ARG (null), CUDA. */
hisa_status hisa_create(const hisa_config* cfg, hisa_ctx** out);

/* Frees every library-owned buffer and the context.  NULL is accepted. */
hisa_status hisa_destroy(hisa_ctx* ctx);

/* Declares relation `name` (unique, <= 63 bytes) of the given arity (only 2
 * is evaluated by this build).  is_idb != 0 marks a derived relation, which
 * may appear in rule heads; EDB relations are loaded.  *rel_id receives its
 * id.  Errors: INVALID_ARG (duplicate name), ARITY (arity != 2), STATE. */
hisa_status hisa_declare_relation(hisa_ctx* ctx, const char* name, uint32_t arity, int is_idb,
                                  uint32_t* rel_id);

/* Appends n tuples to EDB relation rel_id from column arrays cols[0..arity)
 * (structure of arrays, uint32 each; device pointers if cols_on_device, else
 * host).  The library copies them; duplicates are dropped when the relation is
 * indexed (relations are sets, Section 2).  Allowed until the first hisa_run,
 * and again after hisa_reset_edb.  Errors: INVALID_ARG, STATE, OOM, CUDA. */
hisa_status hisa_load_tuples(hisa_ctx* ctx, uint32_t rel_id, const uint32_t* const* cols, uint64_t n,
                             int cols_on_device);

/* One atom: relation and the variable id bound to each column (variables are
 * small integers < 16; equal ids mean equal values). */
typedef struct {
  uint32_t rel;
  uint32_t var[2];
} hisa_atom;

/* head <- body[0], ..., body[n_body-1], neq[0][0] != neq[0][1], ...
 * 1 <= n_body <= 3; 0 <= n_neq <= 2.  Every head variable must occur in the
 * body.  Three-atom bodies are evaluated as two binary joins through a
 * temporarily materialized relation (Section 5.2), which must need at most two
 * columns. */
typedef struct {
  hisa_atom head;
  uint32_t n_body;
  hisa_atom body[3];
  uint32_t n_neq;
  uint32_t neq[2][2];
} hisa_rule;

/* Adds a rule.  Errors: INVALID_ARG (unknown relation, EDB head, unbound head
 * variable), UNSUPPORTED (cross products, more than two Tmp columns), STATE. */
hisa_status hisa_add_rule(hisa_ctx* ctx, const hisa_rule* rule);

typedef struct {
  uint32_t iterations;      /* K: iterations that derived a tuple (delta_K > 0) */
  uint32_t iterations_run;  /* iterations executed, including the final empty one */
  uint32_t regrows;         /* buffer growth events (Section 5.3) */
  uint32_t graph_launches;  /* CUDA graph launches of the iteration loop */
  double ms_total;          /* wall time of the run */
  double ms_edb;            /* EDB encode, sort, dedup and index build */
  double ms_join, ms_sort, ms_merge; /* per-phase times (HISA_FLAG_PHASE_TIMES) */
  uint64_t tuples_joined;   /* sum over iterations of |new| as materialized: before dedup,
                               except where the grouped bitmap join deduplicated (and
                               differenced) it inside the join (HISA_FLAG_NO_DENSE) */
  uint64_t peak_bytes;      /* peak library-owned device memory */
  uint64_t kernel_launches; /* kernels launched by the run (graph-launched ones included) */
} hisa_run_stats;

/* Evaluates all rules to the least fixpoint.  The EDB is encoded, sorted,
 * deduplicated and indexed first (once; again only after new loads).  IDB
 * relations start empty on every run.  `stats` may be NULL.  Errors:
 * NOT_CONVERGED, OOM, DEVICE_TIMEOUT, UNSUPPORTED, CUDA. */
hisa_status hisa_run(hisa_ctx* ctx, hisa_run_stats* stats);

/* Drops every EDB tuple so new ones can be loaded (rules are kept). */
hisa_status hisa_reset_edb(hisa_ctx* ctx);

/* Number of tuples of relation rel_id (IDB: after the last run). */
hisa_status hisa_relation_size(hisa_ctx* ctx, uint32_t rel_id, uint64_t* n);

/* Copies relation rel_id in ascending lexicographic order of (c0, c1) into
 * cols[0], cols[1] (each with room for `cap` values; device pointers if
 * cols_on_device).  *n receives the size.  Host columns that are page-locked
 * (cudaHostAlloc / pinned) are written over the host link by the device or,
 * for an IDB relation stored column-swapped as append-only levels over a
 * domain of at most 2^16 values, staged in library-owned device memory and
 * copied by the copy engine; other host columns are staged and copied.  Such
 * a column-swapped relation is read through a library-owned bit matrix of
 * 2^(2b) bits (512 MB at b = 16); the matrix and the staging columns stay
 * allocated for later reads and count against hbm_budget_bytes, and any later
 * allocation that would pass the budget, or that the allocator refuses,
 * releases them first.  Where the matrix does not fit, the relation is sorted
 * instead; where the staging does not fit, the device writes the page-locked
 * columns directly.  Errors: CAPACITY (cap < size; *n is still set),
 * INVALID_ARG, OOM, CUDA. */
hisa_status hisa_read_relation(hisa_ctx* ctx, uint32_t rel_id, uint32_t* const* cols, uint64_t cap,
                               uint64_t* n, int cols_on_device);

/* Per-iteration delta sizes |delta_1| .. |delta_K| of IDB relation rel_id from
 * the last run, into host array out[cap]; *n_iters receives K.  Errors:
 * CAPACITY (cap < K; the first cap values are written), INVALID_ARG. */
hisa_status hisa_delta_counts(hisa_ctx* ctx, uint32_t rel_id, uint64_t* out, uint32_t cap,
                              uint32_t* n_iters);

/* ---- batched instances (many independent fixpoints in one run) ----------------------
 *
 * Tuples loaded with hisa_load_instance carry an instance id (0 .. 2^k - 1):
 * every relation then holds the union of independent instances, each with its
 * own EDB, and one run evaluates all of them at once (codes carry the instance
 * id above the two columns, so joins never cross instances).  Plain
 * hisa_load_tuples loads into instance 0.  Requires instance bits + domain
 * bits <= 32; the run is host-driven so that per-instance delta sizes can be
 * read back after every iteration. */
hisa_status hisa_load_instance(hisa_ctx* ctx, uint32_t rel_id, uint32_t instance, const uint32_t* const* cols,
                               uint64_t n, int cols_on_device);
/* Tuples of one instance of relation rel_id after the last run. */
hisa_status hisa_instance_size(hisa_ctx* ctx, uint32_t rel_id, uint32_t instance, uint64_t* n);
/* Copies one instance's tuples (ascending (c0, c1)) like hisa_read_relation. */
hisa_status hisa_read_instance(hisa_ctx* ctx, uint32_t rel_id, uint32_t instance, uint32_t* const* cols,
                               uint64_t cap, uint64_t* n, int cols_on_device);
/* |delta_1| .. |delta_K| of one instance (K = its last productive iteration). */
hisa_status hisa_instance_delta_counts(hisa_ctx* ctx, uint32_t rel_id, uint32_t instance, uint64_t* out,
                                       uint32_t cap, uint32_t* n_iters);

/* ---- serving: continuous batching of independent requests ---------------------------
 *
 * A request is one instance's EDB tuples for relation rel_id (host columns,
 * copied at submit).  hisa_serve_step admits pending requests at iteration
 * boundaries while instance slots are free and the estimated device memory of
 * the admitted instances stays within the budget, runs up to max_iterations
 * iterations of the shared fixpoint (admitted instances join it with their
 * non-recursive rules at the next iteration), and retires every instance whose
 * delta became empty: its tuples and delta sizes are copied to host memory and
 * its slot and tuples are released.  Results stay available until
 * hisa_serve_release.  The rules must be added before hisa_serve_open;
 * hisa_load_tuples / hisa_run are not used in a serving session. */
typedef struct {
  uint32_t admitted;    /* requests admitted in this call */
  uint32_t retired;     /* requests completed in this call */
  uint32_t active;      /* instances on the device after the call */
  uint32_t pending;     /* submitted, not yet admitted */
  uint32_t iterations;  /* iterations run by this call */
  /* host wall time of this call's phases, ms: admission (slot choice, EDB
   * re-staging and indexing), the iterations' kernels, the per-instance delta
   * sizes read back, retirement (finished instances' tuples copied aside),
   * compaction (retired instances' tuples removed from full).  With
   * HISA_FLAG_PHASE_TIMES each phase ends with a stream synchronisation, so
   * its device work is counted in it; otherwise device work is counted where
   * the host first waits for it. */
  double ms_admit, ms_iterate, ms_rows, ms_retire, ms_compact;
} hisa_serve_stats;
/* Fixes the session's limits: up to max_instances concurrent instances (a
 * power of two is best), EDB values <= max_value, estimated bytes of admitted
 * instances <= budget_bytes (0: no limit).  Errors: INVALID_ARG, STATE. */
hisa_status hisa_serve_open(hisa_ctx* ctx, uint32_t max_instances, uint32_t max_value, uint64_t budget_bytes);
hisa_status hisa_serve_submit(hisa_ctx* ctx, uint32_t rel_id, const uint32_t* const* cols, uint64_t n,
                              uint64_t* ticket);
hisa_status hisa_serve_step(hisa_ctx* ctx, uint32_t max_iterations, hisa_serve_stats* stats);
/* *done = 1 once the request's fixpoint is complete. */
hisa_status hisa_serve_poll(hisa_ctx* ctx, uint64_t ticket, int* done);
/* The tickets the most recent hisa_serve_step retired, in slot order, into
 * tickets[cap]; *n receives their number (tickets may be NULL to query it).
 * Lets a caller collect results without polling every outstanding ticket.
 * Errors: STATE (no serving session), CAPACITY (*n is still set). */
hisa_status hisa_serve_retired(hisa_ctx* ctx, uint64_t* tickets, uint32_t cap, uint32_t* n);
/* A completed request's tuples of IDB relation rel_id, ascending (c0, c1),
 * into cols[0], cols[1] (room for cap tuples; device pointers if
 * cols_on_device, else host; cols may be NULL to query sizes), *n receives
 * the size; its delta sizes go to the host array deltas[dcap], *n_iters
 * receives K.  Completed results stay in device memory until released.
 * Errors: STATE (not complete), CAPACITY (sizes are still set). */
hisa_status hisa_serve_result(hisa_ctx* ctx, uint64_t ticket, uint32_t rel_id, uint32_t* const* cols, uint64_t cap,
                              uint64_t* n, uint64_t* deltas, uint32_t dcap, uint32_t* n_iters, int cols_on_device);
/* Forgets a completed request and frees its stored result. */
hisa_status hisa_serve_release(hisa_ctx* ctx, uint64_t ticket);

/* Per-kernel accounting of the last run made with HISA_FLAG_PHASE_TIMES (the
 * loop is then host-driven and every launch is bracketed by CUDA events on the
 * context's stream).  One entry per kernel kind that ran: launches, summed
 * device time, and the algorithmic bytes those launches had to move (what the
 * step reads and writes at minimum, from the sizes of each iteration).
 * Iterations that were re-run after a buffer grew are not counted.  Up to cap
 * entries go to `out`; *n receives the number of kinds.  Errors: CAPACITY. */
typedef struct {
  char name[24];
  uint64_t launches;
  double ms;
  double bytes;
} hisa_kernel_stat;
hisa_status hisa_kernel_stats(hisa_ctx* ctx, hisa_kernel_stat* out, uint32_t cap, uint32_t* n);

/* Static text of a status code. */
const char* hisa_status_string(hisa_status s);

/* Message of the last error on this context ("" if none). */
const char* hisa_last_error(hisa_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* HISA_H_ */
