/*
 * fj.h -- C ABI of libfj.so: Free Join plans executed over COLT indexes on a
 * GB300 (sm_103a).
 *
 * Paper: Wang, Willsey, Suciu, "Free Join: Unifying Worst-Case Optimal and
 * Traditional Joins" (arXiv 2301.10841).  The library takes what the paper's
 * entry point takes (Section 5.1): base relations stored column-wise and a
 * full conjunctive query (Section 2.1, Eq. 1), plus either a left-deep binary
 * plan to convert (Section 4.1) or a Free Join plan (Def. 3.5).  It builds
 * COLT levels lazily on the GPU (Section 4.2, Def. 4.2) and runs the plan
 * with vectorized, batch-at-a-time execution (Section 4.3) and the
 * fewest-keys dynamic cover (Section 4.4).
 *
 * Conventions shared by every call:
 *   - Values are int32 (signed comparison); row offsets are uint32, so a
 *     relation holds fewer than 2^32 - 1 rows; counts are uint64.
 *   - Variable ids are small integers in [0, FJ_MAX_VARS).
 *   - No call throws.  Every fallible call returns an fj_status; on failure
 *     fj_last_error() holds a one-line message for the calling thread.
 *   - "Device pointer" means memory of the context's GPU; "host pointer"
 *     means ordinary (or pinned) CPU memory.
 *   - Work is enqueued on the context's CUDA stream.  Calls that return
 *     results to the host synchronize that stream once before returning.
 */
#ifndef FJ_H_
#define FJ_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t fj_status;

#define FJ_OK 0
#define FJ_ERR_INVALID_ARG (-1)      /* bad pointer, size or id */
#define FJ_ERR_INVALID_PLAN (-2)     /* violates Def. 3.5 / Def. 3.7 */
#define FJ_ERR_OOM (-3)              /* device allocation failed */
#define FJ_ERR_OUTPUT_OVERFLOW (-4)  /* materialized output above list_limit */
#define FJ_ERR_COUNT_OVERFLOW (-5)   /* COUNT(*) does not fit in uint64 */
#define FJ_ERR_TIMEOUT (-6)          /* a bounded device wait ran out */
#define FJ_ERR_CUDA (-7)             /* a CUDA runtime call failed */
#define FJ_ERR_UNSUPPORTED (-8)      /* a shape this build does not handle */

#define FJ_MAX_VARS 32   /* distinct variables per query */
#define FJ_MAX_ATOMS 16  /* atoms per query */
#define FJ_MAX_NODES 16  /* nodes per Free Join plan */
#define FJ_MAX_SUB 16    /* subatoms per node */
#define FJ_MAX_ARITY 8   /* variables per atom */
#define FJ_MAX_PREDS 4   /* pushed-down predicates per atom */

typedef struct fj_ctx fj_ctx;
typedef struct fj_rel fj_rel;
typedef struct fj_prepared fj_prepared;
typedef struct fj_batch fj_batch;
typedef struct fj_model fj_model;

/* ------------------------------------------------------------------------ */
/* Context                                                                   */
/* ------------------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (for example torch.cuda.current_stream().cuda_stream) or NULL for the
 * legacy default stream; the library enqueues all of its work there and
 * never synchronizes the device.  The context owns a private stream-ordered
 * memory pool for COLT levels and intermediate batches.  *out receives the
 * handle; destroy it with fj_ctx_destroy.  Errors: FJ_ERR_INVALID_ARG,
 * FJ_ERR_CUDA. */
fj_status fj_ctx_create(int device, void* cuda_stream, fj_ctx** out);

/* Release every relation, prepared plan and buffer the context owns (their
 * handles become invalid: do not release them again).  Safe on NULL. */
void fj_ctx_destroy(fj_ctx* ctx);

/* Replace the stream work is enqueued on (same device).  FJ_ERR_INVALID_ARG
 * on a NULL context. */
fj_status fj_ctx_set_stream(fj_ctx* ctx, void* cuda_stream);

/* Last error message of the calling thread (never NULL; "" after success). */
const char* fj_last_error(void);

/* ------------------------------------------------------------------------ */
/* Relations (Section 2.1; Section 4.2: "each column is stored as a vector")  */
/* ------------------------------------------------------------------------ */

/* Register a column-stored relation whose `n_cols` int32 columns of `n_rows`
 * values each already live in device memory (`d_cols[j]` a device pointer,
 * 4-byte aligned).  The pointers are BORROWED: the caller keeps them alive
 * and unchanged until fj_release_relation; the library never writes or frees
 * them.  `name` is copied (may be NULL).  Errors: FJ_ERR_INVALID_ARG
 * (n_cols outside [1, FJ_MAX_ARITY*4], n_rows >= 2^32 - 1, NULL column). */
fj_status fj_load_relation(fj_ctx* ctx, const char* name, int n_cols,
                           const int32_t* const* d_cols, uint64_t n_rows,
                           fj_rel** out);

/* Same, but the columns are HOST pointers: the library allocates device
 * columns it owns and copies the data on the context's stream (page-locked
 * host memory makes the copy asynchronous and fastest).  The host buffers may
 * be reused once the call returns only after the stream is synchronized;
 * fj_execute_plan synchronizes it.  Errors as fj_load_relation, plus
 * FJ_ERR_OOM and FJ_ERR_CUDA. */
fj_status fj_load_relation_host(fj_ctx* ctx, const char* name, int n_cols,
                                const int32_t* const* h_cols, uint64_t n_rows,
                                fj_rel** out);

/* Forget a relation (and free its columns if the library owns them).  Any
 * prepared plan that references it must be freed first.  Safe on NULL. */
void fj_release_relation(fj_ctx* ctx, fj_rel* rel);

/* Number of rows of a relation (0 on NULL). */
uint64_t fj_relation_rows(const fj_rel* rel);

/* ------------------------------------------------------------------------ */
/* Queries and plans (Section 2.1 Eq. 1; Section 3.2 Def. 3.4-3.7)           */
/* ------------------------------------------------------------------------ */

/* Pushed-down selection on one atom column (Section 2.1: "selections are
 * pushed down to the base tables"): keep rows with  value(col) OP value. */
#define FJ_LT 0
#define FJ_LE 1
#define FJ_GT 2
#define FJ_GE 3
#define FJ_EQ 4
#define FJ_NE 5
typedef struct {
  int col;       /* index j into the atom's vars (0 <= j < n_vars) */
  int op;        /* FJ_LT .. FJ_NE */
  int32_t value;
} fj_pred;

/* An atom R(x1..xk): variable vars[j] is read from column cols[j] of the
 * relation (cols NULL means column j).  The variables of one atom are
 * distinct (Section 2.1).  A self-join is two atoms over the same relation;
 * each atom gets its own COLT (Section 2.1: "we simply rename one"). */
typedef struct {
  fj_rel* rel;
  int n_vars;
  const int* vars;
  const int* cols;
  int n_preds;
  const fj_pred* preds;
} fj_atom;

/* Q(head) :- atoms.  The query is full: head_vars lists every variable of the
 * atoms exactly once, in output column order (NULL head_vars means first
 * appearance across atoms in order). */
typedef struct {
  int n_atoms;
  const fj_atom* atoms;
  int n_head;
  const int* head_vars;
} fj_query;

/* A subatom R(y) with y a subset of the atom's variables (Def. 3.4).  The
 * variables may be listed in any order; the library uses the atom's column
 * order.  n_vars may be 0 (the empty subatom R(), which iterates the leaf
 * vector, i.e. the multiplicity). */
typedef struct {
  int atom;       /* index into fj_query.atoms */
  int n_vars;
  const int* vars;
} fj_subatom;

/* A node phi_k: its subatoms; sub[0] is the designated (static) cover. */
typedef struct {
  int n_sub;
  const fj_subatom* sub;
} fj_node;

/* A Free Join plan [phi_0 .. phi_{n-1}] (Def. 3.5).  When returned by the
 * library, every array it points to is owned by the plan and released by
 * fj_plan_free. */
typedef struct {
  int n_nodes;
  const fj_node* nodes;
} fj_plan;

/* Check that `plan` partitions every atom of `query` into subatoms
 * (Def. 3.5) and is valid (Def. 3.7: no two subatoms of one atom in a node;
 * every node has a cover, i.e. a subatom holding vs(phi_k) - avs(phi_k)),
 * and that sub[0] of every node is a cover.  Host only.  Returns FJ_OK or
 * FJ_ERR_INVALID_PLAN / FJ_ERR_INVALID_ARG with the reason in
 * fj_last_error(). */
fj_status fj_validate_plan(const fj_query* query, const fj_plan* plan);

/* binary2fj (Section 4.1, Fig. 9): convert the left-deep binary plan
 * [R_order[0], ..., R_order[n-1]] (atom indices, a permutation of
 * 0..n_atoms-1) into a Free Join plan; then, if apply_factor != 0, apply
 * factor (Fig. 10), moving probe subatoms one node earlier while their
 * variables are available there and the earlier node has no subatom of the
 * same atom, stopping at the first that cannot move.  Host only.  *out is
 * library-owned; release with fj_plan_free.  Errors: FJ_ERR_INVALID_ARG. */
fj_status fj_binary_to_free_plan(const fj_query* query, const int* order,
                                 int n, int apply_factor, fj_plan** out);

/* The Generic Join plan of a total variable order (Section 3.2, Eq. 3;
 * Section 2.3): one node per variable x of var_order (every variable of the
 * query once), holding the subatom R(x) of every atom R that contains x, in
 * atom order.  With FJ_FLAG_EAGER_ALL, the smallest batch and
 * FJ_FLAG_NO_FUSED_SCAN it is the paper's Generic Join baseline (Section
 * 5.1: all tries built eagerly, no vectorization).  Host only; *out is
 * library-owned (fj_plan_free).  Errors: FJ_ERR_INVALID_ARG,
 * FJ_ERR_UNSUPPORTED (more than FJ_MAX_NODES variables). */
fj_status fj_generic_join_plan(const fj_query* query, const int* var_order, int n,
                               fj_plan** out);

/* Release a plan returned by fj_binary_to_free_plan, fj_generic_join_plan or
 * fj_choose_plan.  Safe on NULL. */
void fj_plan_free(fj_plan* plan);

/* GHT schema of atom `atom` under `plan` (Section 3.3, build phase): the
 * subatoms of the atom in plan order give the levels y0..y(l-1), and an empty
 * last level is appended unless the last subatom is its node's cover.
 * Writes into level_sizes[0..*n_levels) the number of variables per level and
 * into vars_out the variables level by level (capacity FJ_MAX_ARITY*2 and
 * FJ_MAX_ARITY respectively suffice).  Host only. */
fj_status fj_ght_schema(const fj_query* query, const fj_plan* plan, int atom,
                        int* n_levels, int* level_sizes, int* vars_out);

/* Covers of node k (Def. 3.7): writes the indices into node.sub of every
 * subatom that holds vs(phi_k) - avs(phi_k); *n_covers receives how many
 * (capacity FJ_MAX_SUB).  Host only. */
fj_status fj_node_covers(const fj_query* query, const fj_plan* plan, int k,
                         int* n_covers, int* covers_out);

/* ------------------------------------------------------------------------ */
/* Execution (Section 3.3 Fig. 7; Section 4.2 COLT; Section 4.3 Fig. 13;      */
/* Section 4.4 dynamic cover)                                                */
/* ------------------------------------------------------------------------ */

#define FJ_COVER_STATIC 0   /* iterate sub[0] of every node */
#define FJ_COVER_FEWEST 1   /* per partial tuple, the cover with fewest keys
                               (an unforced COLT vector counts its length) */
#define FJ_COVER_LEARNED 2  /* the cover policy (STATIC or FEWEST) that the
                               chooser's network (opts.model, required)
                               predicts cheaper for this plan; decided once
                               at prepare time, reported in
                               FJ_CTR_COVER_POLICY */

#define FJ_OUT_MATERIALIZE 0  /* write every output tuple (bag) */
#define FJ_OUT_COUNT 1        /* COUNT(*) only */
#define FJ_OUT_COUNT_MIN 2    /* COUNT(*) and MIN of each min_vars[i] */
#define FJ_OUT_FACTORIZED 3   /* the bag as a union of products (Section 4.4:
                                 the result kept in trie form): one row per
                                 partial tuple that survives the last node
                                 the plan expands, holding its head
                                 variables bound so far, its multiplicity,
                                 and for every trailing single-subatom node
                                 the COLT vector it would iterate; see
                                 fj_prepared_factor_layout.  Prepared plans
                                 only (the vectors live in the plan's COLT
                                 storage): fj_execute_plan refuses it */

#define FJ_FLAG_EAGER_ALL 1u   /* force every COLT level before the join
                                  ("simple trie", paper Section 5.3) */
#define FJ_FLAG_EAGER_ROOT 2u  /* force every root level before the join
                                  ("simple lazy trie", Section 5.3) */
#define FJ_FLAG_TIMING 4u      /* record CUDA events around the library's
                                  kernels (on the context's stream) and report
                                  device times in the FJ_CTR_*_NS counters */
#define FJ_FLAG_NO_FUSED_SCAN 16u /* node 0 runs through the general node
                                  kernels even where the one-launch scan of a
                                  base-table cover applies (the vectorization
                                  ablations and the Generic Join baseline) */
#define FJ_FLAG_TEST_TIMEOUT 8u  /* test of the bounded waits: the root
                                  build's first grid barrier waits for one
                                  block more than the grid has, so every
                                  block gives up after its spin limit (about
                                  a second) and the execution fails with
                                  FJ_ERR_TIMEOUT; the context stays usable */

typedef struct {
  uint32_t batch_size;   /* cover tuples per vectorized batch (Fig. 13);
                            0 = default 1024; rounded to a supported size */
  float load_factor;     /* COLT hash-level occupancy target; 0 = 0.25.  Each
                            level's table is allocated for all of its atom's
                            rows at this load; a root level built in the
                            one-launch root build spans the whole allocation
                            (its occupancy is then at most this target) */
  int cover_policy;      /* FJ_COVER_* */
  int out_mode;          /* FJ_OUT_* */
  uint64_t list_limit;   /* MATERIALIZE: most rows to keep (0 = no limit) */
  int n_min_vars;        /* COUNT_MIN: variables to take MIN of */
  const int* min_vars;
  uint64_t spin_limit;   /* bound on every device-side wait, in polls (the
                            TMA stages of the node-0 scan, the grid barriers
                            of the root build); 0 = default (about a
                            second); a wait that runs out fails the
                            execution with FJ_ERR_TIMEOUT */
  const void* model;     /* FJ_COVER_LEARNED: an fj_model* (with its
                            feature scaler); else ignored */
  uint32_t flags;        /* FJ_FLAG_* */
} fj_exec_opts;

/* Counter slots of fj_result.counters. */
#define FJ_CTR_COVER_ITERS 0    /* cover elements iterated, all nodes */
#define FJ_CTR_PROBES 1         /* hash-level lookups issued */
#define FJ_CTR_PROBE_HITS 2     /* lookups that found their key */
#define FJ_CTR_ROOTS_BUILT 3    /* root levels built (atoms indexed) */
#define FJ_CTR_SUBTRIES_FORCED 4 /* child vectors turned into maps (level>=1) */
#define FJ_CTR_ROWS_REGROUPED 5 /* offsets moved by forcing, all levels */
#define FJ_CTR_SURVIVORS 6      /* partial tuples that reached the last node */
#define FJ_CTR_CHUNKS 7         /* expansion chunks launched */
#define FJ_CTR_KERNELS 8        /* kernels launched by this execution */
#define FJ_CTR_ATOM_BUILT_MASK 9  /* bit a set: atom a's root level was built */
#define FJ_CTR_EXPAND_NS 10     /* FJ_FLAG_TIMING: device time in k_expand */
#define FJ_CTR_EXPAND_LAUNCHES 11 /* FJ_FLAG_TIMING: k_expand launches timed */
#define FJ_CTR_BUILD_NS 12      /* FJ_FLAG_TIMING: device time forcing COLT */
#define FJ_CTR_SPAN_NS 13       /* FJ_FLAG_TIMING: first to last kernel */
#define FJ_CTR_COVER_POLICY 14  /* cover policy the execution used:
                                   FJ_COVER_STATIC or FJ_COVER_FEWEST (the
                                   one FJ_COVER_LEARNED chose) */

typedef struct {
  uint64_t count;                  /* COUNT(*) over the bag result */
  int32_t mins[FJ_MAX_VARS];       /* MIN of min_vars[i] (COUNT_MIN) */
  uint8_t min_valid[FJ_MAX_VARS];  /* 0: empty result (SQL NULL) */
  int n_head;                      /* columns of d_tuples */
  uint64_t n_out;                  /* rows in d_tuples */
  int32_t* d_tuples;               /* MATERIALIZE: device buffer, row-major
                                      n_out x n_head, head order, unsorted */
  int tuples_owned;                /* 1: d_tuples belongs to this result
                                      (fj_execute_plan) and is released by
                                      fj_result_free; 0: it belongs to the
                                      prepared plan (fj_execute_prepared) and
                                      stays valid until its next execution
                                      or fj_prepared_free */
  uint64_t counters[16];           /* FJ_CTR_* */
} fj_result;

/* One-shot execution: build what the plan needs and run it (lazily, from
 * scratch) and fill *out.  Enqueued on the context's stream; synchronizes it
 * once at the end to read the status, count and MINs.  `plan` must be valid
 * for `query` (checked: FJ_ERR_INVALID_PLAN).  Errors: FJ_ERR_INVALID_ARG,
 * FJ_ERR_INVALID_PLAN, FJ_ERR_OOM, FJ_ERR_OUTPUT_OVERFLOW (more rows than
 * list_limit; count is still exact and d_tuples holds list_limit rows),
 * FJ_ERR_COUNT_OVERFLOW, FJ_ERR_TIMEOUT, FJ_ERR_CUDA, FJ_ERR_UNSUPPORTED. */
fj_status fj_execute_plan(fj_ctx* ctx, const fj_query* query,
                          const fj_plan* plan, const fj_exec_opts* opts,
                          fj_result* out);

/* Prepared execution.  fj_prepare validates and compiles the plan once and
 * allocates COLT storage, with nothing built.  fj_build_colt_level forces
 * schema level `level` of atom `atom` for every entry of the level above it
 * (the eager ablations of Section 5.3; level 0 is the root hash map over the
 * selected base table); it fails with FJ_ERR_UNSUPPORTED for a level the
 * plan only iterates unless prepared with FJ_FLAG_EAGER_ALL.
 * fj_execute_prepared runs the join, reusing (and lazily extending) the
 * levels already built -- COLT is a cache of the base tables.
 * fj_reset_prepared drops every built level so the next execution starts
 * from the base tables again.  The query's and plan's arrays are copied;
 * relations must outlive the prepared plan. */
fj_status fj_prepare(fj_ctx* ctx, const fj_query* query, const fj_plan* plan,
                     const fj_exec_opts* opts, fj_prepared** out);
fj_status fj_build_colt_level(fj_prepared* prep, int atom, int level);
fj_status fj_execute_prepared(fj_prepared* prep, fj_result* out);
/* Enqueue an execution without waiting for it: returns once every kernel is
 * enqueued (plans whose later nodes need a host-side size read still wait for
 * those reads).  fj_prepared_result then synchronizes and fills *out.  The
 * pair is equivalent to fj_execute_prepared, except that a materialized
 * output larger than the prepared buffer fails with FJ_ERR_OUTPUT_OVERFLOW
 * instead of being retried. */
fj_status fj_execute_prepared_async(fj_prepared* prep);
fj_status fj_prepared_result(fj_prepared* prep, fj_result* out);
fj_status fj_reset_prepared(fj_prepared* prep);
void fj_prepared_free(fj_prepared* prep);

/* ------------------------------------------------------------------------ */
/* Batches of independent queries (no counterpart in the paper)             */
/* ------------------------------------------------------------------------ */

/* A batch runs n prepared queries as one unit of work: every execution
 * starts from scratch (COLT unbuilt, as after fj_reset_prepared), the queries
 * run back to back on the context's stream, and the host synchronizes once
 * for all n results.  Inside a batch no node's size is read back by the
 * host: each expanded node runs as one chunk as large as the next node's
 * input buffer, and a node whose input would not fit fails the execution
 * with FJ_ERR_UNSUPPORTED (run that query on its own).  Queries must have
 * COUNT or COUNT_MIN output and no EAGER flags (fj_batch_create returns
 * FJ_ERR_UNSUPPORTED naming the first that does not).
 *
 * FJ_BATCH_GRAPH: fj_batch_create captures the launches of the whole batch
 * once into a CUDA graph (on a private stream); each fj_batch_execute is then
 * one graph launch on the context's stream.  Without it, each execution
 * enqueues the launches again.
 *
 * The batch borrows the prepared queries: they must outlive it and must not
 * run on their own while a batch execution is in flight.  `results` holds n
 * fj_result, filled as fj_prepared_result would fill them. */
#define FJ_BATCH_GRAPH 1
#define FJ_BATCH_CONCURRENT 2  /* with FJ_BATCH_GRAPH: the graph holds eight
                                  independent branches (queries dealt round
                                  robin), which the GPU runs side by side;
                                  root levels are then built by the
                                  multi-launch force instead of the
                                  cooperative kernel */
fj_status fj_batch_create(fj_ctx* ctx, int n, fj_prepared* const* preps, int flags,
                          fj_batch** out);
fj_status fj_batch_execute(fj_batch* batch, fj_result* results);
/* fj_batch_execute in two halves: fj_batch_launch enqueues the batch (one
 * graph launch with FJ_BATCH_GRAPH) on the context's stream and returns;
 * fj_batch_results synchronizes the stream and fills `results`.  Queries
 * prepared with FJ_FLAG_TIMING report the device times of their kernels in
 * a batch too (in a graph, as event-record nodes). */
fj_status fj_batch_launch(fj_batch* batch);
fj_status fj_batch_results(fj_batch* batch, fj_result* results);
void fj_batch_free(fj_batch* batch);

/* ------------------------------------------------------------------------ */
/* Bushy plans (Section 2.2; Section 5.2: materialized intermediates)         */
/* ------------------------------------------------------------------------ */

/* A node of a binary join tree: a leaf (atom >= 0, an index into the
 * query's atoms) or a join (atom < 0) of nodes `left` and `right` (indices
 * into the node array).  The last node is the root; every atom is exactly
 * one leaf. */
typedef struct {
  int atom;
  int left;
  int right;
} fj_bushy_node;

/* Execute a bushy binary plan the way the paper runs one: its left spine is
 * a left-deep plan, converted by binary2fj and factored (Section 4.1), and
 * every right child that is a subtree rather than an atom is evaluated first
 * (recursively, the same way) and its bag of tuples materialized on the
 * device as a relation with one column per variable of the subtree (in
 * increasing variable id), which the spine then joins like a base table.
 * opts applies to the root's execution (its out_mode, MIN variables, batch
 * size, load factor, cover policy, flags); the subtrees materialize their
 * full bags.  The intermediates are released before returning.  The result
 * is the query's bag, as fj_execute_plan would give it; a materialized
 * result owns its tuples (fj_result_free).  Errors: as fj_execute_plan,
 * plus FJ_ERR_INVALID_ARG for a tree that is not a binary tree over every
 * atom, FJ_ERR_UNSUPPORTED for an intermediate of 2^32 - 1 rows or more. */
fj_status fj_execute_bushy(fj_ctx* ctx, const fj_query* query, const fj_bushy_node* nodes,
                           int n_nodes, const fj_exec_opts* opts, fj_result* out);

/* Layout of an FJ_OUT_FACTORIZED result of a prepared plan: each of its
 * n_out rows has *width int32 words -- the values of the *n_prefix head
 * variables prefix_vars[0..*n_prefix) (in head order; capacity
 * FJ_MAX_VARS), the row's multiplicity as two words (low first), and for
 * each of the *n_tails trailing nodes (in plan order; tail_atoms[t] their
 * atoms, capacity FJ_MAX_NODES) the first offset and the length of the
 * COLT vector of that atom the row reaches.  The bag the row stands for is
 * its prefix values, repeated multiplicity times, crossed with the base-table
 * rows of every tail vector (their values of the tail's variables).
 * Errors: FJ_ERR_INVALID_ARG. */
fj_status fj_prepared_factor_layout(const fj_prepared* prep, int* width, int* n_prefix,
                                    int* prefix_vars, int* n_tails, int* tail_atoms);

/* Expand the factorized result `res` (the plan's last execution; its COLT
 * vectors still in place) into res->count flat tuples in head order, written
 * row-major to the device buffer d_dst of dst_rows x n_head int32.  Tuples
 * come in factorized-row order; within a row the multiplicity copies vary
 * slowest and the last tail fastest.  Synchronizes the stream.  Errors:
 * FJ_ERR_INVALID_ARG (another result, or too small a buffer), FJ_ERR_OOM,
 * FJ_ERR_CUDA. */
fj_status fj_prepared_expand(fj_prepared* prep, const fj_result* res, int32_t* d_dst,
                             uint64_t dst_rows);

/* Copy a materialized result's rows (n_out x n_head int32) to `dst`, a
 * device pointer if dst_is_device != 0 else a host pointer.  Synchronizes the
 * stream.  FJ_ERR_INVALID_ARG if the result holds no tuples. */
fj_status fj_result_copy_tuples(fj_ctx* ctx, const fj_result* res, void* dst,
                                int dst_is_device);

/* Release the device buffer of a result (safe to call twice). */
void fj_result_free(fj_ctx* ctx, fj_result* res);

/* ------------------------------------------------------------------------ */
/* The chooser's network (no counterpart in the paper)                       */
/* ------------------------------------------------------------------------ */

/* A three-layer perceptron y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 with
 * float32 parameters, trained by plain gradient descent on the mean squared
 * error; the plan chooser uses it to predict the work of a candidate plan
 * from sampled degree histograms.  Its forward, backward and update kernels
 * run on the context's stream.  Parameters form one array: W1 (h1 x in_dim,
 * row-major), b1 (h1), W2 (h2 x h1), b2 (h2), W3 (1 x h2), b3 (1); they start
 * at zero and are set by the caller (fj_model_set_params).  Inputs are
 * device pointers to n x in_dim row-major float32 rows (n <= max_batch, else
 * FJ_ERR_INVALID_ARG); targets and outputs are n float32 on the device.
 * Errors: FJ_ERR_INVALID_ARG, FJ_ERR_OOM, FJ_ERR_CUDA, with the reason in
 * fj_model_last_error(). */
fj_status fj_model_create(fj_ctx* ctx, int in_dim, int h1, int h2, int max_batch,
                          fj_model** out);
size_t fj_model_n_params(const fj_model* model);
fj_status fj_model_set_params(fj_model* model, const float* host, size_t n);
fj_status fj_model_get_params(fj_model* model, float* host, size_t n);
/* Predictions for n rows into d_y (enqueued, not waited for). */
fj_status fj_model_forward(fj_model* model, const float* d_x, int n, float* d_y);
/* Gradient of the mean squared error (host, in the parameter layout) and
 * the loss, without changing the parameters.  Synchronizes. */
fj_status fj_model_gradients(fj_model* model, const float* d_x, const float* d_t, int n,
                             float* host_grads, float* host_loss);
/* One descent step: parameters -= lr * gradient; *host_loss (if not NULL)
 * receives the loss before the step (then synchronizes). */
fj_status fj_model_train_step(fj_model* model, const float* d_x, const float* d_t, int n,
                              float lr, float* host_loss);
/* Feature scaler of the model: the chooser standardizes each feature as
 * (x - mean[i]) / scale[i] before the forward pass (n = in_dim, scales > 0).
 * Host arrays, copied. */
fj_status fj_model_set_scaler(fj_model* model, const float* mean, const float* scale, size_t n);
/* Save the model (shape, parameters, scaler) to a file, and load one into a
 * new model on `ctx` with room for `max_batch` rows per forward pass.  The
 * file: 8 bytes "FJMLP001", int32 in_dim, h1, h2, has_scaler, the float32
 * parameters in the layout above, then in_dim means and in_dim scales when
 * has_scaler; little-endian.  Errors: FJ_ERR_INVALID_ARG (unreadable or
 * malformed file), FJ_ERR_OOM, FJ_ERR_CUDA. */
fj_status fj_model_save(fj_model* model, const char* path);
fj_status fj_model_load(fj_ctx* ctx, const char* path, int max_batch, fj_model** out);
const char* fj_model_last_error(void);
void fj_model_free(fj_model* model);

/* ------------------------------------------------------------------------ */
/* The learned plan chooser (no counterpart in the paper)                    */
/* ------------------------------------------------------------------------ */

/* A candidate plan is a left-deep join order, converted by binary2fj and
 * factored (Section 4.1), with a cover policy (FJ_COVER_STATIC or
 * FJ_COVER_FEWEST).  Its FJ_CHOOSER_IN_DIM features, in order: for each of
 * the order's first four atoms, log2(rows + 1) / 32 and the 32-bucket
 * sampled key-degree histogram (fj_degree_histogram, 1% sample, seed
 * 31 * atom + column index within the atom) of the column it joins on (the
 * first atom: its first variable shared with the second; the others: their
 * first variable already bound), zeros for missing positions; then
 * n_atoms / 8, n_vars / 32, 1 if the query is cyclic (sum of arities minus
 * the number of variables >= n_atoms), the constant 1, and 1 for
 * FJ_COVER_FEWEST (else 0).  The relations' columns must be device columns
 * (they are sampled on the GPU). */
#define FJ_CHOOSER_IN_DIM 137
/* Features of n_candidates candidates: candidate c is the order
 * orders[c * n_atoms .. (c + 1) * n_atoms) (every atom once) with
 * cover_policies[c]; host_out receives n_candidates x FJ_CHOOSER_IN_DIM
 * floats, row-major.  Each histogram is sampled once per call.
 * Synchronizes the context's stream.  Errors: FJ_ERR_INVALID_ARG,
 * FJ_ERR_OOM, FJ_ERR_CUDA, with the reason in fj_chooser_last_error(). */
fj_status fj_plan_features(fj_ctx* ctx, const fj_query* query, int n_candidates,
                           const int* orders, const int* cover_policies, float* host_out);
/* Choose a plan: the candidates are the declared order 0..n_atoms-1 and up
 * to max_candidates - 1 other left-deep orders whose prefixes are connected
 * (drawn without replacement by a SplitMix64 stream seeded with `seed`),
 * each with both cover policies; the network predicts each candidate's work
 * from its standardized features and the smallest prediction wins.  With
 * model == NULL the declared order with the static cover is returned (the
 * plain converted binary plan, the chooser's fallback).  *out_plan is
 * library-owned (fj_plan_free); *out_cover_policy receives the policy to
 * execute it with; out_order (n_atoms ints, may be NULL) the chosen order.
 * Every candidate gives the same result.  Errors: as fj_plan_features. */
fj_status fj_choose_plan(fj_ctx* ctx, const fj_query* query, const fj_model* model,
                         int max_candidates, uint64_t seed, fj_plan** out_plan,
                         int* out_cover_policy, int* out_order);
const char* fj_chooser_last_error(void);

/* Sampled key-degree histogram of one int32 device column (n < 2^31 rows),
 * the chooser's feature (no counterpart in the paper).  Row i is sampled
 * iff fmix32((i mod 2^32) xor seed) % mod == 0 (the 32-bit MurmurHash3
 * finalizer); a key counted c times among the m sampled rows has estimated
 * degree c n / m and lands in the largest bucket b < 32 with c n >= m 2^b;
 * host_hist (32 floats) receives the fraction of distinct sampled keys per
 * bucket (all zero when nothing is sampled).  Enqueued on the context's
 * stream and synchronized.  Errors: FJ_ERR_INVALID_ARG, FJ_ERR_OOM,
 * FJ_ERR_CUDA, with the reason in fj_stats_last_error(). */
fj_status fj_degree_histogram(fj_ctx* ctx, const int32_t* d_col, uint64_t n, uint32_t mod,
                              uint32_t seed, float* host_hist);
const char* fj_stats_last_error(void);

/* ------------------------------------------------------------------------ */
/* Join without allocation (no counterpart in the paper)                     */
/* ------------------------------------------------------------------------ */

/* The bag COUNT of the equi-join Q(x) :- R(x), S(x), computed without any
 * device allocation, for callers that cannot allocate on this path: code
 * running while a stream is captured into a CUDA graph, services holding a
 * fixed pre-reserved memory budget, or hosts that provide a stream but no
 * allocator.  The paper has no counterpart; fj_execute_plan computes the
 * same COUNT for the same query.
 *
 * d_r_key (n_r values) and d_s_key (n_s values) are int32 device columns; the
 * result is written to *d_count (a device uint64).  Work is enqueued on
 * `cuda_stream` (a cudaStream_t, NULL for the legacy default stream) of the
 * current device and not waited for.
 *
 * Scratch is a fixed 8 MiB array inside the library (held by every GPU that
 * loads it, until the process exits), so S may have at most 524288 rows:
 * larger inputs fail with FJ_ERR_INVALID_ARG before any GPU work.  The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress
 * with the device current); make that first call before any stream capture.
 * All calls share the array: each clears what it uses, and calls that
 * overlap on the GPU (other streams or threads) race.  A CUDA error already
 * pending when the call starts is reported as FJ_ERR_CUDA and left pending
 * (nothing is launched).  Errors: FJ_ERR_INVALID_ARG, FJ_ERR_CUDA, with the
 * reason in fj_noalloc_last_error(). */
fj_status fj_join2_count_noalloc(const int32_t* d_r_key, uint64_t n_r,
                                 const int32_t* d_s_key, uint64_t n_s,
                                 uint64_t* d_count, void* cuda_stream);
const char* fj_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FJ_H_ */
