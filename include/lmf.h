/*
 * lmf.h -- C ABI of the GB300 aggregate-batch engine.
 *
 * The engine evaluates one batch of group-by aggregates over the natural join
 * of an acyclic schema without materialising the join (Sec. 1.1, problem
 * statement; Sec. 3.1-3.2, aggregates decomposed into views along the edges of
 * a join tree).  A batch is a list of queries Q(F; alpha) (Eq. query, Sec. 2):
 * F is 0..3 categorical group-by attributes, alpha is a product of factors,
 * each a power x^p (p = 1, 2) of a continuous attribute or a threshold
 * indicator 1[x <= t] / 1[x > t] (the Kronecker deltas of Sec. 1.1).
 *
 * Evaluation is one bottom-up pass over the join tree: every child relation
 * is reduced on its join key into a device-resident view, views sharing a
 * parent key are merged (Sec. 3.4), and the root relation is scanned once
 * while probing the views (Sec. 3.5).  All compute runs in CUDA kernels for
 * sm_103a; there is no CPU fallback.
 *
 * Conventions for every entry point
 *   - Return value: LMF_OK (0) or a negative lmf_status; nothing crosses the
 *     ABI as an exception.  lmf_error_message() gives a one-line detail of the
 *     last failure on a context.
 *   - Pointers named dev_* or documented as device pointers are CUDA device
 *     pointers on the context's device; everything else is host memory.
 *   - One context per host thread; a context is not thread safe.  There is no
 *     global mutable state.
 *   - Calls that take (ctx, batch_id) return LMF_ERR_ARG for a null ctx or a
 *     batch id lmf_declare_batch did not hand out, LMF_ERR_STATE when the
 *     batch needs a plan and has none; a failing CUDA call gives LMF_ERR_CUDA
 *     (LMF_ERR_OOM for a failed allocation).  Outputs are meaningful only on
 *     LMF_OK.
 *   - LMF_LOG=1 in the environment prints every plan (root, probe groups,
 *     record sizes, root-scan form and launch shape) and the stage times of
 *     lmf_run_profiled to stderr.
 *   - LMF_JIT_DUMP=<directory> writes the CUDA source of every root scan and
 *     tree pass the planner compiles there (<kernel>_<hash of the source>.cu).
 */
#ifndef LMF_H_
#define LMF_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lmf_ctx lmf_ctx;
typedef int32_t lmf_status;

/* status codes */
#define LMF_OK               0
#define LMF_ERR_ARG         -1   /* bad argument: null pointer, bad id, bad size */
#define LMF_ERR_NOT_TREE    -2   /* declared edges do not form a join tree */
#define LMF_ERR_DTYPE       -3   /* column dtype/role does not fit its use */
#define LMF_ERR_KEY         -4   /* key or category value out of its range */
#define LMF_ERR_OOM         -5   /* device allocation failed */
#define LMF_ERR_CUDA        -6   /* a CUDA call failed */
#define LMF_ERR_TIMEOUT     -7   /* a device-side wait ran out of its limit */
#define LMF_ERR_OVERFLOW    -8   /* an exact integer count would overflow */
#define LMF_ERR_STATE       -9   /* call out of order (e.g. run before plan) */
#define LMF_ERR_UNSUPPORTED -10  /* valid query shape this engine does not evaluate */

/* column dtypes */
#define LMF_I32 0
#define LMF_F32 1
#define LMF_F64 2
#define LMF_I64 3                /* result dtype of exact counts */

/* column roles */
#define LMF_KEY  0               /* int32 join key, values >= 0 */
#define LMF_CONT 1               /* continuous attribute (f32 or f64) */
#define LMF_CAT  2               /* int32 category in [0, cat_domain) */

/* factor kinds */
#define LMF_POW 0                /* attr^power, power in {1, 2} */
#define LMF_LE  1                /* 1[attr <= threshold] */
#define LMF_GT  2                /* 1[attr >  threshold] */

/* plan options */
#define LMF_PREC_PLAIN_FP32  0   /* root Gram on CUDA cores, FP32 products */
#define LMF_PREC_SPLIT_BF16  1   /* root Gram on tcgen05 tensor cores, 3-way split bf16 */
#define LMF_BATCH_SINGLE     0   /* lmf_run enqueues the kernels one by one */
#define LMF_BATCH_GRAPH      1   /* lmf_run replays one captured CUDA graph */
#define LMF_ROOT_DECLARED    0   /* the relation that is nobody's child */
#define LMF_ROOT_EXPLICIT    1   /* lmf_plan_opts.root_rel */
#define LMF_ROOT_HEURISTIC   2   /* the root rule of Sec. 3.3: largest total group-by
                                    weight, ties to the largest relation */
#define LMF_ROOT_PER_QUERY   3   /* per-query roots (Sec. 3.3): the declared root when the
                                    whole batch evaluates there, else the aggregates grouped by
                                    a root each (see lmf_plan) */

#define LMF_MAX_GROUP_BY 3
#define LMF_MAX_FACTORS  16

typedef struct {
  const char* name;       /* attribute name; join keys share names across relations */
  int32_t dtype;          /* LMF_I32 / LMF_F32 / LMF_F64 */
  int32_t role;           /* LMF_KEY / LMF_CONT / LMF_CAT */
  const void* data;       /* nrows elements; device pointer, or pinned host pointer
                             when on_host is LMF_HOST_COPY or LMF_HOST_MAPPED */
  int32_t cat_domain;     /* LMF_CAT: number of categories */
  int32_t on_host;        /* LMF_DEVICE, LMF_HOST_COPY or LMF_HOST_MAPPED */
} lmf_column;

/* lmf_column.on_host */
#define LMF_DEVICE      0  /* device memory, borrowed */
#define LMF_HOST_COPY   1  /* pinned host memory, copied to a device staging buffer by every lmf_run */
#define LMF_HOST_MAPPED 2  /* pinned (mapped) host memory read in place by the kernels over the host
                              link, no staging copy: for columns the scan streams once (a root's
                              columns); lmf_register_relation fails with LMF_ERR_ARG when the
                              pointer is not device-accessible page-locked memory */

typedef struct {
  const char* attr;
  int32_t kind;           /* LMF_POW / LMF_LE / LMF_GT */
  int32_t power;          /* LMF_POW: 1 or 2 */
  double threshold;       /* LMF_LE / LMF_GT */
} lmf_factor;

typedef struct {
  int32_t n_group_by;                     /* 0..LMF_MAX_GROUP_BY */
  const char* group_by[LMF_MAX_GROUP_BY]; /* categorical attributes */
  int32_t n_factors;                      /* 0 (COUNT) .. LMF_MAX_FACTORS */
  const lmf_factor* factors;
} lmf_agg_spec;

typedef struct {
  int32_t precision;      /* LMF_PREC_* */
  int32_t batching;       /* LMF_BATCH_* */
  int32_t tile_rows;      /* root rows per tile; 0 = tuned default */
  int32_t ctas_per_sm;    /* resident CTAs per SM for the root scan; 0 = default */
  int32_t root_mode;      /* LMF_ROOT_* */
  int32_t root_rel;       /* LMF_ROOT_EXPLICIT: relation id of the root */
  int32_t no_merge;       /* 1: one record array per child view instead of one per
                             parent key (turns off merge case (1) of Sec. 3.4) */
  int32_t flags;          /* LMF_PLAN_* bits */
} lmf_plan_opts;

/* lmf_plan_opts.flags: the plain root scan, and for a batch with filtered
   aggregates the tree pass (its row pass and its search for a row's node over
   the nodes' thresholds), are compiled at plan time with the plan's layout as
   constants (the compilation step of Sec. 1.2 / App. C, done with NVRTC)
   unless this bit is set or NVRTC cannot be loaded; the interpreted kernels
   (same arithmetic, same results) run otherwise. */
#define LMF_PLAN_NO_JIT 1
/* lmf_plan_opts.flags: keep every Gram block of the plain-precision root scan at
   the row level (FP32 products of the whole z = [1, x_root, view means]).  By
   default a plan whose child keys are all unique takes the key-level form: the
   scan sums only the products of two root features row by row and builds, per
   probe group, the reverse view (count and sums of the features the group's
   Gram blocks and grouped outputs need); every block with a view mean is then
   sum_k m(k) R[k][.] over the group's keys (the aggregate at the group's own
   root, Sec. 3.3).  Same results within the error rule; needs the plan-time
   compiler. */
#define LMF_PLAN_ROW_GRAM 2

/* Statistics of a plan, for reporting (lmf_plan_info). */
typedef struct {
  int32_t n_views;            /* child views built per run */
  int32_t n_probe_groups;     /* merged views probed by the root scan */
  int32_t z_len;              /* length of the per-row vector z = [1, x_root, view means] */
  int32_t n_gram_aggs;        /* aggregates read off the root Gram */
  int32_t n_grouped_aggs;     /* aggregates with group-by attributes */
  int32_t n_filtered_aggs;    /* aggregates with threshold indicators */
  int32_t n_kernels_per_run;  /* kernel launches per lmf_run */
  int32_t unique_keys;        /* 1 when every child key is unique (no fan-out) */
  int32_t root_grid;          /* CTAs of the root scan */
  int32_t precision;          /* precision actually used */
  int32_t root_rel;           /* relation id of the root actually used */
  int32_t merged;             /* 1 when views sharing a parent key are merged */
  int32_t tree_nodes;         /* filtered batches: distinct nodes (conjunctions) */
  int32_t tree_groups;        /* ... groups of mutually exclusive nodes */
  int32_t tree_slices;        /* ... histogram slices of the chosen shape */
  int32_t tree_split_w;       /* ... split attributes per slice */
  int32_t tree_node_w;        /* ... nodes per slice */
  int32_t tree_ctas_per_sm;   /* ... CTAs per SM */
  int32_t tree_chunk;         /* ... rows per work item */
  int64_t root_rows;          /* rows of the root relation */
  int64_t scratch_bytes;      /* device bytes owned by the plan */
  int32_t resident_group;     /* probe group whose key is held per CTA (a root sorted on
                                 that foreign key), -1: none */
  int32_t resident_cells;     /* shared-memory counters of the resident-key tables */
  int32_t jit;                /* 1: the root scan runs a kernel compiled for this plan */
  int32_t key_level;          /* 1: key-level Gram blocks (see LMF_PLAN_ROW_GRAM) */
  int32_t n_roots;            /* roots the batch is evaluated at (LMF_ROOT_PER_QUERY), else 1;
                                 with several, the other fields describe the first root's
                                 plan, except the aggregate, view and kernel totals and
                                 root_rel = -1 */
} lmf_plan_stats;

/*
 * Create a context on CUDA device `device` (Sec. 1.2: one engine instance
 * per batch workload).  *out receives the context.  Errors: LMF_ERR_ARG,
 * LMF_ERR_CUDA when the device cannot be used.
 */
lmf_status lmf_create(int device, lmf_ctx** out);

/*
 * Wait for the device, then free every device buffer the context owns (plans,
 * staging copies of host columns, its stream) and the context itself.  Borrowed
 * column memory stays the caller's.  Errors: LMF_ERR_ARG for a null ctx.
 */
lmf_status lmf_destroy(lmf_ctx* ctx);

/*
 * Register a relation R(omega_R) of the database (Sec. 2, query language):
 * `ncols` columns of `nrows` rows each, columnar.  Column memory is borrowed:
 * the caller keeps it alive and unmodified until the last lmf_sync that uses
 * it.  Names must be unique inside the relation; a non-key name must not occur
 * in another relation (the natural join would join on it).  *rel_id receives
 * the relation's id (0, 1, ... in registration order).
 * Errors: LMF_ERR_ARG, LMF_ERR_DTYPE (key/cat columns must be LMF_I32,
 * continuous ones LMF_F32 or LMF_F64), LMF_ERR_STATE after lmf_declare_join.
 */
lmf_status lmf_register_relation(lmf_ctx* ctx, const char* name, int64_t nrows,
                                 const lmf_column* cols, int ncols, int* rel_id);

/*
 * Declare the join tree (Sec. 3.1): edge e joins child_rel[e] to its parent
 * parent_rel[e] on the int32 attribute key_attr[e], present in both.  The
 * edges must form a tree over all registered relations; its root is the
 * relation that is nobody's child.  Child keys are indexed here (the engine's
 * analogue of load time, Sec. 4 setup: not part of a run): key range and
 * multiplicity are measured on the device.  Keys index arrays directly; an
 * attribute whose child keys are too sparse for that (max key >= 4 * rows +
 * 4096) is renumbered once, in engine-owned device copies of its columns on
 * both sides of its edges, by each value's rank among the distinct child keys
 * (values no child holds never join); the borrowed columns are not written.
 * Those copies are a snapshot: later runs read the renumbered copies, so
 * changes the caller makes to the key columns of a renumbered attribute after
 * this call are not seen (declare the join again on a new context instead).
 * Columns of dense-key attributes and all other columns are read live by every
 * run.
 * Errors: LMF_ERR_NOT_TREE, LMF_ERR_ARG (unknown attribute), LMF_ERR_DTYPE,
 * LMF_ERR_KEY (negative child keys), LMF_ERR_UNSUPPORTED (two relations
 * sharing an attribute other than their edge key), LMF_ERR_OOM.
 */
lmf_status lmf_declare_join(lmf_ctx* ctx, int n_edges, const int* parent_rel,
                            const int* child_rel, const char* const* key_attr);

/*
 * Declare a batch of n aggregates (Sec. 1.1, Eq. query).  *batch_id receives
 * its id.  Results of aggregate i: an exact int64 count per group when no
 * factor is a power (COUNT, possibly filtered), otherwise a float64 sum per
 * group.  Groups are dense, row-major over the group-by attributes' values;
 * empty groups read 0.
 * Errors: LMF_ERR_ARG (unknown attribute, bad factor: a power other than 1 or
 * 2, an unknown kind, a NaN threshold), LMF_ERR_DTYPE (group-by on a
 * non-categorical attribute, a factor on a non-continuous one), LMF_ERR_STATE
 * (before lmf_declare_join).
 */
lmf_status lmf_declare_batch(lmf_ctx* ctx, const lmf_agg_spec* aggs, int n, int* batch_id);

/*
 * Plan a batch (Sec. 3.2-3.5 analogue): decompose every aggregate into the
 * child views it needs, merge views that share a parent key, pick the root
 * scan's form and tiles, allocate all device buffers, and measure value
 * ranges of the columns the batch reads (for the exact fixed-point
 * accumulators).  opts may be NULL (defaults: split-bf16 Gram, graph batching).
 * With root_mode LMF_ROOT_PER_QUERY a batch that does not evaluate at the
 * declared root (a group-by or threshold attribute reached through a
 * fanning-out key, Sec. 3.3's per-query roots) is split: aggregates are
 * grouped by the relation holding their first such attribute (the declared
 * root for sums of monomials), each group planned at the first root that evaluates
 * it -- its own attribute's relation, the declared root, then the largest
 * relations -- and every run runs each group's plan and copies its results
 * into this batch's layout (lmf_plan_info reports n_roots).
 * Errors: LMF_ERR_UNSUPPORTED for aggregate shapes outside this engine
 * (e.g. group-by attributes reached through a non-unique key without
 * LMF_ROOT_PER_QUERY, degree-2 monomials under a group-by), LMF_ERR_OOM,
 * LMF_ERR_CUDA.
 */
lmf_status lmf_plan(lmf_ctx* ctx, int batch_id, const lmf_plan_opts* opts);

/*
 * Statistics of a planned batch (views and probe groups of Sec. 3.2-3.4, the
 * root scan's form) into *info (host).  Errors: the common ones.
 */
lmf_status lmf_plan_info(lmf_ctx* ctx, int batch_id, lmf_plan_stats* info);

/*
 * Run a planned batch on `cuda_stream` (a cudaStream_t; NULL = the context's
 * own stream).  Asynchronous: it only enqueues work (host-resident columns
 * are copied in on the same stream first).  Device-detected errors are
 * latched and returned by lmf_sync.  The stream must stay valid until the
 * batch's next run, or until lmf_sync / lmf_read_result have returned: those
 * calls wait on the stream of the last run.  Planning the batch again waits
 * for the whole device before it frees the old plan.
 */
lmf_status lmf_run(lmf_ctx* ctx, int batch_id, void* cuda_stream);

/* stages reported by lmf_run_profiled, in launch order */
#define LMF_STAGE_INPUT    0   /* host-resident column copies, accumulator reset */
#define LMF_STAGE_VIEWS    1   /* child views, deepest first (Sec. 3.2) */
#define LMF_STAGE_ROOT     2   /* the root scan: Gram, counts, grouped tables (Sec. 3.5) */
#define LMF_STAGE_TREE     3   /* threshold-filtered histograms (Sec. 2, regression trees) */
#define LMF_STAGE_FINALIZE 4   /* ordered combine of partials and result placement */
#define LMF_STAGES         5

/*
 * Like lmf_run without graph replay, with a CUDA event recorded on
 * `cuda_stream` at every stage boundary; waits for the run and writes the
 * LMF_STAGES stage durations in milliseconds to stage_ms (host array).
 * Errors: LMF_ERR_ARG for a null stage_ms, else those of lmf_run.
 */
lmf_status lmf_run_profiled(lmf_ctx* ctx, int batch_id, void* cuda_stream, float* stage_ms);

/*
 * Wait for the last run of the batch and return its device status: LMF_OK,
 * LMF_ERR_KEY (a category outside its domain), LMF_ERR_OVERFLOW,
 * LMF_ERR_TIMEOUT, or LMF_ERR_CUDA.
 */
lmf_status lmf_sync(lmf_ctx* ctx, int batch_id);

/*
 * Shape of aggregate `agg`'s result (the output of query Q(F; alpha), Eq.
 * query): *n_groups cells of *dtype (LMF_I64 or LMF_F64), stored at *offset
 * in the batch's int64 or float64 result array; any of the three outputs may
 * be NULL.  Errors: LMF_ERR_ARG for agg outside [0, n), else the common ones.
 */
lmf_status lmf_result_info(lmf_ctx* ctx, int batch_id, int agg, int64_t* n_groups,
                           int32_t* dtype, int64_t* offset);

/* Total cells of the batch's int64 and float64 result arrays (either output
 * may be NULL).  Errors: the common ones. */
lmf_status lmf_result_sizes(lmf_ctx* ctx, int batch_id, int64_t* n_i64, int64_t* n_f64);

/*
 * Copy all results of the last run: n_i64 int64 cells to dst_i64 and n_f64
 * doubles to dst_f64 (either may be NULL to skip), host or device memory
 * (dst_is_device).  Enqueued on `cuda_stream` (NULL: the stream of the last
 * run) after the run; a host copy waits for it.  Results stay owned by the
 * plan; they are overwritten by the next run.  Errors: the common ones.
 */
lmf_status lmf_read_results(lmf_ctx* ctx, int batch_id, int64_t* dst_i64, double* dst_f64,
                            int dst_is_device, void* cuda_stream);

/* Copy one aggregate's result (n_groups cells of its dtype, groups row-major
 * over the group-by values) to host memory dst; waits for the last run.
 * Errors: LMF_ERR_ARG for a null dst or agg outside [0, n), else the common
 * ones. */
lmf_status lmf_read_result(lmf_ctx* ctx, int batch_id, int agg, void* dst);

/* ---------------------------------------------------------------------------
 * Plan choice.  The paper picks the root of each query by a weight rule
 * (Sec. 3.3).  This engine adds a learned cost model over candidate plans
 * (root and Gram form); the rule stays the fallback
 * and the reference its regret is measured against.
 * ------------------------------------------------------------------------- */

/* Number of features lmf_plan_features writes: sizes of the relations and of
   the root, counts of views, probe groups, aggregates of each kind, record
   bytes, z length, key multiplicities, the Gram form (tensor core, key-level),
   the grid, view merging, root position, general-view work, reverse-view
   slots, per-row tables, tree batches, and the mean log2 run length of equal
   foreign keys in the root's order. */
#define LMF_PLAN_FEATURES 26

/*
 * Candidate plans for a declared batch: up to three roots (the declared one,
 * the Sec. 3.3 rule's one, the largest relations) x Gram form (plain FP32 with
 * key-level blocks, plain FP32 all at the row level, split bf16), views merged
 * per parent key, each as explicit plan options derived from *base (NULL: zero
 * options; its CTAs per SM and compile flag carry over).  Writes
 * min(max, count) entries to out (may be NULL) and the count to *n.
 * Errors: LMF_ERR_ARG (null n), LMF_ERR_STATE before lmf_declare_join.
 */
lmf_status lmf_plan_candidates(lmf_ctx* ctx, int batch_id, const lmf_plan_opts* base,
                               lmf_plan_opts* out, int max, int* n);

/*
 * Compile, on up to `threads` host threads (0: 8), the plan-time root scans
 * (and tree passes) of every candidate of lmf_plan_candidates(base) into the
 * process-wide cache of compiled sources, so that planning those candidates
 * afterwards finds them compiled.  The candidates are planned without compiling (the batch is left
 * without a plan: plan it again before running).  *n_compiled (may be NULL)
 * gets the number of sources compiled.  Errors: LMF_ERR_ARG, LMF_ERR_STATE
 * before lmf_declare_join.
 */
lmf_status lmf_plan_precompile(lmf_ctx* ctx, int batch_id, const lmf_plan_opts* base, int threads,
                               int* n_compiled);

/*
 * Features of the batch's current plan (host array of n >= LMF_PLAN_FEATURES
 * floats): sizes, view and group counts, z length, record bytes, aggregate
 * counts, key multiplicity, precision, CTAs per SM, merging, root position.
 * Errors: LMF_ERR_ARG (null feat, n too small), LMF_ERR_STATE before a plan.
 */
lmf_status lmf_plan_features(lmf_ctx* ctx, int batch_id, float* feat, int n);

typedef struct lmf_mlp lmf_mlp;

/*
 * The learned cost model (no counterpart in the paper, which plans by the
 * Sec. 3.3 rule alone): an FP32 MLP in -> hidden -> hidden -> 1 with ReLU,
 * predicting the log run time of a plan from its features.  Its parameters,
 * gradients and Adam moments live on `device`, owned by the model until
 * lmf_mlp_destroy.  Every call below is synchronous and returns LMF_ERR_ARG for
 * a null model or pointer argument, a size that does not match the model or a
 * batch <= 0, LMF_ERR_OOM / LMF_ERR_CUDA on device failures.
 */
/* A model with weights drawn from seed; 1 <= in_dim, hidden <= 4096. */
lmf_status lmf_mlp_create(int device, int in_dim, int hidden, uint64_t seed, lmf_mlp** out);
lmf_status lmf_mlp_destroy(lmf_mlp* m);
/* Parameter count and flat host copies of n = that count floats (layout
 * W1[in][h] b1[h] W2[h][h] b2[h] w3[h] b3). */
lmf_status lmf_mlp_num_params(lmf_mlp* m, int64_t* n);
lmf_status lmf_mlp_get_params(lmf_mlp* m, float* host, int64_t n);
lmf_status lmf_mlp_set_params(lmf_mlp* m, const float* host, int64_t n);
/* Input standardisation (x - mean) / std (host arrays of in_dim floats, std > 0)
 * and output scale y = y_std * out + y_mean (y_std > 0). */
lmf_status lmf_mlp_set_norm(lmf_mlp* m, const float* mean, const float* std, float y_mean, float y_std);
/* Predictions for `batch` feature rows x_dev[batch][in] (device) into y_dev[batch] (device). */
lmf_status lmf_mlp_forward(lmf_mlp* m, const float* x_dev, int batch, float* y_dev);
/*
 * Mean squared error on standardised targets y_dev (device, already
 * (y - y_mean) / y_std) and its gradient w.r.t. every parameter, written to
 * grad_dev (device, may be NULL); *loss (host, may be NULL).
 */
lmf_status lmf_mlp_grad(lmf_mlp* m, const float* x_dev, const float* y_dev, int batch, float* grad_dev,
                        float* loss);
/* One Adam step (beta 0.9 / 0.999) on that loss. */
lmf_status lmf_mlp_train_step(lmf_mlp* m, const float* x_dev, const float* y_dev, int batch, float lr,
                              float* loss);

/*
 * Plan the batch with the candidate the model predicts fastest (every
 * candidate is planned without compiling to compute its features; only the
 * chosen one is compiled).  model == NULL falls back to
 * the Sec. 3.3 root rule with *base.  The chosen options go to *chosen (may be
 * NULL).  Errors: LMF_ERR_STATE before lmf_declare_join, those of lmf_plan.
 */
lmf_status lmf_plan_learned(lmf_ctx* ctx, int batch_id, lmf_mlp* model, const lmf_plan_opts* base,
                            lmf_plan_opts* chosen);

/* ---------------------------------------------------------------------------
 * Consumers of a batch (Sec. 2): models trained from aggregates the engine
 * already holds in device memory.  Each is one small launch on cuda_stream
 * (NULL: the legacy default stream), asynchronous, deterministic (fixed-order
 * reductions).  Inputs and outputs are device pointers.
 * ------------------------------------------------------------------------- */

/*
 * Ridge linear regression by batch gradient descent over the covar matrix
 * (Sec. 2, objective J and its gradient; Sec. 4 setup: Barzilai-Borwein steps
 * with Armijo backtracking).  dev_sigma: m x m doubles, row-major, the covar
 * matrix sum X X^T over (X_1 = 1, features ..., label) -- the label last, its
 * parameter fixed at -1; count = |D|; lam >= 0 the penalty on theta_1..n.
 * Writes theta (m - 1 doubles) to dev_theta and the iterations run to
 * dev_iters (one int).  Stops when ||grad|| <= tol * max(1, ||grad_0||) or
 * after max_iter iterations.  Limits: 2 <= m <= 96.  Errors: LMF_ERR_ARG,
 * LMF_ERR_CUDA.
 */
lmf_status lmf_ridge_bgd(const double* dev_sigma, int m, double count, double lam, int max_iter, double tol,
                         double* dev_theta, int* dev_iters, void* cuda_stream);

/* One categorical pair of lmf_mutual_information: device pointers to the
 * marginal counts beta (dom_i) and gamma (dom_j) and the joint counts delta
 * (dom_i x dom_j, row-major), e.g. results of COUNT grouped by X_i, by X_j and
 * by (X_i, X_j). */
typedef struct {
  const int64_t* beta;
  const int64_t* gamma;
  const int64_t* delta;
  int32_t dom_i, dom_j;
} lmf_mi_pair;

/*
 * Mutual information of n_pairs categorical pairs (Sec. 2, Eq. mi: the sum of
 * delta/alpha * log(alpha delta / (beta gamma)) over the cells with delta > 0,
 * natural logarithm), alpha = the COUNT.  dev_pairs: device array of n_pairs
 * lmf_mi_pair; dev_mi: n_pairs doubles.  Errors: LMF_ERR_ARG (null pointers,
 * alpha <= 0), LMF_ERR_CUDA.
 */
lmf_status lmf_mutual_information(const lmf_mi_pair* dev_pairs, int n_pairs, int64_t alpha, double* dev_mi,
                                  void* cuda_stream);

/*
 * Chow-Liu tree over n attributes (Sec. 2): pairs in decreasing mutual
 * information (ties: the pair (i, j), i < j, first in row-major order), each
 * kept unless it closes a cycle.  dev_mi: n x n doubles (entries i < j read);
 * dev_edges: 2 (n - 1) ints, the kept pairs (i, j) in the order taken;
 * dev_n_edges: one int.  Limit n <= 64.  Errors: LMF_ERR_ARG, LMF_ERR_CUDA.
 */
lmf_status lmf_chow_liu(const double* dev_mi, int n, int* dev_edges, int* dev_n_edges, void* cuda_stream);

/*
 * The covar Gram of one relation (the covar matrix of Sec. 2, Eq. lr-sigma,
 * over a single relation), computed without allocating any device memory.
 * The allocation-free form has no counterpart in the paper: it exists for callers
 * that cannot call cudaMalloc -- code running under a memory pool or custom
 * allocator that forbids outside allocations, code that must avoid the
 * implicit synchronisation an allocation can cause, or a process whose device
 * memory is already handed to another framework.
 *
 * dev_cols: host array of ncols device pointers, each to nrows FP32 values.
 * dev_gram: device buffer of (ncols + 1)^2 doubles, written row-major with
 *           G = sum_r z_r z_r^T, z_r = [1, x_1(r), ..., x_ncols(r)] (G[0][0] = nrows).
 * cuda_stream: the stream to enqueue on (NULL: the legacy default stream).
 * The same kernel as the plain root scan (FP32 products, ordered FP64
 * combine) runs with its scratch -- per-CTA partial Grams and counts -- in a
 * fixed array compiled into the library (about 2.5 MB: at most 304 CTAs of
 * 32 x 32 doubles), which every GPU that loads the library keeps until the
 * process exits.  Limit: ncols <= 31; larger sizes, negative sizes and null
 * pointers return LMF_ERR_ARG; CUDA failures return LMF_ERR_CUDA.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  All
 * calls share the array, so calls that overlap on the GPU race; enqueue them
 * on one stream or wait between them.  Asynchronous: the result is ready when
 * the stream reaches it.
 */
lmf_status lmf_gram_noalloc(const float* const* dev_cols, int ncols, int64_t nrows, double* dev_gram,
                            void* cuda_stream);

/*
 * Failure-detection check (no counterpart in the paper).  Every device wait of
 * the engine is bounded: the tensor-core root scan waits on an mbarrier for
 * its MMAs, and after a fixed number of polls (about 0.3 s) it stops waiting,
 * sets the timeout bit of the plan's status word and returns, so that lmf_sync
 * reports LMF_ERR_TIMEOUT and the context stays usable.  This call runs that
 * same bounded wait on a barrier nothing ever arrives at, on ctx's device and
 * stream, and reads the status back: it returns LMF_ERR_TIMEOUT when the wait
 * gave up and reported it (the expected result), LMF_OK if the wait
 * completed, LMF_ERR_CUDA on a CUDA failure.  Synchronous; allocates one word.
 */
lmf_status lmf_wait_selftest(lmf_ctx* ctx);

/* Static text of a status code (never NULL; unknown codes give "unknown status"). */
const char* lmf_status_string(lmf_status s);

/* Detail of the last failure on ctx (empty string when none, or for a null
 * ctx); owned by the context, valid until its next call. */
const char* lmf_error_message(lmf_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LMF_H_ */
