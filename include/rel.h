/*
 * rel.h -- C ABI of the GB300 (sm_103a) relational hot path: a fused
 * filter + hash group-by with exact int64 aggregates, and a hash equi-join
 * (build, count, probe with match-pair emission and payload gather).
 *
 * What the operators compute follows the paper's statement of the profiled
 * relational operators (arxiv 2608.13696): columnar, Arrow-like inputs and an
 * operator API that runs one or more kernels per call (Sec. 2.3); group-by
 * aggregation in shared memory (Sec. 7, single_pass_shmem_aggs_kernel);
 * expressions evaluated inside the operator instead of by an interpreter
 * (Sec. 7, compute_column_kernel); the join's build / count / retrieve steps
 * over a hash table read randomly (Sec. 7, insert_if_n, count, retrieve) and
 * the gather out[i] = in[map[i]] (Sec. 7, transform_kernel).
 *
 * Conventions for every entry point:
 *  - Pointers named *data, keys, payload, out_* and ws are DEVICE pointers
 *    owned by the caller; the library never allocates device or pinned
 *    memory.  Descriptors, plans, rel_join_table and *_host pointers are HOST
 *    memory owned by the caller.
 *  - A workspace (ws) starts on a 256-byte boundary, as every cudaMalloc and
 *    PyTorch allocation does; any other address is REL_E_INVALID before any
 *    device work (the tables in it are read with 32-byte vector loads).
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  A call that writes a *_host count synchronises that stream
 *    before returning; with a NULL *_host pointer the call does not block.
 *  - Errors are return codes (rel_status); nothing throws across the ABI.
 *    rel_last_error() gives a thread-local message for the last failure.
 *  - Result rows come in an unspecified order.
 *  - Every device-side wait is bounded; a wait that gives up returns
 *    REL_E_TIMEOUT instead of hanging.
 */
#ifndef REL_H
#define REL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t rel_status;
#define REL_OK 0
#define REL_E_INVALID (-1)     /* bad descriptor, size or pointer              */
#define REL_E_CAPACITY (-2)    /* output or workspace too small; see *_host    */
#define REL_E_CUDA (-3)        /* a CUDA runtime call failed                   */
#define REL_E_TIMEOUT (-4)     /* a bounded device-side wait gave up           */
#define REL_E_UNSUPPORTED (-5) /* valid request outside the library's limits    */
#define REL_E_OVERFLOW (-6)    /* hash table sized by the plan was too small   */

/* column element types */
#define REL_U8 0
#define REL_I32 1
#define REL_I64 2

/* aggregate operators */
#define REL_SUM 0
#define REL_COUNT 1
#define REL_MIN 2
#define REL_MAX 3

/* group-by variants (a plan's choice; results never depend on it) */
#define REL_VAR_AUTO 0        /* let rel_plan_size choose                       */
#define REL_VAR_SMEM 1        /* per-CTA shared-memory tables, merged at the end */
#define REL_VAR_GLOBAL 2      /* one global open-addressing table               */
#define REL_VAR_PARTITIONED 3 /* hash-partition the rows, then one shared-memory
                                 table per partition (key + int64 value inputs)  */

/* limits of one group-by descriptor */
#define REL_MAX_COLS 8
#define REL_MAX_KEYS 4
#define REL_MAX_PREDS 4
#define REL_MAX_AGGS 8

typedef struct {
  const void* data; /* device pointer, n_rows elements of `type`            */
  int32_t type;     /* REL_U8, REL_I32 or REL_I64                           */
  int32_t reserved; /* 0                                                    */
} rel_col;

/* Row filter term: lo <= col[i] <= hi (inclusive, compared as int64). */
typedef struct {
  int32_t col;
  int32_t reserved;
  int64_t lo, hi;
} rel_range_pred;

/* One aggregate.  Its input for row i is
 *     base[i] * prod_{f < nf} (c[f] + s[f] * fcol[f][i])     (mod 2^64)
 * with every column read as int64 (u8 zero-, i32 sign-extended).  SUM adds
 * inputs mod 2^64, MIN / MAX compare them as signed int64, COUNT counts the
 * group's rows and ignores the input. */
typedef struct {
  int32_t op;       /* REL_SUM, REL_COUNT, REL_MIN, REL_MAX                    */
  int32_t base_col;
  int32_t nf;       /* 0, 1 or 2                                               */
  int32_t reserved;
  int32_t fcol[2];
  int64_t c[2];
  int64_t s[2];
} rel_agg;

/* Filtered group-by:
 *   rows  : i in [0, n_rows) with every predicate true;
 *   key   : one key column -> its int64 value; several (u8 / i32 only, at
 *           most 64 bits together) -> their bit patterns concatenated, the
 *           first column in the most significant position;
 *   output: one row per key that has at least one qualifying row. */
typedef struct {
  int64_t n_rows;
  int32_t n_cols, n_keys, n_preds, n_aggs;
  const rel_col* cols;        /* n_cols   */
  const int32_t* key_cols;    /* n_keys   */
  const rel_range_pred* preds;/* n_preds  */
  const rel_agg* aggs;        /* n_aggs   */
} rel_groupby_desc;

/* plan flags */
#define REL_PLAN_EXACT 1u   /* count distinct qualifying keys exactly (GPU pre-pass) */
#define REL_PLAN_LEARNED 2u /* sample sketch + planner network: size and variant     */
#define REL_PLAN_GENERIC 4u /* force the descriptor-interpreting kernel              */
#define REL_PLAN_SKETCH 8u  /* sample sketch: heavy hitters pinned per CTA           */
/* Force a variant (bits 8..9 of flags; 0 = the planner's choice):
 * REL_PLAN_FORCE(REL_VAR_SMEM): per-CTA table of next_pow2(2 * est) slots
 *   (at most 4096; what does not fit spills to the global table);
 * REL_PLAN_FORCE(REL_VAR_GLOBAL): no per-CTA layer, every row updates the
 *   global table;
 * REL_PLAN_FORCE(REL_VAR_PARTITIONED): partitioned; only for one int32 or
 *   int64 key, no filter, and SUM, COUNT (and MIN, MAX) of one int64 value
 *   column, with fewer than 2^32 rows (REL_E_UNSUPPORTED otherwise). */
#define REL_PLAN_FORCE(v) ((uint32_t)(v) << 8)
#define REL_PLAN_FORCE_MASK 0x300u
/* Set in plan->flags by rel_groupby_auto when the first plan overflowed and
 * the call re-planned with the exact pre-pass. */
#define REL_PLAN_FELL_BACK 0x10000u
/* Set in plan->flags by a REL_PLAN_LEARNED plan that a full-data HyperLogLog
 * sized (see rel_plan_size). */
#define REL_PLAN_HLL_SIZED 0x20000u
/* Test hook for the device-side wait limit, not for production use.  Set in
 * plan->flags before rel_groupby_agg: the staged kernel's consumers never hand
 * a shared-memory stage back to its producer, so once a CTA's ring has gone
 * round once, the producer's bounded wait, and then the consumers', give up
 * after 20 ms (instead of the normal 2 s); the producer still waits for the
 * copies it issued, nothing is left in flight, and the call returns
 * REL_E_TIMEOUT.  Only plans that run the staged kernel with a CTA that gets
 * more tiles than stages (e.g. tile_rows = 256, n_stages = 2 on 10^6 rows)
 * reach the wait; other plans run normally.  The paper has no counterpart:
 * this tests the library's failure detection without faulting a GPU. */
#define REL_PLAN_TEST_STALL 0x40000000u

#define REL_MAX_HOT 32

/* A plan fixes the table sizes; rows fall through thread-private slots, then
 * a CTA-shared table, then the global table (each of the first two optional),
 * so the result never depends on the plan -- only the speed does. */
typedef struct {
  int64_t slots;            /* global hash-table slots (power of two >= 16)     */
  int32_t variant;          /* REL_VAR_* label of the choice                    */
  int32_t smem_slots;       /* CTA-shared table slots: 0 or a power of two in
                               [16, 4096]                                       */
  uint64_t workspace_bytes; /* bytes rel_groupby_agg needs in ws               */
  uint64_t scratch_bytes;   /* bytes rel_plan_size itself needs in ws          */
  int64_t est_groups;       /* estimated (or, with REL_PLAN_EXACT, exact)
                               number of groups                                 */
  uint32_t flags;           /* REL_PLAN_* used                                  */
  int32_t tiny_slots;       /* thread-private slots per CTA: 0, 8, 16 or 32     */
  uint32_t tiny_mult;       /* multiplier of the thread-private slot hash; 0
                               picks the default                                */
  int32_t n_hot;            /* > 0: these keys are preloaded into the thread-
                               private slots, which then admit no other key     */
  int64_t hot_keys[REL_MAX_HOT];
  int32_t tile_rows;        /* rows per staged tile (256..2048, power of two); 0 = auto */
  int32_t n_stages;         /* staging ring depth (2..8); 0 = auto                    */
  int32_t part_bits;        /* REL_VAR_PARTITIONED: log2 of the partition count
                               (4..14); smem_slots is then each partition's table */
  int32_t reserved;
} rel_plan;

#define REL_OP_GROUPBY 0
#define REL_OP_JOIN_PROBE 1

/* Sizing step (the operator's small "decide the next step" kernel, Sec. 2.3).
 *  op = REL_OP_GROUPBY, desc = const rel_groupby_desc*:
 *    groups_hint > 0: size the table for that many groups (no GPU work);
 *    flags & REL_PLAN_EXACT: count distinct qualifying keys on the GPU; needs
 *      plan->scratch_bytes of ws (query with ws = NULL: returns
 *      REL_E_CAPACITY after filling scratch_bytes).  The count first uses a
 *      key set of at most 2^24 slots and reads the keys a second time, into
 *      the full set, only when the distinct keys overflow it;
 *    otherwise: size for n_rows groups (always sufficient, rarely economical).
 *    flags & REL_PLAN_LEARNED (without a hint or REL_PLAN_EXACT): run
 *      rel_sketch, then the registered planner network (rel_planner_set) on
 *      its features; est_groups = max(ceil(1.25 * 2^(y0 + 1)), sample distinct
 *      keys), the variant is the network's most likely one that the
 *      descriptor supports.  For one int32 / int64 key without a filter,
 *      at least 2^22 rows, and a sample whose distinct keys were more than
 *      3/4 seen once (a long tail the sample cannot size), one streaming
 *      pass of a full-data HyperLogLog (4096 registers) gives est = its
 *      estimate x 1.25 instead, and the variant follows the rule by group
 *      count; plan->flags then has REL_PLAN_HLL_SIZED.  Needs
 *      rel_sketch_ws_bytes() + 18432 bytes of ws and returns REL_E_INVALID
 *      when no network is registered.  An estimate
 *      can be too low: rel_groupby_agg then returns REL_E_OVERFLOW
 *      (rel_groupby_auto re-plans exactly).
 *    flags & REL_PLAN_SKETCH (with any of the above): also run rel_sketch and
 *      pin the sample's most frequent keys in the thread-private slots (all
 *      of them when the sample suggests few groups, the heavy hitters when it
 *      is skewed), with a hash multiplier that places them without
 *      collisions.  Needs rel_sketch_ws_bytes() of ws as well.
 *    Fills slots, variant, tiny/smem slots, hot keys, workspace_bytes,
 *    est_groups.
 *  op = REL_OP_JOIN_PROBE, desc = const rel_join_probe_desc*: counts the
 *    pairs the probe will emit (the paper's "count" step) into est_groups.
 *  Returns REL_OK, REL_E_INVALID, REL_E_CAPACITY, REL_E_CUDA, REL_E_TIMEOUT. */
rel_status rel_plan_size(int32_t op, const void* desc, uint32_t flags, int64_t groups_hint,
                         void* ws, size_t ws_bytes, rel_plan* plan, void* stream);

/* Run the group-by with a plan from rel_plan_size (the caller may change
 * tiny_slots / smem_slots / slots within their stated ranges).
 *  ws       : >= plan->workspace_bytes device bytes, any content on entry;
 *             the call zeroes what it uses.  Must not be shared by calls that
 *             overlap on the GPU.
 *  out_keys : int64[out_capacity] group keys.
 *  out_aggs : n_aggs device pointers, each int64[out_capacity].
 *  n_groups_host: receives the number of groups (after a stream sync).
 * Returns REL_OK; REL_E_CAPACITY when groups > out_capacity (*n_groups_host
 * = groups; outputs partially written); REL_E_OVERFLOW when the groups did
 * not fit plan->slots (re-plan larger, e.g. with REL_PLAN_EXACT);
 * REL_E_INVALID / REL_E_UNSUPPORTED for bad or out-of-limit requests;
 * REL_E_TIMEOUT, REL_E_CUDA. */
rel_status rel_groupby_agg(const rel_groupby_desc* desc, const rel_plan* plan, void* ws,
                           size_t ws_bytes, int64_t* out_keys, int64_t* const* out_aggs,
                           int64_t out_capacity, int64_t* n_groups_host, void* stream);

/* Device bytes rel_groupby_agg needs for `slots` table slots and `n_aggs`
 * aggregates. */
uint64_t rel_groupby_ws_bytes(int64_t slots, int32_t n_aggs);

/* Device bytes rel_groupby_agg needs for a (possibly edited) plan over
 * n_rows rows with n_aggs aggregates -- the partitioned variant also keeps a
 * 16-byte record per row, and a second one per row above 256 partitions
 * (its scatter runs in two levels). */
uint64_t rel_plan_ws_bytes(const rel_plan* plan, int32_t n_aggs, int64_t n_rows);

/* Plan and run in one call, with the learned planner's overflow fallback:
 * plan with `flags` (as rel_plan_size with groups_hint 0), run; when the run
 * overflows a plan that was not exact, plan again with REL_PLAN_EXACT
 * (keeping REL_PLAN_SKETCH, REL_PLAN_GENERIC and a forced variant) and run
 * again.  ws must hold rel_groupby_auto_ws_bytes(desc) bytes (enough for any
 * plan of desc).  plan_out (host, may be NULL) receives the plan that gave
 * the result, REL_PLAN_FELL_BACK set in its flags after a re-plan.  Outputs
 * and return codes as rel_groupby_agg; REL_E_CAPACITY before any device work
 * when ws is smaller than stated. */
rel_status rel_groupby_auto(const rel_groupby_desc* desc, uint32_t flags, void* ws,
                            size_t ws_bytes, int64_t* out_keys, int64_t* const* out_aggs,
                            int64_t out_capacity, int64_t* n_groups_host, rel_plan* plan_out,
                            void* stream);

/* Device bytes rel_groupby_auto needs for desc (0 for an invalid desc). */
uint64_t rel_groupby_auto_ws_bytes(const rel_groupby_desc* desc);

/* ------------------------------------------------------ sample sketch */

#define REL_SKETCH_TOP 32
#define REL_SKETCH_FEATURES 264

/* Summary of a 4096-row sample of a group-by input (the planner's view of
 * the data; the paper has no planner, this is what the sizing step reads).
 * Sample: every row when n_rows <= 4096, else 64 windows of 64 consecutive
 * rows starting at floor(w * (n_rows - 64) / 63); rows the filter rejects
 * are dropped ("kept" = the rest).  runs counts maximal runs of equal keys
 * among kept rows inside each block of 64 sample positions.  hll holds 256
 * HyperLogLog registers (p = 8) of splitmix64(key): register h >> 56, value
 * = leading zeros of the low 56 bits + 1 (57 if zero).  top_* lists up to 32
 * keys by count descending, key ascending.  features = hll / 57 followed by
 * log2(n_rows), ndv / kept, log2(key_max - key_min + 1), top-1 share, top-8
 * share, singletons / ndv, kept / runs, key width / 64. */
typedef struct {
  int64_t n_rows;
  int32_t sample_rows, kept, ndv, singletons, runs, key_bits;
  int64_t key_min, key_max;
  int64_t top_key[REL_SKETCH_TOP];
  int32_t top_count[REL_SKETCH_TOP];
  uint8_t hll[256];
  float features[REL_SKETCH_FEATURES];
} rel_sketch_info;

/* Device bytes rel_sketch needs in ws. */
uint64_t rel_sketch_ws_bytes(void);

/* One single-CTA kernel over the sample; fills *out (host) after a stream
 * sync.  Returns REL_OK, REL_E_INVALID, REL_E_CAPACITY (ws too small),
 * REL_E_CUDA. */
rel_status rel_sketch(const rel_groupby_desc* desc, void* ws, size_t ws_bytes,
                      rel_sketch_info* out, void* stream);

/* Sketches of n inputs in one launch (one CTA each) and one read-back:
 * out[i] as rel_sketch(descs + i).  ws: rel_sketch_batched_ws_bytes(n). */
uint64_t rel_sketch_batched_ws_bytes(int32_t n);
rel_status rel_sketch_batched(const rel_groupby_desc* descs, int32_t n, void* ws, size_t ws_bytes,
                              rel_sketch_info* out, void* stream);

/* Group-by without any device allocation, for callers that cannot allocate
 * device memory: an engine whose own pool owns all of the GPU's memory and
 * forbids other allocations, a plugin whose host process caps device memory,
 * or a latency-critical path that must not call cudaMalloc / cudaFree (they
 * can synchronise the device).  The paper has no counterpart; this is an
 * interface convenience.
 *
 * Same result as rel_groupby_agg, but the hash table lives in a scratch array
 * compiled into the library (about 4.5 MiB of device memory that every GPU
 * which loads the library keeps until the process exits), sized for
 * max_groups <= REL_STATIC_MAX_GROUPS.  The caller passes the inputs (desc)
 * and the outputs as for rel_groupby_agg, plus max_groups, an upper bound on
 * the number of groups.  max_groups outside 1..REL_STATIC_MAX_GROUPS is
 * rejected with REL_E_UNSUPPORTED before any device work; more groups than
 * the table sized from max_groups can hold gives REL_E_OVERFLOW.
 * n_groups_host is required here (NULL gives REL_E_INVALID): the call syncs
 * the stream, writes the group count there and reads the overflow flag.
 *
 * Every call looks up the scratch array's device address on the current
 * device (cudaGetSymbolAddress); the first call on a device may load the
 * library's device code, so make it before any stream capture.  Every call
 * on a device shares the one array:
 * each call clears what it uses before its kernels run, so sequential calls
 * are independent, but calls that overlap on the GPU (different streams or
 * threads without ordering between them) race and give wrong results. */
#define REL_STATIC_MAX_GROUPS 32768
rel_status rel_groupby_agg_static(const rel_groupby_desc* desc, int64_t max_groups,
                                  int64_t* out_keys, int64_t* const* out_aggs,
                                  int64_t out_capacity, int64_t* n_groups_host, void* stream);

/* The learned sizing rule, on the host: from a sketch and the planner
 * network's 4 outputs y (host floats: log2 of the group count, then the
 * logits of REL_VAR_SMEM, REL_VAR_GLOBAL, REL_VAR_PARTITIONED) to the
 * estimate and variant REL_PLAN_LEARNED uses.  est_groups = the smaller of
 * n_rows and ceil(1.25 * 2^(clamp(y0, 0, 61) + 1)) (n_rows when y0 is not
 * finite), raised to the sample's distinct keys (info->ndv); variant = the
 * largest logit among the allowed variants (REL_VAR_PARTITIONED only when
 * partitioned_ok), ties to the lower-numbered one.  The paper has no planner;
 * this is the decision rule of the learned form built on its operators.
 * No device work.  Returns REL_OK or REL_E_INVALID (NULL pointers, n_rows < 0). */
rel_status rel_plan_learned_rule(const rel_sketch_info* info, const float* y, int64_t n_rows,
                                 int32_t partitioned_ok, int64_t* est_groups, int32_t* variant);

/* Learned plans for n group-bys at once (the batched mode's sizing step):
 * one rel_sketch_batched launch, one network forward over all n feature
 * rows, then rel_plan_learned_rule per input with the variant chosen among
 * REL_VAR_SMEM and REL_VAR_GLOBAL (the batched launch has no partitioned
 * variant).  flags: REL_PLAN_LEARNED, optionally | REL_PLAN_SKETCH (pin the
 * sample's heavy hitters as rel_plan_size does); anything else gives
 * REL_E_UNSUPPORTED.  descs: n host descriptors; plans: n host plans,
 * filled as rel_plan_size fills them.  ws: rel_plan_size_batched_ws_bytes(n)
 * device bytes.  Syncs the stream.  Returns REL_OK, REL_E_INVALID (bad
 * descriptor, no registered network), REL_E_CAPACITY (ws too small),
 * REL_E_UNSUPPORTED, REL_E_CUDA. */
uint64_t rel_plan_size_batched_ws_bytes(int32_t n);
rel_status rel_plan_size_batched(const rel_groupby_desc* descs, int32_t n, uint32_t flags,
                                 void* ws, size_t ws_bytes, rel_plan* plans, void* stream);

/* HyperLogLog of every key of one int32 / int64 column (no filter): the
 * learned planner's full-data check for long tails.  p = 12: 4096 registers;
 * h = fmix64(key ^ 2^63) (the MurmurHash3 64-bit finalizer), register h >> 52,
 * value = leading zeros of the low 52 bits + 1 (53 when they are all zero);
 * estimate as Flajolet, Fusy, Gandouet and Meunier (2007) with the
 * small-range correction (standard error 1.04 / 64).  The paper has no
 * planner; this is a sizing step of the learned form.  keys: device array of
 * n; ws: rel_key_hll_ws_bytes() device bytes; regs_host: host uint32[4096];
 * syncs the stream.  Returns REL_OK, REL_E_INVALID, REL_E_CAPACITY,
 * REL_E_CUDA. */
uint64_t rel_key_hll_ws_bytes(void);
rel_status rel_key_hll(const void* keys, int32_t key_type, int64_t n, void* ws, size_t ws_bytes,
                       uint32_t* regs_host, double* estimate, void* stream);

/* ---------------------------------------------------- planner network */

/* A small network maps a sketch's 264 features to an estimate of log2(number
 * of groups) and logits over three group-by variants (REL_VAR_SMEM,
 * REL_VAR_GLOBAL, REL_VAR_PARTITIONED).  The paper has no planner; this is
 * the sizing step learned from runs of this library.  264 -> 64 -> 64 -> 4,
 * ReLU hidden layers, BF16 weights and activations multiplied with FP32
 * accumulation.  Parameters (FP32 master copy, and a BF16 copy of the same
 * layout) in order: W1[64][264] b1[64] W2[64][64] b2[64] W3[4][64] b3[4].
 * Every pointer below is device memory owned by the caller. */
#define REL_MLP_IN 264
#define REL_MLP_HIDDEN 64
#define REL_MLP_OUT 4
#define REL_MLP_PARAMS 21380

/* bf16_params[i] = round-to-nearest-even BF16 of params[i]. */
rel_status rel_mlp_round(const float* params, void* bf16_params, void* stream);

/* out[b][0..4) for b < batch; x is batch x 264 FP32 (rounded to BF16 on
 * entry).  acts (batch x 128 floats) receives the hidden pre-activations for
 * rel_mlp_backward, or is NULL. */
rel_status rel_mlp_forward(const void* bf16_params, const float* params, const float* x,
                           int32_t batch, float* out, float* acts, void* stream);

/* Scratch bytes rel_mlp_backward needs for a batch. */
uint64_t rel_mlp_ws_bytes(int32_t batch);

/* Gradient of the batch-mean loss (y0 - t_ndv)^2 + CE(softmax(y1..3), t_var)
 * with respect to every parameter (grad: REL_MLP_PARAMS floats, overwritten);
 * *loss (device float) receives the batch-mean loss.  x, acts and out as
 * produced by rel_mlp_forward; t_var in {0, 1, 2}. */
rel_status rel_mlp_backward(const void* bf16_params, const float* x, const float* acts,
                            const float* out, const float* t_ndv, const int32_t* t_var,
                            int32_t batch, void* ws, size_t ws_bytes, float* grad, float* loss,
                            void* stream);

/* One AdamW step (decoupled weight decay on weights, not biases; bias-
 * corrected moments m, v; step >= 1), then refresh the BF16 copy. */
rel_status rel_mlp_adamw(float* params, void* bf16_params, float* m, float* v, const float* grad,
                         int32_t step, float lr, float beta1, float beta2, float eps,
                         float weight_decay, void* stream);

/* Register the network REL_PLAN_LEARNED plans with (device pointers, kept by
 * reference; NULL clears).  Not thread-safe against concurrent planning. */
rel_status rel_planner_set(const void* bf16_params, const float* params);

/* -------------------------------------------------- batched execution */

/* Many small group-bys and joins in two persistent launches (the paper's
 * launches too small to fill the GPU, Sec. 5.3).  The caller describes every
 * instance, rel_batch_prepare writes the descriptors into the workspace and
 * fills a host handle, and rel_batch_run issues the device work only (one
 * memset, two launches, no host synchronisation, no allocation), so a CUDA
 * graph can capture it and replay it while the inputs stay where they are.
 * Results equal those of rel_groupby_agg / rel_join_probe instance by
 * instance (same groups and pairs; order unspecified).  The paper has no
 * batched form; this is an execution mode of this library. */

#define REL_BATCH_MAX_AGGS 4

/* A key/value group-by: one int32 or int64 key column, aggregates of one
 * int64 value column. */
typedef struct {
  const void* keys;        /* device, n_rows keys */
  const int64_t* vals;     /* device, n_rows values; NULL if every op is COUNT */
  int64_t n_rows;
  int32_t key_type;        /* REL_I32 or REL_I64 */
  int32_t n_aggs;          /* 1..4 */
  int32_t ops[REL_BATCH_MAX_AGGS]; /* REL_SUM / REL_COUNT / REL_MIN / REL_MAX */
  int64_t slots;           /* global table slots, power of two >= 16, >= the groups */
  int64_t est_groups;      /* expected groups: decides shared-memory pre-aggregation */
  int64_t* out_keys;       /* device, out_capacity entries */
  int64_t* out_aggs[REL_BATCH_MAX_AGGS];
  int64_t out_capacity;
} rel_batch_groupby;

/* A join partition: build side (unique or not), probe side, outputs. */
typedef struct {
  const int64_t* build_keys;
  const int64_t* build_payload;
  int64_t n_build;         /* < 2^31 */
  const int64_t* probe_keys;
  int64_t n_probe;         /* < 2^31 */
  int32_t* out_probe_idx;
  int32_t* out_build_idx;
  int64_t* out_payload;
  int64_t out_capacity;
} rel_batch_join;

typedef struct {
  int32_t block;           /* threads per CTA: 128, 256 or 512 */
  int32_t items;           /* rows per thread per tile: 4, 8 or 16 */
  int32_t probe_width;     /* threads probing the global table together: 1, 2, 4, 8 */
  int32_t smem_max_groups; /* group-bys with est_groups <= this (at most 2048)
                              pre-aggregate each work item (up to 32 tiles) in
                              shared memory; 0 = none */
} rel_batch_config;

/* Host handle filled by rel_batch_prepare (opaque, caller-owned). */
typedef struct {
  uint64_t words[40];
} rel_batch_handle;

/* Device bytes the batch needs (descriptors, counters, every table). */
uint64_t rel_batch_ws_bytes(const rel_batch_groupby* gb, int32_t n_gb, const rel_batch_join* jn,
                            int32_t n_jn);

/* Validate, lay out and upload the batch (synchronises the stream once).
 * REL_E_INVALID for a bad instance or config, REL_E_UNSUPPORTED beyond a
 * limit, REL_E_CAPACITY when ws is too small. */
rel_status rel_batch_prepare(const rel_batch_groupby* gb, int32_t n_gb, const rel_batch_join* jn,
                             int32_t n_jn, const rel_batch_config* cfg, void* ws, size_t ws_bytes,
                             rel_batch_handle* handle, void* stream);

/* Zero the batch's tables and counters and run both launches on stream. */
rel_status rel_batch_run(const rel_batch_handle* handle, void* stream);

/* After a run: per instance (group-bys first, then joins) the number of
 * groups / pairs (even when larger than out_capacity) and a flag word: bit 0
 * table overflow (re-plan that instance larger), bit 1 output capacity
 * exceeded.  Synchronises the stream. */
rel_status rel_batch_results(const rel_batch_handle* handle, int64_t* n_out, uint32_t* flags,
                             void* stream);

/* Time each candidate config (one warm-up run, then `reps` runs, median) and
 * leave the fastest prepared in *handle and copied to *best; ms (host,
 * n_cands floats, may be NULL) receives every candidate's time, or -1 for a
 * candidate that failed validation. */
rel_status rel_batch_autotune(const rel_batch_groupby* gb, int32_t n_gb, const rel_batch_join* jn,
                              int32_t n_jn, const rel_batch_config* cands, int32_t n_cands,
                              int32_t reps, void* ws, size_t ws_bytes, rel_batch_handle* handle,
                              rel_batch_config* best, float* ms, void* stream);

/* ------------------------------------------------------------- sharding */

/* Sharded group-by across G ranks (one GPU each): every rank aggregates its
 * own rows (rel_groupby_agg), splits its partial groups by owner with this
 * call, exchanges them (an all-to-all of the per-owner ranges), and merges
 * the partials it owns with a second group-by (sum of sums, sum of counts,
 * min of mins, max of maxes).  The path shards the rows (the paper profiles
 * one GPU; its Sec. 6.1 notes multi-GPU underutilisation under skew); sum,
 * count, min and max are exact in int64, so the merged groups equal the
 * unsharded ones bit for bit.
 *
 * rel_shard_split: owner(k) = floor(h * world / 2^64), h = (k ^ 2^63) *
 * 0xD1B54A32D192ED03 mod 2^64 (a multiplier independent of the table
 * hashes).  Writes the n groups (keys[i], words[w][i]) to out_keys /
 * out_words grouped by owner -- owner 0's groups first, then owner 1's, ...;
 * order inside an owner's range unspecified -- and the number of groups per
 * owner to counts_host[world] (after a stream sync).  keys, words, outputs:
 * device int64 arrays of n; words / out_words: n_words (<= REL_MAX_AGGS)
 * device pointers (host arrays).  ws: rel_shard_ws_bytes(world) device bytes.
 * 1 <= world <= REL_SHARD_MAX_WORLD.  Returns REL_OK, REL_E_INVALID,
 * REL_E_UNSUPPORTED (world out of range), REL_E_CAPACITY (ws too small),
 * REL_E_CUDA. */
#define REL_SHARD_MAX_WORLD 64
uint64_t rel_shard_ws_bytes(int32_t world);
rel_status rel_shard_split(const int64_t* keys, const int64_t* const* words, int32_t n_words,
                           int64_t n, int32_t world, int64_t* out_keys, int64_t* const* out_words,
                           int64_t* counts_host, void* ws, size_t ws_bytes, void* stream);

/* ----------------------------------------------------------------- join */

/* Handle to a built join table.  It lives in caller memory, points into the
 * caller's workspace, and stays valid while that workspace is untouched. */
typedef struct {
  void* ws;
  int64_t slots;
  int64_t n_build;
  int32_t log2_slots;
  int32_t magic;
  uint64_t reserved[4];
} rel_join_table;

typedef struct {
  const rel_join_table* table;
  const int64_t* probe_keys; /* device, n_probe */
  int64_t n_probe;
} rel_join_probe_desc;

/* Device bytes rel_join_build needs for n_build build rows: a 256-byte
 * header, next_pow2(2 * n_build) (at least 16) slots of 16 bytes (key, build
 * row index), a copy of the payload column (8 bytes per build row, rounded up
 * to 256 bytes) from which the probe gathers, and a 16-byte side entry per
 * build row for the key INT64_MIN. */
uint64_t rel_join_ws_bytes(int64_t n_build);

/* Build (the paper's insert step): every build row j (key[j], payload[j])
 * enters an open-addressing table at load factor <= 1/2; duplicate keys are
 * kept as separate entries.  keys / payload: device int64[n_build];
 * 0 <= n_build <= 2^31 - 1.  ws >= rel_join_ws_bytes(n_build).  Fills *table.
 * Returns REL_OK, REL_E_INVALID, REL_E_UNSUPPORTED, REL_E_CUDA, REL_E_OVERFLOW. */
rel_status rel_join_build(const int64_t* keys, const int64_t* payload, int64_t n_build,
                          void* ws, size_t ws_bytes, rel_join_table* table, void* stream);

/* Probe (the paper's retrieve step, fused with the payload gather): emits one
 * row (probe_idx i, build_idx j, payload[j]) for every pair with
 * probe_keys[i] == key[j] -- the inner-join bag.  Outputs are device arrays of
 * out_capacity elements.  *n_pairs_host receives the pair count; REL_E_CAPACITY
 * when it exceeds out_capacity (outputs then hold an unspecified subset).
 * Probes on one table must not overlap on the GPU (they share a cursor). */
rel_status rel_join_probe(const rel_join_table* table, const int64_t* probe_keys,
                          int64_t n_probe, int32_t* out_probe_idx, int32_t* out_build_idx,
                          int64_t* out_payload, int64_t out_capacity, int64_t* n_pairs_host,
                          void* stream);

/* ---------------------------------------------------------- diagnostics */

/* Thread-local message for the last non-OK status on this thread. */
const char* rel_last_error(void);

/* Number of kernels this library has launched in this process. */
uint64_t rel_launch_count(void);

/* Library version, e.g. 100 for 0.1.0. */
int32_t rel_version(void);

/* Kernel timing for measurement.  rel_profile_start() clears the record and
 * makes every later kernel launch of this library record a CUDA event pair on
 * its own stream; rel_profile_stop() waits for those events, writes up to
 * `max` records in launch order (kernel id, milliseconds) and returns the
 * number of records taken (possibly > max), or -1 on a CUDA error.  Host
 * only; not thread-safe against concurrent launches from other threads. */
void rel_profile_start(void);
int64_t rel_profile_stop(int32_t* kernel_ids, float* ms, int64_t max);

/* Name of a kernel id reported by rel_profile_stop ("?" if unknown). */
const char* rel_kernel_name(int32_t kernel_id);

#ifdef __cplusplus
}
#endif

#endif /* REL_H */
