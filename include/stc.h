/*
 * stc.h -- C ABI of a GB300 (sm_103a) sparse COO tensor contraction library.
 *
 * The operation is the sparse tensor contraction of Swift (arXiv 2410.10094):
 *
 *     Z = X (x)_{cy}^{cx} Y,    z[fX, fY] = sum_c x[fX, c] * y[c, fY]     (Eq. 1, Eq. 2)
 *
 * X and Y are COO lists (Section 2.1.2); X mode cx[i] is paired with Y mode cy[i] and the
 * two must have equal lengths (Section 2.2). The output's modes are X's free modes in
 * ascending order followed by Y's free modes in ascending order (Eq. 4, Fig. 2), unless an
 * explicit output order permutes them.
 *
 * Conventions for every entry point:
 *   - Mode numbers are 0-based. Coordinates are int32, 0 <= coord < mode length.
 *   - "device" pointers are CUDA global memory on the context's device; "host" pointers
 *     are ordinary CPU memory read during the call only.
 *   - Work is enqueued on the stream argument (a cudaStream_t; NULL = legacy default
 *     stream). A call returns after its device work is complete unless stated otherwise.
 *   - Inputs stay owned by the caller and must stay valid until the call returns.
 *     Results are owned by the library and released with stc_result_free().
 *   - Every entry point returns a stc_status; nothing throws across the ABI. On failure a
 *     message for the calling thread is available from stc_last_error().
 *   - Floating point is FP64 (IEEE binary64): products are rounded before they are added
 *     (no fused multiply-add), sums are accumulated in binary64 in an unspecified order.
 */
#ifndef STC_H
#define STC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum stc_status {
  STC_OK = 0,
  STC_ERR_INVALID_ARG = 1,        /* null pointer, bad order, bad mode list, bad permutation */
  STC_ERR_SHAPE_MISMATCH = 2,     /* paired modes have different lengths (Section 2.2) */
  STC_ERR_KEY_OVERFLOW = 3,       /* a key space (product of mode lengths) needs > 64 bits */
  STC_ERR_OUT_OF_MEMORY = 4,      /* device allocation failed or the context budget is exceeded */
  STC_ERR_TABLE_FULL = 5,         /* an accumulation table overflowed (internal: retried, see stc_opts) */
  STC_ERR_TIMEOUT = 6,            /* a bounded wait gave up */
  STC_ERR_CUDA = 7,               /* a CUDA runtime call failed; see stc_last_error() */
  STC_ERR_COORD_OUT_OF_RANGE = 8, /* an input coordinate is negative or >= its mode length */
  STC_ERR_UNSUPPORTED = 9,        /* valid input outside what the library implements */
  STC_ERR_CANCELLED = 10          /* a queued server request was cancelled (stc_server_cancel) */
} stc_status;

#define STC_MAX_ORDER 8            /* modes per input tensor */
#define STC_MAX_NNZ 2147483647LL   /* entries per input tensor (int32 positions) */

typedef struct stc_ctx stc_ctx;
typedef struct stc_result stc_result;

/* A sparse tensor in key form: each entry's row-major linear index over `shape` (the last
 * mode fastest) instead of its coordinates, e.g. a result made with stc_opts.output_keys. */
typedef struct stc_keyed {
  int32_t order;          /* number of modes, 1..STC_MAX_ORDER */
  const int64_t* shape;   /* host, [order] */
  int64_t nnz;            /* 0..STC_MAX_NNZ */
  const uint64_t* keys;   /* device, [nnz], each < prod(shape) */
  const double* vals;     /* device, [nnz] */
} stc_keyed;

/* A COO tensor (Section 2.1.2): nnz (coordinate, value) pairs. Repeated coordinates are
 * allowed and are additive. */
typedef struct stc_coo {
  int32_t order;          /* number of modes, 0..STC_MAX_ORDER */
  const int64_t* shape;   /* host, [order], each >= 1 */
  int64_t nnz;            /* 0..STC_MAX_NNZ */
  const int32_t* coords;  /* device, [nnz][order] row-major; may be NULL when nnz == 0 */
  const double* vals;     /* device, [nnz]; may be NULL when nnz == 0 */
} stc_coo;

/* Accumulation strategy. AUTO picks from the key spaces and sizes: one global table when the
 * output key space is small (the whole table stays in L2) or when X has far fewer entries than
 * free keys (more than about two free keys per entry, sixteen when n_Y >= 16 K), otherwise
 * per-X-free-group tables in shared memory (Section 4.3). */
enum { STC_STRATEGY_AUTO = 0, STC_STRATEGY_GLOBAL = 1, STC_STRATEGY_GROUPED = 2 };

/* Per-group accumulator of the GROUPED strategy. HASH: a probing table sized from the
 * group's bound (Section 4.3); where keys and output positions fit 32 bits, each output is
 * written as soon as its key is first claimed. HASH_SCAN: the same table, accumulated in
 * shared memory and written by a scan of the table after the group. DENSE: the group's output
 * row swept in segments of 2^16 Y free keys; the keys present are found with a bitmap over the
 * segment (no hashing or probing), products are stashed in shared memory and repeated keys
 * folded into their first product (F_Y at most 2^20). ROWS: for output rows of at most 64 Y
 * free keys that receive many products each (both operands' contract keys skewed): one warp
 * per group, each lane adding its products into a private dense row in shared memory without
 * atomics, the rows summed in lane order at the end (F_Y at most 64, else
 * STC_ERR_INVALID_ARG). AUTO: ROWS when F_Y <= 64 and the products average at least 64 per
 * output cell; otherwise DENSE for the groups larger than the warp-sized hash tables when
 * F_Y <= 2^20, HASH for the others. */
enum { STC_ACC_AUTO = 0, STC_ACC_HASH = 1, STC_ACC_DENSE = 2, STC_ACC_HASH_SCAN = 3, STC_ACC_ROWS = 4 };

/* Contract keys (Section 4.1.2). DIRECT: Y is grouped over the K = prod(paired lengths)
 * contract keys themselves (counting sort over K bins). DENSE: the contract keys of Y are
 * first renumbered 0..D-1 and X and Y are rewritten with the id in place of their paired modes
 * (as stc_dense_ids does); stats.contract_ids = D. AUTO: DENSE when K > 2^26 (always, since
 * direct counting stops there) or when K exceeds both 2^22 and 8 (nX + nY); DIRECT otherwise.
 * A DIRECT request with K > 2^26 is renumbered too. */
enum { STC_IDS_AUTO = 0, STC_IDS_DIRECT = 1, STC_IDS_DENSE = 2 };

/* Operand roles. Y is the tensor grouped by contract key (the array of Section 4.2), X the one
 * streamed against it and grouped by free key. Eq. 2 gives the same output with the operands
 * swapped and the output modes permuted back, and the paper's cost (Section 4.4: a processing
 * term, nnz_X x cmode_Yavg and nnz_Z) is symmetric, as its Set 3 swap experiment shows
 * (Section 5.4); on the device the grouping of Y costs more per entry than the survey of X. AUTO therefore swaps
 * when Y has more than four times X's entries; AS_GIVEN never swaps; SWAPPED always does.
 * stats.swapped records the choice. */
enum { STC_OPERANDS_AUTO = 0, STC_OPERANDS_AS_GIVEN = 1, STC_OPERANDS_SWAPPED = 2 };

typedef struct stc_opts {
  int32_t strategy;       /* STC_STRATEGY_*; 0 = AUTO */
  int32_t record_times;   /* nonzero: time each stage with CUDA events (stc_result_stats) */
  double load_factor;     /* global-table load factor in (0, 0.9]; 0 = default 0.5 */
  double group_load_factor; /* largest load of a per-group shared-memory table, in (0, 0.9];
                               0 = default 0.75. A group of bound t goes to the smallest table
                               class with t <= group_load_factor * slots. */
  int32_t accumulator;    /* STC_ACC_*; 0 = AUTO */
  int32_t contract_ids;   /* STC_IDS_*; 0 = AUTO */
  int32_t operands;       /* STC_OPERANDS_*; 0 = AUTO */
  int32_t table_shrink;   /* fault injection, normally 0: the first attempt of the one-global-table
                             strategy divides its table's capacity (sized from the exact product
                             count, Section 4.3) by 2^table_shrink (0..30). A table too small for
                             the distinct output keys overflows; the call sees the overflow
                             (STC_ERR_TABLE_FULL inside the call), discards that attempt and runs
                             the expansion again with the full capacity; stats.retries counts it. */
  int32_t output_keys;    /* nonzero: the result holds each output entry's key (its row-major linear
                             index over the output shape, uint64) instead of its coordinates, for
                             the next contraction of a chain (stc_contract_keyed); needs the
                             output modes in concatenation order (out_order NULL or identity);
                             stc_contract and stc_contract_keyed only */
  int32_t probe;          /* one-global-table strategy: lanes that probe the table together.
                             0 = AUTO; 1 = every lane probes its own key over single slots
                             (linear probing, Section 2.3.1); 4 or 8 = warp-cooperative probing:
                             tiles of that many lanes take their keys in turn and read buckets of
                             that many consecutive slots, one slot per lane, with one ballot for
                             the key and one for the first free slot. Other values:
                             STC_ERR_INVALID_ARG. */
} stc_opts;

/* Per-call statistics of a finished contraction. */
typedef struct stc_stats {
  uint64_t products;      /* P = number of (x, y) pairs with equal contract coordinates */
  uint64_t survivors;     /* X entries whose contract key has at least one Y entry */
  uint64_t out_capacity;  /* output entries allocated (an upper bound on nnz) */
  uint64_t table_slots;   /* global-table slots (GLOBAL) or overflow-table slots (GROUPED) */
  uint64_t groups;        /* non-empty X free groups (GROUPED) */
  int32_t strategy;       /* STC_STRATEGY_GLOBAL or STC_STRATEGY_GROUPED */
  int32_t nstages;        /* valid entries of stage_ms when record_times was set */
  uint32_t launches;      /* CUDA kernels this call launched (memsets and copies not counted) */
  int32_t accumulator;    /* GROUPED: STC_ACC_HASH or STC_ACC_DENSE when every group used that
                             accumulator, STC_ACC_AUTO when both ran, STC_ACC_ROWS for the
                             lane-private dense rows */
  float stage_ms[8];      /* 0 group Y, 1 survey X, 2 group X, 3 plan, 4 accumulate, 5 compact/write */
  uint64_t contract_ids;  /* distinct contract keys of Y when the contract keys were renumbered
                             to dense ids (STC_IDS_DENSE), else 0 */
  int32_t swapped;        /* 1 when the operands were swapped (STC_OPERANDS_*) */
  int32_t retries;        /* expansions run again after a table overflowed (see stc_opts.table_shrink) */
} stc_stats;

/* Human-readable name of a status code (static storage). */
const char* stc_status_string(stc_status s);

/* Last error message of the calling thread ("" if none). Valid until the thread's next call. */
const char* stc_last_error(void);

/* Create a context on CUDA device `device`. `mem_budget_bytes` caps the device memory the
 * context may hold at once for scratch and results (0 = no cap beyond the device's). The
 * context owns a stream-ordered memory pool; freed blocks are kept for reuse. */
stc_status stc_create(stc_ctx** ctx, int device, size_t mem_budget_bytes);

/* Destroy a context. All results created from it must have been freed. */
stc_status stc_destroy(stc_ctx* ctx);

/* Contract X and Y (Eq. 2). Arguments:
 *   X, Y        input tensors (device coordinate and value arrays, host shapes)
 *   ncontract   number of paired modes m, 0 <= m <= min(X.order, Y.order); m = 0 is the
 *               outer product, m = order of both gives an order-0 (scalar) output
 *   cx, cy      host, [m]; X mode cx[i] pairs with Y mode cy[i]; the lists order the
 *               contract key (first listed mode most significant, Section 2.4.1)
 *   out_order   host, [orderZ] or NULL; output mode q holds entry out_order[q] of the
 *               concatenation (X free modes ascending, Y free modes ascending)
 *   opts        host or NULL (defaults)
 *   stream      cudaStream_t the work is enqueued on
 *   out         receives the result
 * Output: every coordinate that received at least one product, once, with the sum of its
 * products (a structural nonzero is kept even if it sums to 0.0), in unspecified order.
 * Large contract key spaces are first renumbered to dense ids (opts.contract_ids, Section
 * 4.1.2): stats.contract_ids then holds the number of distinct contract keys of Y, which
 * must stay below 2^26 (else UNSUPPORTED).
 * Errors: INVALID_ARG, SHAPE_MISMATCH, KEY_OVERFLOW (output key space > 2^64 - 2),
 * COORD_OUT_OF_RANGE (checked on the device), OUT_OF_MEMORY, UNSUPPORTED, CUDA. */
stc_status stc_contract(stc_ctx* ctx, const stc_coo* X, const stc_coo* Y, int32_t ncontract,
                        const int32_t* cx, const int32_t* cy, const int32_t* out_order,
                        const stc_opts* opts, void* stream, stc_result** out);

/* Device bytes the context holds now (scratch of calls in flight + live results) and the
 * number of live results. held_bytes and live_results may be NULL. */
stc_status stc_ctx_stats(const stc_ctx* ctx, uint64_t* held_bytes, int64_t* live_results);

/* One contraction of a batch: the arguments of stc_contract. */
typedef struct stc_problem {
  stc_coo X;
  stc_coo Y;
  int32_t ncontract;
  const int32_t* cx;        /* host, [ncontract] */
  const int32_t* cy;        /* host, [ncontract] */
  const int32_t* out_order; /* host or NULL */
} stc_problem;

/* Contract n independent problems together (each exactly as stc_contract would). The batch
 * shares every pass: Y of all problems is grouped in one counting sort over the concatenated
 * contract-key bins, X of all problems is surveyed once, its entries are grouped by
 * (problem, X free key) through one probing table that gives each pair a small number
 * (Section 4.1.2), and one launch per table class accumulates the groups of all problems
 * (small groups one warp each). outs: host, [n], receives one result per problem; the
 * results share one device allocation that is released when the last of them is freed.
 * Limits: the batch's total nnz of X and of Y each at most STC_MAX_NNZ, the sum of the
 * contract key spaces at most 2^26. Errors as stc_contract; on error no result is returned. */
stc_status stc_contract_batch(stc_ctx* ctx, int32_t n, const stc_problem* problems, const stc_opts* opts,
                              void* stream, stc_result** outs);

/* A prepared batch: the problems of stc_contract_batch held by the library across runs, for a
 * batch run again and again on the same device arrays (their contents may change between
 * runs; the arrays themselves, shapes and mode lists may not). The plan keeps the problems'
 * descriptors and every scratch array on the device. Its first runs are ordinary batches
 * (with stc_opts.group_load_factor 0 they also let the context's autotuner time each of its
 * candidates for the batch's size bucket: load factor, group-per-warp granularity, expansion
 * split); once the choice is settled the
 * whole launch sequence of one run (grouping of Y, survey and grouping of X, binning,
 * placement of every problem's output from its exact bound, accumulation) is captured in one
 * CUDA graph, and every later run replays it: one output allocation of the previous run's
 * exact size, one graph launch, one wait. A run whose outputs outgrow that size is run again
 * the ordinary way (and captured anew). Runs of one plan must not overlap.
 *   stc_batch_plan_create: n >= 1 problems (host arrays copied, device arrays borrowed for
 *     the plan's lifetime); opts as stc_contract_batch.
 *   stc_batch_plan_run: outs host [n], one result per problem, sharing one device block as
 *     stc_contract_batch's do; returns after the run's device work completes.
 *   stc_batch_plan_stats: runs so far, runs that replayed the graph, and the choice the graph
 *     was captured with (0s before a capture): the group load factor, the largest table a
 *     group gets in a warp of its own (256 or 1024 slots; larger groups take a CTA), and the
 *     expansion split (0: the default products per lane per round, 1: half as many). Each
 *     pointer may be NULL.
 * Errors: as stc_contract_batch; INVALID_ARG for NULL arguments or n < 1. */
typedef struct stc_batch_plan stc_batch_plan;
stc_status stc_batch_plan_create(stc_ctx* ctx, int32_t n, const stc_problem* problems, const stc_opts* opts,
                                 stc_batch_plan** out);
stc_status stc_batch_plan_run(stc_batch_plan* plan, void* stream, stc_result** outs);
stc_status stc_batch_plan_stats(const stc_batch_plan* plan, int64_t* runs, int64_t* graph_runs,
                                double* group_load_factor, int32_t* warp_table_max, int32_t* expansion_depth);
stc_status stc_batch_plan_destroy(stc_batch_plan* plan);

/* ---------------------------------------------------------------- serving
 * A server takes contraction requests as they arrive and runs them on worker threads, each
 * with its own CUDA stream. Counting threads (one per worker, each on a stream of its own)
 * compute each request's exact device-memory bound (from the product count of Section 4.3),
 * taking requests in arrival order;
 * the request is then admitted against the server's budget: queued requests that fit are run
 * together as one stc_contract_batch by the next free worker, so requests that arrive while
 * others run join the next batch and batches of different workers overlap on the device
 * (continuous batching). With `plain` set, one worker runs one request at a time with
 * stc_contract: the one-at-a-time baseline. */
typedef struct stc_server stc_server;

typedef struct stc_server_opts {
  uint64_t mem_budget_bytes; /* admission budget for requests in flight; 0 = no limit */
  int32_t max_batch;         /* most requests per batch; 0 = no limit */
  int32_t workers;           /* worker threads (streams); 0 = 2 */
  int32_t plain;             /* nonzero: one request per launch, one worker (baseline) */
  int32_t reserved_;
} stc_server_opts;

/* Create a server on ctx's device; the calling thread's current device must be ctx's. */
stc_status stc_server_create(stc_ctx* ctx, const stc_server_opts* opts, stc_server** out);

/* Queue a request. Its device arrays must stay valid and unchanged until the request is
 * finished (its wait has returned); its host arrays (shapes, mode lists) are copied. Returns
 * at once: the counting pass that sizes the request runs on one of the server's counting threads, and
 * an error it finds (a bad argument, a coordinate out of range) is the request's status at
 * its wait. ticket receives the request's id. */
stc_status stc_server_submit(stc_server* s, const stc_problem* request, uint64_t* ticket);

/* done receives 1 when the request has finished (successfully or not), else 0. */
stc_status stc_server_poll(stc_server* s, uint64_t ticket, int32_t* done);

/* Wait up to timeout_ms (negative: no limit) for a request and take its result (the caller
 * frees it with stc_result_free, which may happen after the server is destroyed; its memory
 * then goes back on the legacy default stream, so work reading it must be finished). times: host, [3] or NULL, receives the request's submit,
 * start and finish times in seconds since the server was created. STC_ERR_TIMEOUT if the
 * request is still running (the ticket stays valid); otherwise the ticket is consumed and the
 * request's own status is returned. */
stc_status stc_server_wait(stc_server* s, uint64_t ticket, int64_t timeout_ms, stc_result** out, double* times);

/* Cancel a request that no worker has taken yet: it never runs, and its wait returns
 * STC_ERR_CANCELLED (consuming the ticket; if its counting pass was running, the wait returns
 * once that pass has finished with the request's arrays). cancelled receives 1 when the
 * request was cancelled, 0 when a worker had already taken it (it then finishes normally) or
 * it had finished. Errors: INVALID_ARG (NULL server or cancelled, unknown ticket). */
stc_status stc_server_cancel(stc_server* s, uint64_t ticket, int32_t* cancelled);

/* Finish every queued request, stop the workers, free uncollected results, destroy. */
stc_status stc_server_destroy(stc_server* s);

/* The exact product count of the contraction (Section 4.3: each X entry meets exactly
 * count_Y[its contract key] Y entries) and the device bytes a stc_contract of the same
 * inputs with default options would hold at its peak (scratch + result), for the operand
 * order and contract-key handling AUTO picks. Used to admit work under a budget.
 * products, bytes_bound: host, each may be NULL. Returns after its device work completes.
 * Errors: as stc_contract. */
stc_status stc_count(stc_ctx* ctx, const stc_coo* X, const stc_coo* Y, int32_t ncontract,
                     const int32_t* cx, const int32_t* cy, void* stream, uint64_t* products,
                     uint64_t* bytes_bound);

/* LN keys of the listed modes of every entry of T (Section 2.4.1, Fig. 3): the coordinates
 * of modes[0..nmodes) read as digits of one mixed-radix number, modes[0] most significant,
 * each digit's radix its mode length. keys_out: device, [T.nnz], written. Returns after its
 * device work completes. Errors: INVALID_ARG (NULL pointers, a mode listed twice or out of
 * range), KEY_OVERFLOW (the listed lengths multiply past 2^64), COORD_OUT_OF_RANGE, CUDA. */
stc_status stc_linearize(stc_ctx* ctx, const stc_coo* T, int32_t nmodes, const int32_t* modes,
                         uint64_t* keys_out, void* stream);

/* Group n keys in [0, k) with a counting sort (Section 4.1.1, Fig. 6): count, exclusive
 * scan, scatter. offsets_out: device, [k+1], offsets_out[v] = first slot of key v and
 * offsets_out[k] = n. perm_out: device, [n], perm_out[s] = index of the key placed in
 * slot s; the order inside one key's run is unspecified. keys: device, [n]. Requires
 * n <= STC_MAX_NNZ and k <= 2^26 (larger k: UNSUPPORTED; renumber with stc_dense_ids first).
 * Returns after its device work completes. Errors: INVALID_ARG, COORD_OUT_OF_RANGE (a key
 * >= k), OUT_OF_MEMORY, UNSUPPORTED, CUDA. */
stc_status stc_group_keys(stc_ctx* ctx, const uint64_t* keys, int64_t n, uint64_t k,
                          uint32_t* offsets_out, uint32_t* perm_out, void* stream);

/* Small numbers for large keys (Section 4.1.2, Fig. 7): ids_out[i] = the dense id of
 * keys[i], with ids in [0, D), equal keys sharing one id and distinct keys distinct ids,
 * where D = the number of distinct keys, written to *ndistinct. Every 64-bit value is a
 * valid key. Which key gets which id is unspecified (the paper numbers keys in order of
 * first sight; here they are numbered in the order of their hash-table slots), so ids
 * feed stc_group_keys with k = D.
 *   keys: device, [n], read only; ids_out: device, [n], written; ndistinct: host.
 *   n <= STC_MAX_NNZ; the call allocates a table of about 64 n bytes from the context and
 *   returns after its device work completes (it reads D back).
 * Errors: INVALID_ARG (NULL pointer, n out of range), OUT_OF_MEMORY, CUDA. */
stc_status stc_dense_ids(stc_ctx* ctx, const uint64_t* keys, int64_t n, uint32_t* ids_out,
                         uint64_t* ndistinct, void* stream);

/* stc_group_keys without allocation. The paper has no counterpart: this entry point exists
 * for callers that must not allocate device memory, for example a process whose device memory
 * is already fully carved up by its own allocator, or a loop that forbids allocation after
 * start-up. It performs the same counting sort as stc_group_keys, with the same arguments
 * and results, but takes no context and calls no allocator: its scratch (key counts, a
 * cursor copy, scan partials and a status word) is one fixed array of about 2 MB in device
 * memory that every device loading this library holds until the process exits.
 *   - Limit: k <= 262144 (2^18) and n <= STC_MAX_NNZ; a larger k returns
 *     STC_ERR_INVALID_ARG with a message naming the limit.
 *   - It runs on the caller's current device. The first call on a device looks up the
 *     array's device address (set-up). If the look-up fails the call returns STC_ERR_CUDA
 *     and the next call tries again.
 *   - No call can be captured into a CUDA graph: every call reads its status word back to
 *     the host and waits for its stream (below).
 *   - All calls on a device share the one array. The call clears what must start at zero,
 *     but calls whose work overlaps on the GPU (other streams, other host threads) race on
 *     it: serialise them.
 *   - Every call copies its status word to the host and waits for its stream before it
 *     returns; it reports STC_ERR_COORD_OUT_OF_RANGE for a key >= k, as stc_group_keys
 *     does. */
stc_status stc_group_keys_static(const uint64_t* keys, int64_t n, uint64_t k, uint32_t* offsets_out,
                                 uint32_t* perm_out, void* stream);

/* Measured peak rates of the device's FP64 multiply pipe and of FP64 atomic adds resolved in
 * L2 (measurement support; the paper has no counterpart: its CPU program has no such limits to
 * report). Contractions whose products mostly fall on few outputs (both operands' contract
 * keys skewed) are bound by these rather than by memory bandwidth.
 *   dmul_per_s: rounded FP64 multiplies per second, from independent multiply chains filling
 *     every SM; l2_atomic_per_s: FP64 atomicAdd per second to hashed slots of an 8 MB array
 *     (resident in L2). Either may be NULL. Each is timed with CUDA events after one warm-up
 *     launch, on a private stream of `device`; the call takes tens of milliseconds and
 *     restores the calling thread's current device.
 * Errors: INVALID_ARG (both NULL, bad device), CUDA. */
stc_status stc_measure_peaks(int device, double* dmul_per_s, double* l2_atomic_per_s);

/* Result accessors. Coordinates are device int32 [nnz][order] row-major, values device
 * double [nnz]; both stay valid until stc_result_free(). shape is host, [order]. */
stc_status stc_result_info(const stc_result* r, int64_t* nnz, int32_t* order, const int64_t** shape);
stc_status stc_result_data(const stc_result* r, const int32_t** coords, const double** vals);
stc_status stc_result_stats(const stc_result* r, stc_stats* stats);
stc_status stc_result_free(stc_result* r);

/* A view of a result as an input tensor, for chains of contractions (the output of one
 * feeding the next, as in Section 5.4's motivation): out->coords, vals and shape point into
 * the result (device, device and host memory), valid until stc_result_free(r). Nothing is
 * copied. out: host, written. Errors: INVALID_ARG when r or out is NULL. */
stc_status stc_result_as_coo(const stc_result* r, stc_coo* out);

/* Results made with stc_opts.output_keys: the output keys (device uint64 [nnz], valid until
 * stc_result_free) and a key-form view of the result for the next contraction of a chain.
 * keys receives NULL for a result in coordinate form; stc_result_as_keyed returns INVALID_ARG
 * for one. */
stc_status stc_result_keys(const stc_result* r, const uint64_t** keys);
stc_status stc_result_as_keyed(const stc_result* r, stc_keyed* out);

/* Z = X (x) Y (Eq. 2) with X given in key form, as the output of an earlier contraction is
 * handed to the next one of a chain without being turned into coordinates (the chains of
 * contractions of Section 5.4). X's contracted modes must be a contiguous block at the end of
 * its modes (cx[i] = X.order - m + i) or at the start (cx[i] = i): each key then splits, by one
 * division, into its free part (already the row-major index over X's free modes, carried into
 * the output key as it is) and its contract part, whose m digits pair with Y's modes cy. The
 * operands keep their roles (no swap) and the contract key space must fit direct counting
 * (at most 2^26 keys). Output, options (output_keys included) and errors as stc_contract;
 * INVALID_ARG also for a contract block that is not contiguous at an end of X's modes. */
stc_status stc_contract_keyed(stc_ctx* ctx, const stc_keyed* X, const stc_coo* Y, int32_t ncontract,
                              const int32_t* cx, const int32_t* cy, const int32_t* out_order, const stc_opts* opts,
                              void* stream, stc_result** out);

#ifdef __cplusplus
}
#endif

#endif /* STC_H */
