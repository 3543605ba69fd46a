/*
 * pccp.h -- C ABI of the GB300 (sm_103a) PCCP propagate-and-search library.
 *
 * The method: a constraint model is compiled to guarded commands over a store
 * of integer intervals (the lattice IZ = ZInc x ZDec, paper Sec. 2; the
 * guarded normal form of Sec. 3, Prop. 3).  Propagation joins every command's
 * tell into the store until nothing changes (the least fixed point of
 * Theorem 1, reached by any fair order: Def. 4 and the fix D = fix O
 * theorem).  On the GPU the commands of one store run concurrently with no
 * locks; every tell is an atomic max on a lower bound or an atomic min on an
 * upper bound in shared memory (the load/store semantics of Sec. 4, whose
 * soundness and completeness theorems make the result independent of the
 * interleaving).  Search is propagate-and-branch with full recomputation from
 * a root store (Sec. 5, "Turbo").
 *
 * Conventions for every call:
 *  - Return 0 (PCCP_OK) on success and a negative PCCP_ERR_* code otherwise;
 *    pccp_error_string() names the code.  No call aborts the process.
 *  - Host pointers are read during the call only; the caller keeps ownership.
 *    Device pointers stay owned by the caller and must stay valid until the
 *    work queued on the stream has finished.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  The work runs on the device that is current at the call, which
 *    must be the device the model was created on.
 *  - All values are int32.  Variable indices are 0-based.
 */
#ifndef PCCP_H
#define PCCP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define PCCP_OK 0
#define PCCP_ERR_INVALID (-1)  /* bad argument: index out of range, lb0 > ub0, empty
                                  linear row, reified b not Boolean, NULL pointer ... */
#define PCCP_ERR_OVERFLOW (-2) /* some intermediate of a propagator could leave int32 */
#define PCCP_ERR_SMEM (-3)     /* model (table + stores) does not fit shared memory */
#define PCCP_ERR_TIMEOUT (-4)  /* a device-side wait or iteration budget ran out */
#define PCCP_ERR_CUDA (-5)     /* a CUDA runtime call failed */
#define PCCP_ERR_UNSUPPORTED (-6) /* valid model outside this build's packed limits
                                     (> 65535 variables, |coef| > 32767, ...) */
#define PCCP_ERR_SCRATCH (-7)  /* request larger than the fixed scratch of the
                                  allocation-free entry point */

/* ---- per-store status written by pccp_propagate ------------------------ */
#define PCCP_FIXPOINT 0 /* lb/ub hold the least fixed point */
#define PCCP_FAILED 1   /* some interval became empty; lb/ub contents unspecified */
#define PCCP_ERROR 2    /* iteration budget exhausted; lb/ub contents unspecified */

/* ---- model ------------------------------------------------------------- */

/* A constraint model: the PCCP program of one problem instance (Sec. 2).
 *
 * Variables 0..n_vars-1 have root domains [lb0[v], ub0[v]] (lb0 <= ub0).
 * Three row kinds, each compiled to guarded commands:
 *   temporal  {x, y, d}      : x + d <= y.  The compilation [[x + y <= c]] of
 *                              Sec. 2 with y negated: ub(x) <= ub(y) - d and
 *                              lb(y) >= lb(x) + d.
 *   linear    c, terms       : sum_k coef_k * var_k <= c.  The resource-sum
 *                              compilation of Sec. 2, generalised to any
 *                              coefficient sign: each term is bounded by c
 *                              minus the minimum of the other terms
 *                              (the term itself is excluded from that sum).
 *                              Rows are CSR: terms linear_off[i] ..
 *                              linear_off[i+1]-1; zero coefficients are dropped;
 *                              a row must keep at least one term.
 *   reified   {b, x, y, d}   : b <=> (x <= y and y < x + d), the overlap Booleans
 *                              of the scheduling model (Sec. 2), compiled as the
 *                              four asks of [[phi <=> psi]]; b's root domain must
 *                              lie within [0, 1].
 * objective: variable minimised by pccp_solve (-1: stop at the first solution).
 * branch_vars: variables search branches on, in input order.
 * All arrays are host memory, copied by pccp_model_create.                 */
typedef struct {
  int32_t n_vars;
  const int32_t* lb0;        /* [n_vars] */
  const int32_t* ub0;        /* [n_vars] */
  int32_t n_temporal;
  const int32_t* temporal;   /* [n_temporal][3] = {x, y, d} */
  int32_t n_linear;
  const int32_t* linear_c;   /* [n_linear] */
  const int32_t* linear_off; /* [n_linear + 1], linear_off[0] = 0 */
  const int32_t* term_coef;  /* [linear_off[n_linear]] */
  const int32_t* term_var;   /* [linear_off[n_linear]] */
  int32_t n_reified;
  const int32_t* reified;    /* [n_reified][4] = {b, x, y, d} */
  int32_t objective;
  int32_t n_branch;
  const int32_t* branch_vars; /* [n_branch] */
  int32_t bool_store;  /* how the stores keep Boolean variables that appear only as
                          reified b's and in all-positive 0/1 linear rows: 1 as
                          bits (two bits of a shared 64-bit word each, 32 x
                          smaller stores; the table is then read from global
                          memory), -1 as intervals, 0 the library's choice (bits
                          only when an interval store would not fit in shared
                          memory).  Results are the same. */
} pccp_model_desc;

typedef struct pccp_model pccp_model; /* opaque; owns a device copy of the table */

/* Validates `desc`, packs its rows into the structure-of-arrays propagator
 * table (the guarded normal form of Sec. 3) and copies it to the current
 * device (synchronously).  The library may keep the variables in shared
 * memory in an order of its own (pccp_model_info.reordered); every array a
 * call reads or writes stays in the order of `desc`.  On success *out
 * receives a model that must be released with pccp_model_destroy.  Errors:
 * INVALID, OVERFLOW, UNSUPPORTED, CUDA (then *out is NULL). */
int pccp_model_create(const pccp_model_desc* desc, pccp_model** out);

/* Frees the model, its device table and the buffers of pccp_propagate_host
 * (synchronises the device first).  No call on the model may be in progress.
 * NULL is accepted. */
void pccp_model_destroy(pccp_model* model);

/* Sizes of a created model, for planning buffers and roofline accounting. */
typedef struct {
  int32_t n_vars;
  int32_t n_temporal, n_linear, n_terms, n_reified;
  int32_t table_bytes;      /* packed table, copied to shared memory per CTA when it
                               fits beside a store (else read from global memory) */
  int64_t bytes_per_sweep;  /* algorithmic bytes of one evaluation of every row:
                               temporal 20, reified 40, linear 12 + 12 * len */
  int32_t max_store_vars;   /* largest n_vars a single CTA can stage beside the table
                               (stores of more variables read the table from global
                               memory, down to the shared-memory limit of one store) */
  int32_t n_segments;       /* byte ranges of whole rows (<= 32 KB each) that one sweep
                               streams when the table is read from global memory */
  int32_t reordered;        /* 1: the library keeps the variables in shared memory in
                               its own order (chosen at create for fewer bank conflicts;
                               every array the caller sees stays in the caller's order) */
  int32_t bool_vars;        /* Booleans kept as bits (see pccp_model_desc.bool_store) */
  int32_t store_bytes;      /* shared memory of one store: 8 B per other variable and
                               8 B per 32 Booleans kept as bits */
  int32_t temporal_levels;  /* topological levels of the temporal rows (the longest
                               chain of rows), 0 when they have a cycle (see
                               pccp_launch_config.temporal_levels) */
} pccp_model_info;

int pccp_model_get_info(const pccp_model* model, pccp_model_info* info);

/* ---- propagation ------------------------------------------------------- */

/* Propagates a batch of stores to their least fixed points, in place.
 *   lb, ub     : DEVICE int32 arrays [n_stores][n_vars] (row-major).  Each
 *                store is first joined with the model's root domains; the
 *                result is the least fixed point above that (Theorem 1).
 *   status     : DEVICE int32 [n_stores]: PCCP_FIXPOINT / PCCP_FAILED /
 *                PCCP_ERROR.  lb/ub of a non-FIXPOINT store are unspecified.
 *   iterations : DEVICE int32 [n_stores] or NULL: fixed-point iterations run
 *                for each store (with the table in shared memory every row
 *                is evaluated once per iteration, the eventless loop of
 *                Sec. 5; see skip_stable in pccp_launch_config).
 *   n_stores   : >= 0 (0 queues nothing).
 * Asynchronous on `stream`.  Errors: INVALID, SMEM, CUDA.
 * Calls on one model may run concurrently on different streams. */
int pccp_propagate(const pccp_model* model, int32_t n_stores, int32_t* lb, int32_t* ub,
                   int32_t* status, int32_t* iterations, void* stream);

/* Launch shape of the propagation kernel.  A team (team_threads threads, whole
 * warps) owns one store at a time; a CTA holds one copy of the propagator
 * table in shared memory and teams_per_cta team stores.  Zero fields take the
 * library's defaults.  The result does not depend on the shape (any fair
 * interleaving reaches the same fixed point, Sec. 3). */
typedef struct {
  int32_t team_threads;   /* 32..1024, multiple of 32 */
  int32_t teams_per_cta;  /* 1..15 (team_threads * teams_per_cta <= 1024) */
  int32_t ctas_per_sm;    /* cap on resident CTAs per SM used for the grid */
  int32_t max_iterations; /* per-store iteration budget (exceeded: PCCP_ERROR) */
  int32_t skip_stable;    /* 1: re-run a row only after one of its variables changed
                             (change bitmaps per team; Sec. 6); -1: the eventless loop
                             of Sec. 5; 0: the library's choice (on for tables read
                             from global memory, off for tables in shared memory).
                             Same fixed point either way. */
  int32_t stream_table;   /* tables too large for shared memory: 0 read rows in place
                             (through L1/L2); 1 stream them through a ring of
                             shared-memory buffers by TMA bulk copies, segment by
                             segment, every sweep.  Same fixed point either way. */
  int32_t temporal_levels; /* models whose temporal rows x + d <= y form an acyclic
                              graph: 1 two warps of a team carry the bounds along
                              its chains in one pass each sweep (rows grouped by
                              topological level of x: lower bounds in increasing
                              levels, upper bounds in decreasing ones); -1 a thread
                              per row, which moves a bound one row per sweep; 0 the
                              library's choice (levels in propagation; in searches
                              only for tables read from global memory).  Same fixed
                              point either way (Sec. 3). */
} pccp_launch_config;

/* pccp_propagate with an explicit launch shape (cfg may be NULL) and an
 * optional work report: work is NULL or a DEVICE int32 [n_stores][2]
 * receiving, per store, the rows evaluated and the algorithmic bytes they
 * read (rows, operand bounds, change-tracking words).  With
 * cfg->skip_stable, rows whose variables did not change since their last
 * evaluation are not evaluated again (skipping stable propagators, Sec. 6);
 * the fixed point is unchanged.  Returns PCCP_ERR_SMEM if the requested
 * teams do not fit shared memory. */
int pccp_propagate_ex(const pccp_model* model, int32_t n_stores, int32_t* lb, int32_t* ub,
                      int32_t* status, int32_t* iterations, int32_t* work,
                      const pccp_launch_config* cfg, void* stream);

/* pccp_propagate for stores that live in HOST memory: lb, ub are HOST int32
 * [n_stores][n_vars], updated in place with the fixed points; status and
 * iterations (may be NULL) are HOST int32 [n_stores].  Two ways to move the
 * stores, chosen by chunk_stores:
 *   > 0                : chunked copies, chunk_stores stores per chunk;
 *   0                  : chunked copies: a first chunk of one store per
 *                        team of the GPU, then about four chunks, each a
 *                        whole number of stores per team (the fastest
 *                        measured);
 *   PCCP_HOST_IN_PLACE : no copies: one launch whose teams read their stores
 *                        from host memory and write the fixed points, status
 *                        and iterations back there, over the CPU-GPU link.
 *                        Every array must be page-locked and mapped into the
 *                        device's address space (cudaHostAlloc,
 *                        cudaHostRegister with mapping, a pinned torch tensor:
 *                        with unified addressing all of these are), each one
 *                        allocation; the mapping is checked at both ends of
 *                        each array and INVALID returned if it is missing.
 * Chunked, while one chunk is propagated the next chunks are copied in and
 * the previous ones copied out, on streams of the model's own (copy
 * in, propagate, copy out) through up to four device slots (page-locked
 * memory lets the copies overlap; pageable memory works but serialises
 * them); status and iterations, when mapped as above, are written by the
 * kernels where they lie instead of being copied.  When every array is
 * page-locked, the call's copies and launches are captured once in a CUDA
 * graph kept with the model and replayed, as one launch, by later calls
 * with the same arrays, n_stores and chunk_stores (reuse the buffers to
 * stay on that path; other arrays or sizes capture a new graph, which
 * replaces the kept one).  Streams, events, slots and the graph are created
 * on the model's first such call, grown for larger chunks and freed with
 * the model; calls on one model are serialised (the host
 * thread waits for the one in progress).  Either way the transfers start
 * after the work already queued on `stream`, and later work on `stream`
 * follows them.  Synchronous: returns once every result is in host memory.
 * Errors: INVALID (also chunk_stores < PCCP_HOST_IN_PLACE), SMEM, CUDA. */
#define PCCP_HOST_IN_PLACE (-1)
int pccp_propagate_host(const pccp_model* model, int32_t n_stores, int32_t* lb, int32_t* ub,
                        int32_t* status, int32_t* iterations, int32_t chunk_stores,
                        void* stream);

/* ---- search ------------------------------------------------------------ */

#define PCCP_INPUT_ORDER 0 /* lowest-index unfixed branch variable */
#define PCCP_FIRST_FAIL 1  /* smallest ub - lb, ties to the lower index */
#define PCCP_LEARNED 2     /* highest score of a pccp_policy, ties to the lower index */

typedef struct pccp_policy pccp_policy; /* learned branching policy, see below */

#define PCCP_OPTIMISE 0  /* branch and bound on the objective */
#define PCCP_COUNT_ALL 1 /* enumerate every solution (objective bounded by obj_ub) */

/* Result status of a search. */
#define PCCP_RES_OPTIMAL 0    /* tree exhausted, >= 1 solution (count-all: complete) */
#define PCCP_RES_INFEASIBLE 1 /* tree exhausted, no solution */
#define PCCP_RES_LIMIT 2      /* a node or time limit stopped the search */

typedef struct {
  int32_t strategy;      /* PCCP_INPUT_ORDER or PCCP_FIRST_FAIL */
  int32_t mode;          /* PCCP_OPTIMISE or PCCP_COUNT_ALL */
  int32_t deterministic; /* 1: one team walks the tree in the sequential DFS
                            order, so node counts are reproducible; 0: every
                            team pulls subproblems from a shared queue, hands
                            open branches to waiting teams and shares the
                            incumbent (node counts then vary, except count-all
                            and proof trees) */
  int32_t obj_ub;        /* inclusive upper bound told on the objective at every
                            node; INT32_MAX for none */
  int64_t node_limit;    /* stop after this many nodes (<= 0: none); per instance */
  int64_t time_limit_ms; /* stop after this many ms of device time (<= 0: none) */
  int32_t threads;       /* threads per team (multiple of 32, <= 1024; 0 = auto) */
  int32_t blocks;        /* CTAs for the parallel search (0 = auto) */
  int32_t skip_stable;   /* as in pccp_launch_config (0: the library's choice); also
                            lets a left child run only the rows of the decided
                            variable first */
  int32_t stream_table;  /* as in pccp_launch_config; batched searches stream only
                            when some table does not fit one CTA beside its store
                            (one team per CTA then) */
  const pccp_policy* policy; /* required with PCCP_LEARNED, created on this device */
  int32_t teams_per_cta;    /* batched search: models searched side by side in one CTA,
                               each by its own team in its own slot of shared memory
                               (1..15; 0 = the library's choice) */
  int32_t props_per_thread; /* propagator rows per thread per sweep: with threads == 0
                               the team size is the largest model's rows divided by
                               this, rounded up to whole warps (0 = not used) */
  int32_t queue_granularity;/* parallel search: subproblems the queue keeps ready per
                               waiting team; teams stop donating above it (0 = 1) */
  int32_t donate_nodes;     /* parallel search: after this many nodes in one
                               subproblem a team hands its shallowest open right branch
                               to the queue at each branching while teams wait for
                               work (0 = the library's choice, 4; < 0 = never) */
  int32_t temporal_levels;  /* as in pccp_launch_config (0: the library's choice: levels
                               for tables read from global memory only, since the
                               nodes of a search are mostly one decision away from a
                               fixed point, where the levels save few sweeps) */
} pccp_solve_opts;

/* Counters and outcome of one search.  A node is every store propagated,
 * including the root and failed children.  Split rule: [l,u] at
 * m = l + (u - l) / 2, left child ub <= m explored first, right lb >= m + 1;
 * after a solution of objective z every later node is told ub(obj) <= z - 1. */
typedef struct {
  int32_t status;        /* PCCP_RES_* */
  int32_t has_solution;
  int32_t objective;     /* lb(objective) of the recorded solution */
  int32_t* witness;      /* IN: HOST int32 [n_vars] buffer or NULL; OUT: lb of the
                            recorded solution (optimise: the last improving
                            one; count-all: the first found) */
  int64_t nodes;
  int64_t fails;
  int64_t solutions;
  int64_t iterations;    /* fixed-point iterations summed over nodes */
  int64_t rows_evaluated;/* propagator rows evaluated (stable rows are skipped) */
  int32_t max_depth;
  float elapsed_ms;      /* device time of the search kernel */
  float model_ms;        /* batched searches: device time of this model's own search,
                            from its first node to its end (time to proof for a
                            complete search); pccp_solve with deterministic = 0: 0 */
} pccp_result;

/* Solves one model.  Synchronous: returns after the result is filled.
 * deterministic = 1: one team in the sequential order.  deterministic = 0:
 * every team of the GPU over a shared queue of subproblems of the model (the
 * EPS variant of Sec. 5 with work donation; see pccp_solve_batch), the
 * table staged once per CTA when it fits; with stream_table and a table too
 * large for shared memory, a breadth-first frontier of subproblems (about 4
 * per team) is searched by persistent teams instead.
 * Errors: INVALID, SMEM, TIMEOUT (a device wait gave up), CUDA. */
int pccp_solve(const pccp_model* model, const pccp_solve_opts* opts, pccp_result* result,
               void* stream);

/* Solves n_models models in one persistent launch.
 * opts->deterministic = 1: each model is searched by one team in the
 * sequential order (node_limit and time_limit_ms apply per model), so every
 * model's counts are those of pccp_solve with deterministic = 1.
 * opts->deterministic = 0: every team of the GPU works over one shared queue
 * of subproblems (decision paths) of all the models, each model with its own
 * shared incumbent; a team that has searched donate_nodes nodes of a
 * subproblem while others wait hands its shallowest open right branch to the
 * queue; node_limit applies per model and time_limit_ms to the whole launch.
 * Optima, count-all counts and the counts of proof trees are exact in both
 * forms; other node counts of the parallel form depend on timing.
 * Deterministic form: a CTA holds teams_per_cta
 * teams side by side, each in its own slot of shared memory; the models are
 * queued largest table first and every team pulls the next one when it
 * finishes.  A model's table prefix is staged in its team's slot when it
 * fits beside the store, else read in place from global memory.
 * results[i] is filled for models[i] (its witness pointer is honoured).
 * Synchronous.  Errors: INVALID, SMEM (a store does not fit a slot),
 * TIMEOUT, CUDA. */
int pccp_solve_batch(const pccp_model* const* models, int32_t n_models,
                     const pccp_solve_opts* opts, pccp_result* results, void* stream);

/* ---- reusable batch, queued without synchronisation -------------------- */

/* A batch of models prepared once for repeated searches (the batched
 * configuration of the search: many models in one persistent launch).
 * pccp_batch_create allocates and uploads the model descriptors and the
 * result, witness and decision-stack buffers (synchronous).  The launch
 * shape is fixed here: `threads` per team (0 = the library's choice; a
 * multiple of 32) and `teams_per_cta` teams side by side per CTA (0 = the
 * library's choice), as in pccp_solve_batch; later searches of the batch
 * use it whatever their options say (stream_table is not used).  The models
 * must outlive the batch.  Errors: INVALID, SMEM, CUDA. */
typedef struct pccp_batch pccp_batch;
int pccp_batch_create(const pccp_model* const* models, int32_t n_models, int32_t threads,
                      int32_t teams_per_cta, pccp_batch** out);

/* The launch shape a batch was planned with (threads per team, teams per
 * CTA, CTAs). */
int pccp_batch_get_shape(const pccp_batch* batch, int32_t* threads, int32_t* teams_per_cta,
                         int32_t* ctas);

/* Queues one search of every model of the batch on `stream`, with the same
 * semantics and results as pccp_solve_batch: opts->deterministic = 1, one
 * team per model in the sequential order (node counts reproducible);
 * 0, every team over one shared queue of subproblems of all models with
 * work donation.  Enqueues only memsets or an initialisation kernel and one
 * search kernel: no host synchronisation and no allocation, so it may be
 * captured in a CUDA graph and replayed.  Calls on one batch must not
 * overlap on the GPU. */
int pccp_batch_solve_async(pccp_batch* batch, const pccp_solve_opts* opts, void* stream);

/* Synchronises `stream` and copies the last queued search's results (and
 * the witnesses of results[i].witness != NULL) to the host; elapsed_ms is 0
 * (time the graph or the stream), model_ms is each model's own time. */
int pccp_batch_results(pccp_batch* batch, pccp_result* results, void* stream);

void pccp_batch_destroy(pccp_batch* batch);

/* ---- allocation-free batched solve ------------------------------------- */

/* No counterpart in the paper.  Same contract and results as
 * pccp_solve_batch, for callers that may not allocate device memory (hosts
 * that reserve all memory at start-up and allocate nothing after a
 * no-allocation point; plug-ins whose application owns the device allocator
 * and forbids them to grow it): this call makes no cudaMalloc / cudaFree /
 * memory-pool call of any kind.
 * Its scratch (model descriptors, results, witnesses, decision stacks, work
 * counter) is one fixed array of PCCP_NOALLOC_SCRATCH_BYTES in the library's
 * device memory; every GPU that loads the library holds it until the process
 * exits.  A request whose scratch does not fit returns PCCP_ERR_SCRATCH before
 * anything is queued: descriptors 40 B + results 64 B per model and 4 B per
 * variable of every model (plus, when tables are streamed, one decision
 * stack of 8 B per possible decision for each team).
 * The first call on a device loads the library's device code there if it
 * has not been loaded yet (CUDA loads modules lazily by default), which
 * reserves the array, and looks up the array's address with that device
 * current: make that first call before any no-allocation point.  The call
 * copies through host memory and synchronises `stream` before it returns,
 * so it must not be issued while `stream` is being captured into a graph
 * (pccp_batch_solve_async is the capturable form).  All calls on a device
 * share the array, so calls that overlap on the GPU race: serialise them
 * (for instance on one stream).  results[i].elapsed_ms is the host wall time
 * of the whole call.  Errors: INVALID, SCRATCH, SMEM, TIMEOUT, CUDA. */
#define PCCP_NOALLOC_SCRATCH_BYTES (8u << 20)
int pccp_solve_batch_noalloc(const pccp_model* const* models, int32_t n_models,
                             const pccp_solve_opts* opts, pccp_result* results, void* stream);

/* ---- learned branching (no counterpart in the paper) --------------------
 * A policy is an MLP 12 -> 128 -> 128 -> 1 (ReLU) that scores each unfixed
 * branch variable of a node from 12 features (its bounds relative to the
 * root, log width, temporal in/out degree and summed offsets, reified rows
 * touching it, its demand on the linear rows (for a task's start time: the
 * sum over resources of usage / capacity), its input position, the depth
 * and the objective's progress).  The search splits the highest-scoring variable
 * (ties to the lower index) with the usual lower-half rule, so a complete
 * search still proves the same optimum; only the order of the tree changes.
 * Weights are BF16 on the device (FP32 masters for training); every product
 * runs on the tensor cores with FP32 accumulation. */
typedef struct {
  const float* w1; /* [128][12] */
  const float* b1; /* [128] */
  const float* w2; /* [128][128] (out, in) */
  const float* b2; /* [128] */
  const float* w3; /* [128] */
  float b3;
} pccp_policy_weights;

/* Host weights are copied (synchronous).  Errors: INVALID (NULL or non-finite
 * weights), CUDA. */
int pccp_policy_create(const pccp_policy_weights* weights, pccp_policy** out);
void pccp_policy_destroy(pccp_policy* policy);
/* Current FP32 weights into caller HOST arrays of the sizes above. */
int pccp_policy_get_weights(const pccp_policy* policy, float* w1, float* b1, float* w2, float* b2,
                            float* w3, float* b3);
/* Gradient of the mean loss of the last pccp_policy_train_step (the step
 * Adam then took) with respect to the FP32 parameters, into caller HOST
 * arrays of the shapes above.  Synchronises the device.  INVALID before the
 * first step. */
int pccp_policy_get_gradients(const pccp_policy* policy, float* w1, float* b1, float* w2,
                              float* b2, float* w3, float* b3);
/* Features of every branch variable of n_stores stores (DEVICE lb/ub
 * [n_stores][n_vars], joined with the root; depth DEVICE [n_stores] or NULL
 * for 0) into DEVICE out [n_stores][n_branch][12], rounded to BF16 as the
 * network sees them.  Asynchronous. */
int pccp_policy_features(const pccp_model* model, int32_t n_stores, const int32_t* lb,
                         const int32_t* ub, const int32_t* depth, float* out, void* stream);
/* Scores of n_rows DEVICE feature rows [n_rows][12] into DEVICE scores
 * [n_rows], with the search kernels' arithmetic.  Asynchronous. */
int pccp_policy_score(const pccp_policy* policy, int32_t n_rows, const float* features,
                      float* scores, void* stream);
/* One Adam step (beta 0.9 / 0.999) on the mean listwise softmax
 * cross-entropy of n_groups groups of candidate rows: DEVICE features
 * [n_rows][12], DEVICE group_off [n_groups + 1] (rows of group g are
 * group_off[g] .. group_off[g+1]-1), DEVICE target [n_rows] (a distribution
 * per group).  *loss (HOST, may be NULL) receives the mean loss before the
 * step; synchronises the stream when loss != NULL. */
int pccp_policy_train_step(pccp_policy* policy, int32_t n_rows, const float* features,
                           const int32_t* group_off, int32_t n_groups, const float* target,
                           float lr, float* loss, void* stream);

/* Human-readable name of a return code (static storage). */
const char* pccp_error_string(int code);

#ifdef __cplusplus
}
#endif

#endif /* PCCP_H */
