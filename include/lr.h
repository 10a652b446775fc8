/*
 * lr.h -- C ABI of the GB300 list-ranking library (liblr.so).
 *
 * Problem (Section 1.1 of "Engineering Scalable Distributed List Ranking",
 * Sanders, Schimek, Uhl, Weidmann): a successor array succ[0..n-1] describes
 * a set of singly linked lists; a terminal element points to itself
 * (succ[t] == t) and an initial element (head) has no predecessor.  The rank
 * of element i is the number of links from i to the terminal of its list, or,
 * in the weighted problem, the sum of the link weights on that path.
 *
 * Method: sparse ruling set (Section 2.1, Algorithm 1): pick rulers (every
 * head is forced to be one), chase each ruler's packet along succ until the
 * next ruler while recording (ruler, offset) per element, rank the reduced
 * list of rulers recursively (a single-CTA pointer-doubling base case ends the
 * recursion), then give every element rank[ruler] - offset.
 *
 * Conventions shared by every entry point below:
 *  - Pointers named succ/weight/rank/offsets are DEVICE pointers owned by the
 *    caller unless the name ends in _host.  The library never frees them.
 *  - succ is uint32; n <= LR_MAX_N (2^32 - 2).  Terminals satisfy succ[i]==i.
 *  - weight == NULL means unweighted (every link weighs 1).  weight[i] is the
 *    weight of the link i -> succ[i]; a terminal's weight is ignored, so a
 *    terminal's rank is 0 (the paper's unweighted <=> weight 1 / terminal 0
 *    equivalence, Section 1.1).
 *  - Arithmetic is exact two's-complement, wrapping in the rank type; int32
 *    weights are sign-extended.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL is the
 *    legacy default stream).  Argument errors are returned at once.  Errors
 *    that depend on the data (out-of-range successor, cycle, two
 *    predecessors, capacity) are recorded on the device and returned by
 *    lr_get_device_status(stream) (or at once when lr_opts.sync is set).
 *    On any error the contents of rank are unspecified.
 *  - The library owns only its workspace: one grow-only device arena per
 *    stream, reused across calls, unless the caller passes lr_opts.workspace.
 *    Calls on one stream must not overlap from several host threads.
 */
#ifndef LR_H
#define LR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t (struct CUstream_st *). */
typedef struct CUstream_st *lr_stream;

#define LR_MAX_N 4294967294LL /* 2^32 - 2: ids fit uint32 with two sentinels */

typedef enum lr_status {
    LR_OK = 0,
    LR_ERR_INVALID_ARGUMENT = 1, /* NULL pointer with n > 0, bad size or dtype   */
    LR_ERR_OUT_OF_RANGE = 2,     /* some succ[i] >= n (or >= its instance size)  */
    LR_ERR_CYCLE = 3,            /* an element is not reachable from any head    */
    LR_ERR_NOT_A_LIST = 4,       /* an element has two or more predecessors      */
    LR_ERR_OUT_OF_MEMORY = 5,    /* device or pinned allocation failed           */
    LR_ERR_BUDGET = 6,           /* serving: request larger than the budget      */
    LR_ERR_TIMEOUT = 7,          /* a bounded wait ran out                       */
    LR_ERR_CUDA = 8,             /* a CUDA runtime call failed                   */
    LR_ERR_CAPACITY = 9,         /* more lists than lr_opts.max_lists promised   */
    LR_ERR_NOT_FOUND = 10,       /* serving: unknown ticket                      */
    LR_ERR_CANCELLED = 11,       /* serving: server shut down before the run     */
    LR_ERR_CAPTURE = 12,         /* call would sync or allocate during capture   */
    LR_ERR_INTERNAL = 13         /* a self-check of the library failed           */
} lr_status;

typedef enum lr_dtype { LR_NONE = 0, LR_I32 = 1, LR_I64 = 2 } lr_dtype;

/*
 * Tuning knobs of the ruling-set recursion (filled by the autotuner; zero
 * fields take the built-in defaults).  Rulers per level: ceil(n / f_inv).
 *
 * LR_TUNING (environment, read at every call; a nonzero field of an
 * explicit lr_tuning takes precedence) overrides them for measurement, as comma-separated
 * key=value pairs: f0, f, cutoff, block, ctas (the fields below); xchg=0
 * (visits by load and store instead of an atomic exchange); log=0 / log=1
 * (force the level-0 form); algo, contract, spawn; ord (batches: 0 chases
 * by per-CTA slices of ruler ids, 1 takes level 0's rulers in element
 * order, 2, the default, every level of 2^20 elements or more); pf (the
 * element order's L2 prefetch lead in K elements, 0 off, 4 by default).
 */
typedef struct lr_tuning {
    uint32_t f0_inv;     /* 1/f at level 0 (default by n: 4 below 2^16, 8 below  */
                         /* 2^22, 16 below 2^27, 48 below 2^29, 96 from 2^29;   */
                         /* a batch keeps 16 from 2^22 up)                       */
    uint32_t f_inv;      /* 1/f at levels >= 1 (default 8)                       */
    uint32_t cutoff;     /* largest level ranked by the single-CTA base case     */
                         /* (default and maximum 12288)                          */
    uint32_t chase_block;/* threads per CTA of the chase kernel (default 256)    */
    uint32_t chase_ctas; /* CTAs per SM of the chase kernel (default: occupancy; */
                         /* a batch's level 0, chased in element order, 1024    */
                         /* threads per SM)                                      */
    uint32_t algorithm;  /* LR_ALGO_SRS (0, default) or LR_ALGO_WYLLIE            */
    uint32_t contract;   /* tile-local contraction: 0 auto (default),            */
                         /* LR_CONTRACT_OFF or LR_CONTRACT_ON                     */
    uint32_t spawn;      /* 1: ruler spawning at level 0 (Section 2.2); 0 off    */
    uint32_t chase0;     /* level-0 chase form: 0 auto (default),                */
                         /* LR_CHASE0_EXCHANGE or LR_CHASE0_LOG                   */
} lr_tuning;

/*
 * Level-0 chase form of the default algorithm (Algorithm 1's ruler chasing
 * and ruler propagation at the first level).  Both give identical results.
 *  - LR_CHASE0_EXCHANGE: the prep pass packs every element into a record;
 *    the chase swaps (ruler, offset) into each record with one atomic
 *    exchange, and propagation streams the records.  On GB300 that is two
 *    random DRAM accesses per element (the gather and the later write-back).
 *  - LR_CHASE0_LOG: the chase only gathers succ[] and appends each element
 *    it reaches to a per-thread log; propagation radix-partitions the log by
 *    element id into windows of 16384 ranks and assembles each window in
 *    shared memory.  One random access per element plus streaming passes.
 *    Unweighted lists with int32 ranks and n <= 2^30 only (the exchange
 *    form is used otherwise).
 * Auto (0) takes the log form for single-instance unweighted int32 calls
 * with n >= 2^25 and no extra outputs or spawning, where it is faster on
 * GB300, and the exchange form otherwise.
 */
#define LR_CHASE0_AUTO 0u
#define LR_CHASE0_EXCHANGE 1u
#define LR_CHASE0_LOG 2u

/*
 * Ruler spawning (Section 2.2): when a chasing thread's CTA has no queued
 * ruler left, the thread claims an unvisited element of the CTA's slice of
 * ids as a new ruler and chases from it, so that every thread keeps a wave
 * until no unvisited element is left; waves that reach a spawned ruler stop
 * there.  More rulers (about t ln(n/t) for t waves) in exchange for shorter
 * segments.  Level 0 of the default algorithm, exchange chase only; not
 * combined with extra outputs or the log path (ignored there).  Results are
 * identical with and without.
 */

/*
 * Tile-local contraction (Section 2.3, restated for one GPU): before the
 * ruling set, every maximal sublist inside a tile of 4096 consecutive ids is
 * contracted in shared memory to one node, the ruling set ranks the list of
 * those nodes, and a final pass restores every element.  It pays when links
 * mostly stay inside tiles (locality and identity orders).  Auto (the
 * default) lets the prep pass count the links that stay inside their tile
 * and contracts when at least half do, decided at the wait that counts the
 * lists; it applies to single-instance calls that count their lists anyway
 * (max_lists == 0, no workspace, not during capture, no extra outputs,
 * n >= 16384).  LR_CONTRACT_ON contracts without counting;
 * LR_CONTRACT_OFF never contracts.  Results are identical either way.
 */
#define LR_CONTRACT_AUTO 0u
#define LR_CONTRACT_OFF 1u
#define LR_CONTRACT_ON 2u

/*
 * Algorithms behind lr_tuning.algorithm.  LR_ALGO_WYLLIE is pointer doubling
 * over the whole list, the baseline the paper compares against (Sections 1
 * and 3): ceil(log2 n) rounds, each replacing every unfinished element's
 * (successor, partial rank) by its successor's, double buffered.  Same
 * inputs, outputs, errors and batch form as the default; about log2(n)
 * random accesses per element instead of one or two, so it serves as the
 * comparison workload.  Its workspace is lr_workspace_size with the same
 * tuning; max_lists does not apply and it never synchronises.
 */
#define LR_ALGO_SRS 0u
#define LR_ALGO_WYLLIE 1u

typedef struct lr_opts {
    lr_dtype wtype;           /* weight type: LR_NONE (unweighted), LR_I32, LR_I64   */
    lr_dtype rtype;           /* rank type: LR_I32 or LR_I64                          */
    const lr_tuning *tuning;  /* NULL: defaults / autotuned table                     */
    void *workspace;          /* optional caller-owned device memory                  */
    size_t ws_bytes;          /* its size; must be >= lr_workspace_size(...)          */
    int32_t validate;         /* 1: also detect two predecessors (LR_ERR_NOT_A_LIST) */
    int32_t sync;             /* 1: wait for the device and return its status         */
    uint64_t seed;            /* ruler sampling seed (results do not depend on it)    */
    int64_t max_lists;        /* > 0: promise at most this many lists (heads).  The   */
                              /* call then never synchronises and can be captured in  */
                              /* a CUDA graph.  0: count the heads first (one sync).  */
    int64_t n_total;          /* batch only: sum of instance sizes if known (>0), so  */
                              /* offsets[k] need not be read back from the device.    */
} lr_opts;

/* Fill *o with defaults: unweighted, int32 ranks, seed 0x5eed, no sync. */
void lr_opts_default(lr_opts *o);

/*
 * Rank one successor array.  weight == NULL: unweighted, rank is int32
 * (n must be < 2^31).  weight != NULL: weight and rank are int64.
 */
lr_status lr_rank(const uint32_t *succ, const void *weight, int64_t n, void *rank,
                  lr_stream stream);

/* Same with explicit dtypes, tuning, workspace and validation. */
lr_status lr_rank_ex(const uint32_t *succ, const void *weight, int64_t n, void *rank,
                     const lr_opts *opts, lr_stream stream);

/*
 * Rank k independent instances stored back to back.  offsets (device,
 * int64[k+1], offsets[0] == 0, non-decreasing) delimits instance j as
 * elements offsets[j] .. offsets[j+1]-1; succ holds LOCAL ids in
 * [0, offsets[j+1]-offsets[j]).  weight/rank as in lr_rank (int64 when
 * weighted).  All instances run in one launch sequence over the forest they
 * form (Section 1.1 allows a set of lists).  Sum of sizes <= LR_MAX_N.
 */
lr_status lr_rank_batch(const int64_t *offsets, const uint32_t *succ, const void *weight,
                        void *rank, int32_t k, lr_stream stream);

lr_status lr_rank_batch_ex(const int64_t *offsets, const uint32_t *succ, const void *weight,
                           void *rank, int32_t k, const lr_opts *opts, lr_stream stream);

/*
 * Rank k independent instances that live in separate device buffers, as one
 * forest in one launch sequence (Section 1.1's set of lists; the serving
 * loop ranks waiting requests this way, where they already are).
 *   offsets      device int64[k+1], offsets[0] == 0, non-decreasing:
 *                instance j has offsets[j+1] - offsets[j] elements.
 *   succ_ptrs    device array of k device pointers, uint32 LOCAL successors
 *                of instance j ([0, its size); a tail points to itself).
 *   weight_ptrs  NULL (unweighted) or a device array of k device pointers to
 *                weights of opts->wtype.
 *   rank_ptrs    device array of k device pointers to ranks of opts->rtype,
 *                written by the call.
 * Every buffer is owned by the caller and must hold its instance's size in
 * elements (shorter buffers are undefined behaviour); an empty instance's
 * pointers are never read.  The kernels address the buffers through the
 * offset table, so the call first reads the table back (one wait on the
 * stream; not capturable: LR_ERR_CAPTURE) and returns LR_ERR_INVALID_ARGUMENT
 * unless it starts at 0 and never decreases (and, if opts->n_total > 0,
 * ends at n_total); the sum of sizes is at most LR_MAX_N.  opts as in
 * lr_rank_batch_ex (NULL: int64 weights and ranks when weight_ptrs is set,
 * else int32 ranks): max_lists (> 0) saves counting the lists, validate
 * checks in-degrees, sync waits and returns the device status.  A caller
 * workspace is not supported here (LR_ERR_INVALID_ARGUMENT), nor are extra
 * outputs.  A successor outside its instance is LR_ERR_OUT_OF_RANGE, through
 * the device status like every data error.
 */
lr_status lr_rank_batch_ptrs(const int64_t *offsets, const uint32_t *const *succ_ptrs,
                             const void *const *weight_ptrs, void *const *rank_ptrs, int32_t k,
                             const lr_opts *opts, lr_stream stream);

/*
 * Extra outputs of the default algorithm (Section 1.1 defines the result
 * as each element's rank AND the terminal of its list; its in-place form
 * counts the terminal's own weight).  All pointers are device memory owned
 * by the caller, n entries each, none aliasing succ, weight or rank:
 *   term            uint32: the terminal (last element) of i's list; in the
 *                   batched form a LOCAL id within i's instance.  NULL: not
 *                   produced.
 *   prefix          opts->rtype: head-relative rank, the sum of the link
 *                   weights from i's head to i (0 at a head; the list's
 *                   total at its terminal).  NULL: not produced.
 *   inclusive_tail  1: rank[i] also counts the terminal's own weight
 *                   weight[t], so rank[t] = weight[t].  Unweighted, the
 *                   terminal weighs 0 (Section 1.1: weight 1 on every
 *                   element but the terminal), so the flag changes nothing.
 *                   prefix is the same either way.
 * Not available with LR_ALGO_WYLLIE (LR_ERR_INVALID_ARGUMENT).  Errors as
 * for lr_rank_ex; on error the extra outputs are unspecified too.
 */
typedef struct lr_outputs {
    uint32_t *term;
    void *prefix;
    int32_t inclusive_tail;
} lr_outputs;

lr_status lr_rank_outputs(const uint32_t *succ, const void *weight, int64_t n, void *rank,
                          const lr_outputs *outs, const lr_opts *opts, lr_stream stream);

lr_status lr_rank_batch_outputs(const int64_t *offsets, const uint32_t *succ, const void *weight,
                                void *rank, int32_t k, const lr_outputs *outs, const lr_opts *opts,
                                lr_stream stream);

/*
 * End-to-end form with HOST buffers (pageable or pinned): copies succ and
 * weight to the device, ranks, copies rank back and waits.  Returns the
 * final status (argument or device error).
 */
lr_status lr_rank_host(const uint32_t *succ_host, const void *weight_host, int64_t n,
                       void *rank_host, const lr_opts *opts, lr_stream stream);

/*
 * Same, without waiting: copy-in, ranking and copy-out are enqueued on
 * `stream` (through device staging buffers owned by the stream's context) and
 * the call returns.  rank_host is valid once the stream has been synchronised;
 * lr_get_device_status(stream) then returns the status.  Host buffers should
 * be pinned for the copies to be asynchronous; the caller keeps them alive and
 * untouched until then.  Calls on two or more streams overlap one call's
 * copies with another call's kernels, but the streams' kernels then share
 * the GPU and finish together; lr_pipeline below keeps the ranking of a
 * sequence of host lists back to back.  With opts->max_lists == 0 the call
 * still waits once to count the lists; pass a bound to keep it fully
 * asynchronous.
 */
lr_status lr_rank_host_async(const uint32_t *succ_host, const void *weight_host, int64_t n,
                             void *rank_host, const lr_opts *opts, lr_stream stream);

/*
 * Bytes of workspace a call with these sizes needs when the caller passes
 * lr_opts.workspace.  k = 0 for lr_rank_ex.  Uses opts->max_lists as the
 * bound on the number of lists (0: assumes every element may be a head).
 * Host-only; needs no GPU.
 */
size_t lr_workspace_size(int64_t n_total, int32_t k, const lr_opts *opts);

/* Same for a call with extra outputs: only which pointers of *outs are
 * non-NULL (and inclusive_tail) matters; outs == NULL is lr_workspace_size. */
size_t lr_workspace_size_outputs(int64_t n_total, int32_t k, const lr_outputs *outs,
                                 const lr_opts *opts);

/*
 * Shape of the recursion of the last ruling-set call on `stream` (after it
 * completes; waits for the stream): the sizes of the levels that ran, level
 * 0 first (n), then the rulers of each level, down to the base case.
 * Writes up to max_levels entries and returns how many levels ran (0 when
 * the last call did not run the ruling set itself, e.g. pointer doubling or
 * a contracted call; -1 on a CUDA error).  The descriptors live in the
 * call's workspace: valid until the next call on the stream or until a
 * caller-owned workspace is reused.
 */
int32_t lr_level_sizes(lr_stream stream, int64_t *sizes, int32_t max_levels);

/*
 * Wait for `stream` and return (and clear) the status the device recorded
 * for the last call issued on it.
 */
lr_status lr_get_device_status(lr_stream stream);

/*
 * Rank without allocating.  The paper has no counterpart: this is a service
 * for callers that cannot call cudaMalloc when they need a ranking (a process
 * whose allocator already holds all free device memory, a latency-critical
 * loop that must not risk an allocation's implicit synchronisation, a plug-in
 * in a host that forbids allocations after start-up).
 *  - succ: device uint32[n]; rank: device int32[n] (unweighted ranks).
 *    Caller-owned; n <= LR_NOALLOC_MAX_N, larger n returns
 *    LR_ERR_INVALID_ARGUMENT.
 *  - Workspace is a fixed 64 MiB scratch array compiled into liblr.so; every
 *    GPU that loads the library holds it until the process exits.  The
 *    library's set-up on a device (done by the first lr_* call made with
 *    that device current) looks up the array's device address, which is
 *    also what places the array there; make some lr_* call on each device
 *    early, before the process has taken all free device memory, and before
 *    any stream capture begins.  If the array could not be placed then, the
 *    first lr_rank_noalloc call tries again and returns
 *    LR_ERR_OUT_OF_MEMORY when the device has no room.  No cudaMalloc,
 *    cudaFree or other allocating call is made.  The ruling-set settings
 *    are fixed (LR_TUNING and autotuned entries are not consulted).  Inputs
 *    with so many lists that the recursion does not fit the scratch return
 *    LR_ERR_CAPACITY.
 *  - All calls share the scratch, which keeps the last call's contents
 *    (everything that must start at zero is cleared by each call).  Calls
 *    that overlap on the GPU race, and the host side is not thread-safe:
 *    serialise calls.
 *  - The call waits for the device and returns the final status (argument
 *    or data error), like lr_opts.sync = 1.
 */
#define LR_NOALLOC_MAX_N (1LL << 22)
lr_status lr_rank_noalloc(const uint32_t *succ, int64_t n, int32_t *rank, lr_stream stream);

/* Human-readable name of a status code (static string). */
const char *lr_status_string(lr_status s);

/* Library version string (static). */
const char *lr_version(void);

/*
 * Profiling.  While enabled, every call records CUDA events around its
 * phases on its own stream; lr_profile_read waits for them and returns the
 * accumulated device milliseconds per phase and the number of kernels the
 * library launched since the last reset.
 */
typedef struct lr_profile {
    double ms_prep;      /* level-0 pass: validate, pack, has-predecessor bitmap */
    double ms_select;    /* head detection and ruler numbering, all levels      */
    double ms_chase0;    /* level-0 ruler chasing (the dominant kernel)          */
    double ms_chase_rest;/* ruler chasing at levels >= 1                         */
    double ms_base;      /* base case                                            */
    double ms_finalize;  /* ruler propagation, all levels                        */
    int64_t calls;       /* ranked calls covered                                 */
    int64_t chase0_launches;
    int64_t kernel_launches;
    int64_t elements;    /* elements ranked (sum of n)                           */
    int64_t chase0_log_launches; /* of chase0_launches: the log form            */
} lr_profile;

lr_status lr_profile_enable(int32_t on);
lr_status lr_profile_read(lr_profile *out, int32_t reset);

/*
 * Memory-system probe (measurement only; the paper has no counterpart).
 * The chase of Algorithm 1 is a dependent random walk, so its ceiling on a
 * GPU is the rate at which random accesses are served, not the streaming
 * bandwidth, and that rate depends on the footprint the accesses cover.  On
 * the caller's device buffer (>= 16 MiB, 256-byte aligned; its size is the
 * footprint; its contents are destroyed) this measures a streaming copy, a
 * dependent random 4-byte gather (the chase's own access), independent
 * random 4-byte gathers with 8 in flight per thread, the same confined per
 * warp to one random 2 MiB region at a time, and a dependent random 8-byte
 * atomic exchange.  Each walk follows one seeded random cycle through the
 * buffer.  Waits for the device.
 */
typedef struct lr_probe_result {
    double copy_gbs;            /* streaming read + write, GB/s                  */
    double gather_gsteps;       /* dependent random 4-byte loads, G steps/s      */
    double gather_xchg_gsteps;  /* dependent random 8-byte exchanges, G steps/s  */
    size_t footprint_bytes;     /* bytes the random accesses covered             */
    double indep_gather_gsteps; /* independent random 4-byte loads, G/s          */
    double region_gather_gsteps;/* the same inside one 2 MiB region per warp and */
                                /* round, G/s (0 for footprints under 4 MiB)     */
} lr_probe_result;

lr_status lr_probe_memory(void *buf, size_t bytes, lr_probe_result *out, lr_stream stream);

/* Kernels launched by the library since load (all streams). Host-only. */
int64_t lr_kernel_launch_count(void);

/* ---------------------------------------------------------------- serving
 * Continuous batching: requests of mixed sizes are admitted while their
 * device footprint fits the memory budget, grouped as they arrive into
 * batched launches on one of n_streams streams, and completed individually.
 * A request of at least alone_min_n elements is a batch of its own, and a
 * batch of one request is ranked through the single-list path (as lr_rank_ex
 * ranks it, with its tile-local contraction and level-0 form); smaller
 * requests are ranked together as one forest.
 */
typedef struct lr_server lr_server;

typedef struct lr_server_config {
    size_t budget_bytes;     /* device memory for resident requests (default 40e9)  */
    int32_t n_streams;       /* concurrent batches in flight (default 4)             */
    int32_t max_batch;       /* most requests per launch (default 256)               */
    int64_t max_batch_elems; /* most elements per launch (default 2^28)              */
    int32_t device;          /* CUDA device ordinal (default 0)                      */
    int32_t plain;           /* 1: rank every request alone through the single-list  */
                             /* path, as lr_rank_ex does (baseline mode)             */
    int64_t alone_min_n;     /* a request of at least this many elements is ranked   */
                             /* alone, never batched with others; 0 = default 2^23,  */
                             /* < 0 = batch requests of any size                     */
} lr_server_config;

void lr_server_config_default(lr_server_config *c);

typedef struct lr_request {
    const uint32_t *succ;    /* successor array (host or device, see on_device)     */
    const void *weight;      /* weights or NULL                                     */
    void *rank;              /* output (host or device)                             */
    int64_t n;
    lr_dtype wtype, rtype;
    int32_t on_device;       /* 1: pointers are device memory the caller keeps      */
                             /* alive until lr_server_wait returns; 0: host memory  */
                             /* copied into budgeted device buffers by the server   */
} lr_request;

typedef struct lr_result {
    lr_status status;
    double t_submit_ms, t_admit_ms, t_launch_ms, t_done_ms; /* since server start */
} lr_result;

typedef struct lr_server_stats {
    int64_t completed;
    int64_t elements;
    int64_t batches;
    double p50_ms, p99_ms, mean_ms;   /* submit -> done                            */
    double elements_per_s;            /* completed elements / busy wall time        */
    size_t peak_resident_bytes;
    int64_t ranked_alone;             /* batches of one request (ranked through the */
                                      /* single-list path; all of them in plain     */
                                      /* mode)                                      */
} lr_server_stats;

lr_status lr_server_create(const lr_server_config *cfg, lr_server **out);
lr_status lr_server_submit(lr_server *s, const lr_request *req, uint64_t *ticket);
/* timeout_ms < 0: wait without limit. */
lr_status lr_server_wait(lr_server *s, uint64_t ticket, int64_t timeout_ms, lr_result *res);
lr_status lr_server_stats_get(lr_server *s, lr_server_stats *out);
void lr_server_destroy(lr_server *s);

/*
 * Autotuner.  The best ruler fractions, base-case cutoff and chase block
 * depend on n, on the weights and on whether the input is a batch (small
 * lists are bound by the latency along one segment, large ones by the
 * random-access rate).  lr_autotune measures candidates on the current
 * device by coordinate descent from the built-in defaults (level-0 fraction
 * 1/f0, deeper fraction 1/f, cutoff, chase block, then f0 again), each the
 * fastest of a few timed calls on `stream`, and checks that the winner's
 * ranks equal the defaults' bit for bit (else LR_ERR_INTERNAL).
 *
 * Inputs: the caller's device arrays (succ, weight, offsets as for
 * lr_rank_ex / lr_rank_batch_ex; offsets required when k > 0), or, with
 * succ == NULL, synthetic ones of the same shape generated on the device: k
 * equal random-order instances (one random list when k == 0), weights of
 * opts->wtype in [-1000, 1000].  opts: dtypes, validate, seed and max_lists
 * as for the ranking call; workspace must be NULL; the call allocates and
 * frees its own scratch.  Synchronises `stream`.
 *
 * The winner is stored in a process-wide table keyed by (floor(log2 n),
 * weighted, batched) and written to *out (may be NULL).  Every later call
 * whose opts->tuning is NULL uses its key's entry (an explicit lr_tuning,
 * then LR_TUNING in the environment, take precedence).  The table is saved
 * and loaded as JSON; LR_TUNING_FILE names a file loaded on first use.
 */
typedef struct lr_tune_entry {
    int32_t log2n;       /* floor(log2 n) of the tuned size                      */
    int32_t weighted;    /* 1: weighted                                          */
    int32_t batch;       /* 1: batched form (k > 0)                              */
    lr_tuning tuning;    /* the winner                                           */
    float ms;            /* its time per call on the tuning input                */
} lr_tune_entry;

lr_status lr_autotune(const uint32_t *succ, const void *weight, const int64_t *offsets,
                      int64_t n_total, int32_t k, const lr_opts *opts, lr_stream stream,
                      lr_tuning *out);
lr_status lr_autotune_save(const char *path);
/* Merge the entries of a file saved by lr_autotune_save into the table. */
lr_status lr_autotune_load(const char *path);
/* Copy up to cap entries into out (may be NULL); returns how many exist. */
int32_t lr_autotune_entries(lr_tune_entry *out, int32_t cap);
void lr_autotune_clear(void);

/*
 * Host-buffer pipeline: ranks a sequence of HOST-resident lists (Section 1.1
 * problem, one list or forest per submission) with each list's copies
 * overlapping the ranking of its neighbours.  A pipeline owns CUDA streams
 * on the current device (copy-in, copy-out, and one ranking stream, or two
 * when depth >= 3), `depth` device slots of max_n elements (successors,
 * weights, ranks) and one engine workspace per ranking stream, all allocated
 * by lr_pipeline_create.  Submission j uses slot j % depth; its copy-in
 * waits until the ranking of submission j - depth has read the slot, and its
 * ranking waits for its copy-in and for the copy-out of submission j - depth.
 * With one ranking stream rankings run one after another in submission
 * order; with two, submission k since the last wait ranks on stream k % 2,
 * so two rankings overlap on the device (one list's chase with the other's
 * streaming passes), which raises throughput on large lists.
 *
 * opts (copied at create; NULL = defaults) fixes wtype, rtype, tuning,
 * validate, seed and max_lists for every submission; opts->workspace must be
 * NULL.  With max_lists > 0 (a bound on the lists of every submission; a
 * submission with more fails with LR_ERR_CAPACITY) the engine workspace is
 * allocated at create and submissions neither allocate nor wait.  With
 * max_lists == 0 each submission first counts its lists, so the submitting
 * thread waits for the ranking stream to reach it (the copies of the next
 * submission still overlap this ranking), and the engine grows its own
 * buffers to the count.  depth: 2..4 (0 selects 2).  Device memory:
 * depth * max_n * (4 + weight bytes + rank bytes), plus
 * lr_workspace_size(max_n, 0, opts) per ranking stream when max_lists > 0
 * (the engine's own buffers per ranking stream otherwise).
 *
 * Host buffers should be pinned (cudaHostAlloc / cudaHostRegister); pageable
 * buffers work but their copies block the submitting thread.  The caller
 * keeps every submitted buffer alive and unmodified, and reads no rank
 * buffer, until lr_pipeline_wait returns.  One pipeline is used by one host
 * thread at a time; distinct pipelines are independent.
 */
typedef struct lr_pipeline lr_pipeline;

lr_status lr_pipeline_create(int64_t max_n, const lr_opts *opts, int32_t depth, lr_pipeline **out);
/* Enqueue one list; 0 <= n <= max_n; weight_host non-NULL exactly when
 * opts->wtype != LR_NONE.  Returns argument errors at once; errors the
 * device finds are reported by lr_pipeline_wait. */
lr_status lr_pipeline_submit(lr_pipeline *p, const uint32_t *succ_host, const void *weight_host,
                             int64_t n, void *rank_host);
/* Wait for every submission since the previous wait.  Returns LR_OK, or the
 * status of the first submission that failed, with its 0-based index since
 * the previous wait in *failed_index (-1 when none; may be NULL).  Rank
 * buffers of the other submissions are valid. */
lr_status lr_pipeline_wait(lr_pipeline *p, int64_t *failed_index);
/* Wait, then release the streams, events and device memory. */
void lr_pipeline_destroy(lr_pipeline *p);

#ifdef __cplusplus
}
#endif
#endif /* LR_H */
