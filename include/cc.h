/*
 * cc.h - C ABI of the GB300 (sm_103a) chordless-cycle enumeration library.
 *
 * Method: arXiv 1410.4876 (Jradi, Dias, Castonguay, Longo, do Nascimento), "A GPU-based
 * parallel algorithm for enumerating all chordless cycles in graphs".
 *   - problem statement: Section 1 (a chordless cycle is an induced subgraph that is a
 *     cycle of a finite undirected simple graph) and the input/output of Algorithm 1;
 *   - degree labelling: Section 2;
 *   - initial triplets and triangles: Section 4.3 and Algorithm 2;
 *   - level-by-level path expansion with the label, chord and close tests: Section 4.4
 *     and Algorithm 3, driven by the relaunch loop of Algorithm 4;
 *   - count-only operation: the footnote of Table 1 (Grid 8x10).
 *
 * Conventions used throughout this header
 *   - Length counts vertices.  A cycle of k vertices has k edges; a path <v1..vt> has t.
 *   - max_len bounds the cycle length; 0 means no bound.  L' = min(max_len, n) when
 *     max_len > 0, else n.
 *   - hist[k] (k = 0..L') is the number of chordless cycles with k vertices; entries 0..2
 *     are always zero.  total = sum of hist; it INCLUDES triangles (the paper's Table 1
 *     prints triangles in column C3 and longer cycles in column #clc).
 *   - Cycle hash (order independent, exact, defined by this library because the paper
 *     prints no cycle lists): with mix() the SplitMix64 output finaliser (Steele, Lea and
 *     Flood 2014, constants of Vigna's splitmix64.c) and GAMMA = 0x9E3779B97F4A7C15,
 *         r(v)  = mix((v + 1) * GAMMA)              v = caller's vertex id
 *         h(C)  = mix(sum_{v in C} r(v) + |C| * GAMMA)
 *         hash  = sum over all chordless cycles C of h(C)
 *     all modulo 2^64.  A chordless cycle is determined by its vertex set (it is induced),
 *     so h depends on the set only.  A sum (not XOR) makes a duplicated report visible.
 *   - tcount[t] (optional output) is the number of chordless paths of t vertices that the
 *     expansion stored (the sets T of Algorithm 1 by length, t = 3..L'-1).  These depend on
 *     the degree labelling's tie rule; this library breaks ties by smallest vertex id.
 *   - Canonical ordered cycle (cycle lists): start at the smallest vertex id and continue
 *     towards the smaller of its two cycle neighbours.
 *
 * Ownership: every pointer argument is HOST memory owned by the caller unless stated
 * otherwise; the library copies what it needs.  Device memory is owned by the context
 * (or supplied by the caller through cc_options.workspace).  Nothing here aborts or traps:
 * every failure is a status code.  All device waits are bounded and report
 * CC_ERR_TIMEOUT.  There is no CPU fallback: without a usable sm_103a device the calls
 * that need one fail with CC_ERR_CUDA.
 *
 * Thread safety: a context and the graphs loaded into it must be used from one host
 * thread at a time.
 */
#ifndef CC_H_
#define CC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t cc_status;

#define CC_OK 0
#define CC_PENDING 1              /* cc_batch_poll: not finished within the timeout       */
#define CC_ERR_ARG (-1)           /* bad argument (NULL where required, size mismatch)    */
#define CC_ERR_INVALID_GRAPH (-2) /* CSR is not a simple undirected graph                 */
#define CC_ERR_OOM (-3)           /* device or host allocation failed                     */
#define CC_ERR_CUDA (-4)          /* a CUDA call failed (no device, launch error, ...)    */
#define CC_ERR_TIMEOUT (-5)       /* a bounded device wait gave up                        */
#define CC_ERR_TRUNCATED (-6)     /* cycle list buffer too small; required sizes returned */
#define CC_ERR_UNSUPPORTED (-7)   /* graph beyond the library's limits (see cc_limits)    */
#define CC_ERR_CAPACITY (-8)      /* frontier memory too small to make progress           */

#define CC_MODE_AUTO 0   /* bitset adjacency when n <= 256, CSR adjacency otherwise */
#define CC_MODE_BITSET 1 /* force the shared-memory bitset path (n <= 256)          */
#define CC_MODE_CSR 2    /* force the CSR path (any n up to the CSR limit)          */

typedef struct cc_context cc_context;
typedef struct cc_graph cc_graph;

/* Options of a context.  Zero-initialise and set what you need. */
typedef struct cc_options {
  uint64_t frontier_bytes;     /* device bytes for chordless paths in flight; 0 = default  */
                               /* (min(64 GiB, 40% of free memory)).  When a level would   */
                               /* not fit, the expansion switches to depth-first chunks.  */
  void* stream;                /* cudaStream_t to run on; NULL = a stream the context owns */
  void* workspace;             /* optional caller-owned device buffer (>= 256-byte aligned)*/
  uint64_t workspace_bytes;    /* used as the frontier arena instead of an allocation      */
  uint32_t threads_per_block;  /* expansion kernel block size (64..256, multiple of 32; 0 = 256) */
  uint32_t blocks_per_sm;      /* persistent blocks per SM; 0 = occupancy limit, at most 4 */
  uint32_t mode;               /* CC_MODE_*                                               */
  uint32_t spin_limit;         /* grid-barrier wait limit in polls; 0 = default (~8 s)    */
  uint32_t flags;              /* CC_FLAG_*                                               */
  uint32_t paths_per_thread;   /* bitset and batch expansion: paths a thread takes per    */
                               /* round, 1..4 (one-word rows; fewer for wider rows and    */
                               /* the batch, larger values take the most); 0 = the        */
                               /* build's default for the path                            */
  uint32_t small_phase_paths;  /* bitset graphs: the cluster phase expands levels (or     */
                               /* chunks) of at most this many paths.  0 = 2 * cluster    */
                               /* size * 1024 for graphs of maximum degree <= 5, and no   */
                               /* cluster phase for denser ones; a nonzero value runs     */
                               /* the phase for every bitset graph                        */
  uint32_t reserved;           /* must be 0                                               */
  uint64_t host_frontier_bytes;/* pinned host memory for frontier frames (0 = none).  When */
                               /* cc_enumerate would expand a level in small depth-first  */
                               /* chunks while other frames wait below it, those frames  */
                               /* move to host memory and come back when the device stack */
                               /* empties (Section 6's host-GPU transport); fixed at       */
                               /* creation.  Not used by cc_enumerate_stream or batches.  */
} cc_options;

/* cc_options.flags */
#define CC_FLAG_NO_CLUSTER_PHASE 1u /* bitset graphs: skip the thread-block-cluster phase that  */
                                    /* expands small levels before the persistent grid starts  */
#define CC_FLAG_NO_GRAPH 2u         /* cc_enumerate: launch every kernel directly instead of    */
                                    /* replaying the CUDA graph captured by an earlier call    */
#define CC_FLAG_NO_FUSE 4u          /* bitset graphs: expand one level per grid step (by       */
                                    /* default a level whose children are known exactly and    */
                                    /* fit is expanded together with its children, and only    */
                                    /* the grandchildren are stored)                           */

/* Build limits. */
typedef struct cc_limits {
  uint32_t max_n_bitset;  /* largest n of the bitset path                         */
  uint32_t max_n_csr;     /* largest n of the CSR path                            */
  uint32_t max_n_batch;   /* largest n of a graph in cc_batch_submit              */
  uint32_t max_batch;     /* largest number of graphs in one cc_batch_submit      */
} cc_limits;

/* Timings and counters of the last cc_enumerate on a context. */
typedef struct cc_run_info {
  double ms_proc;          /* device time: labelling, seeding, expansion, reductions  */
  double ms_total;         /* ms_proc plus the result copies back to the host         */
  double ms_engine;        /* device time of the expansion kernel alone                */
  uint64_t steps;          /* expansion steps (levels, or chunks when spilling)       */
  uint64_t paths;          /* chordless paths stored (sum of tcount)                  */
  uint64_t cycles;         /* chordless cycles found (sum of hist)                    */
  uint32_t mode;           /* CC_MODE_BITSET or CC_MODE_CSR                           */
  uint32_t grid_blocks;    /* persistent grid size                                    */
  uint32_t spilled;        /* 1 if some level was expanded in depth-first chunks      */
  uint32_t launches;       /* kernels this library launched for the call              */
  uint64_t peak_bytes;     /* largest arena extent in use                             */
  int32_t dev_error;       /* device-side error word (0 = none; diagnostics)          */
  int32_t dev_error_info;  /* where it was raised                                     */
  uint32_t replayed;       /* 1 if the call replayed a captured CUDA graph            */
  uint32_t host_offloads;  /* times frames were moved to host memory (host frontier)  */
} cc_run_info;

/* Optional cycle list.  Set the capacities and pointers; the call fills count,
 * total_vertices and, if both fit, offsets[0..count] and vertices[0..total_vertices).
 * If they do not fit, cc_enumerate returns CC_ERR_TRUNCATED with the required count and
 * total_vertices filled in (hist and hash are still valid); call again with larger buffers.
 * Cycle order in the list is unspecified; each cycle is in canonical order (above). */
typedef struct cc_cycles {
  uint64_t capacity_cycles;    /* in: offsets has capacity_cycles + 1 entries   */
  uint64_t capacity_vertices;  /* in: vertices has capacity_vertices entries    */
  uint64_t* offsets;           /* out: cycle i is vertices[offsets[i] .. offsets[i+1]) */
  uint32_t* vertices;          /* out: original vertex ids                      */
  uint64_t count;              /* out: number of cycles                         */
  uint64_t total_vertices;     /* out: sum of cycle lengths                     */
} cc_cycles;

/* Create a context on the current CUDA device.  opts may be NULL (all defaults).
 * Errors: CC_ERR_ARG (out NULL, bad option values), CC_ERR_CUDA (no usable device). */
cc_status cc_context_create(const cc_options* opts, cc_context** out);

/* Wait for outstanding work and free everything the context owns. NULL is ignored. */
void cc_context_destroy(cc_context* ctx);

/* Human-readable name of a status code (static string). */
const char* cc_status_str(cc_status s);

/* Fill the build limits. */
void cc_get_limits(cc_limits* out);

/*
 * Load a graph (Section 4.2: the compact representation V_e/E_e).
 *   n        number of vertices (ids 0..n-1)
 *   row_ptr  host array of n+1 offsets, row_ptr[0] = 0, non-decreasing
 *   col_idx  host array of row_ptr[n] neighbour ids; every undirected edge appears in both
 *            rows.  Rows need not be sorted (they are sorted on load).
 * The graph must be simple: no self-loops, no duplicate neighbours, symmetric adjacency,
 * ids < n; otherwise CC_ERR_INVALID_GRAPH.  Isolated vertices and several components are
 * fine.  n larger than cc_limits.max_n_csr gives CC_ERR_UNSUPPORTED.  The CSR is copied to
 * the device; the caller may free its arrays after the call returns.
 */
cc_status cc_graph_load(cc_context* ctx, uint32_t n, const uint32_t* row_ptr,
                        const uint32_t* col_idx, cc_graph** out);

/* Free a loaded graph. NULL is ignored. */
void cc_graph_free(cc_graph* g);

/* Vertex and edge counts and maximum degree of a loaded graph (any pointer may be NULL). */
cc_status cc_graph_info(const cc_graph* g, uint32_t* n, uint64_t* m, uint32_t* max_degree);

/*
 * Change the launch options of a context: threads_per_block, blocks_per_sm, mode,
 * spin_limit, flags, paths_per_thread and small_phase_paths are taken from *opts; the
 * frontier size, stream and workspace fixed at creation are kept.  Errors: CC_ERR_ARG
 * (NULL, or a value outside the ranges documented in cc_options).
 */
cc_status cc_context_set_options(cc_context* ctx, const cc_options* opts);

/*
 * Enumerate all chordless cycles of a loaded graph with at most max_len vertices.
 *   out_hist    host array of L'+1 entries (L' as above); required
 *   out_hash    host pointer to one uint64; required
 *   out_tcount  host array of L'+1 entries, or NULL
 *   out_cycles  cycle list, or NULL for count-only operation
 *   out_info    timings and counters, or NULL
 * Blocks the calling thread until the result is on the host.  Errors: CC_ERR_ARG,
 * CC_ERR_CUDA, CC_ERR_TIMEOUT, CC_ERR_CAPACITY (frontier memory below the minimum of
 * about L' * max_degree paths), CC_ERR_TRUNCATED (see cc_cycles).
 */
cc_status cc_enumerate(cc_graph* g, uint32_t max_len, uint64_t* out_hist, uint64_t* out_hash,
                       uint64_t* out_tcount, cc_cycles* out_cycles, cc_run_info* out_info);

/*
 * One part of an enumeration split over its initial triplets, for several GPUs (or several
 * calls).  Section 4.3 gives every initial triplet its own work item (Algorithm 2), and each
 * triplet roots an independent subtree of chordless paths in Algorithm 3, so the subtrees
 * can be enumerated apart and their results added.  The initial triplet, or triangle,
 * <x, u, y> (original ids, l(u) < l(x) < l(y)) belongs to part
 *     mix((u * n + x) * n + y) mod nparts          (mix: the SplitMix64 finaliser above)
 * which does not depend on the labelling's tie rule or on thread order.  Summing out_hist,
 * out_hash (mod 2^64) and out_tcount over parts 0 .. nparts-1 gives exactly what
 * cc_enumerate returns; cycle lists of the parts are disjoint and together hold every
 * cycle.  nparts = 1 is cc_enumerate.  Arguments and errors as for cc_enumerate, plus
 * CC_ERR_ARG when nparts == 0 or part >= nparts.
 */
cc_status cc_enumerate_part(cc_graph* g, uint32_t max_len, uint32_t part, uint32_t nparts, uint64_t* out_hist,
                            uint64_t* out_hash, uint64_t* out_tcount, cc_cycles* out_cycles,
                            cc_run_info* out_info);

/*
 * Streamed cycle lists.  Table 1 of the paper counts the 71.5 M cycles of the 8 x 10 grid
 * without storing them, and Section 6 leaves a transport between host and GPU memory to
 * future work; this call lists every cycle of any size of output through bounded device
 * buffers.  The enumeration runs in rounds: a round stops when the next step could
 * overflow the device list, the round's cycles are copied to pinned host memory and
 * passed to `sink`, and the engine resumes from the state it left.  (Each stored level
 * carries a bound on the cycles its paths close, the sum of |Adj(v) & Adj(v1)| over its
 * paths; a level whose bound fits the list's room is expanded whole, otherwise a step
 * takes as many paths as the room holds at max_degree - 1 cycles of t + 1 vertices per
 * path.)  The CSR path is used (as for cc_cycles).
 *   chunk_cycles, chunk_vertices  device list capacity per round (cycles, vertices); at
 *                 least max(max_degree - 1, (max_degree - 1) m / 2) and
 *                 max((max_degree - 1) (L' + 1), 3 (max_degree - 1) m / 2), else CC_ERR_ARG.
 *                 Device memory: 12 chunk_cycles + 4 chunk_vertices bytes for the call,
 *                 and the same in pinned host memory, kept by the context for reuse.
 *   sink(user, count, starts, lengths, vertices, total_vertices)  called on the calling
 *                 thread after each round with cycles: cycle i is vertices[starts[i] ..
 *                 starts[i] + lengths[i]) in the canonical order of cc_cycles (original
 *                 ids, smallest first, then towards its smaller neighbour).  Cycles come in
 *                 no particular order.  The arrays are valid during the call only.
 *   out_hist, out_hash, out_tcount, out_info  as for cc_enumerate; out_rounds (or NULL):
 *                 the number of rounds.
 * Errors: those of cc_enumerate, and CC_ERR_ARG for a NULL sink or capacities below the
 * minimum.  Never CC_ERR_TRUNCATED unless the list bound is broken (a bug).
 */
typedef void (*cc_cycle_sink)(void* user, uint64_t count, const uint64_t* starts, const uint32_t* lengths,
                              const uint32_t* vertices, uint64_t total_vertices);
cc_status cc_enumerate_stream(cc_graph* g, uint32_t max_len, uint64_t chunk_cycles, uint64_t chunk_vertices,
                              cc_cycle_sink sink, void* user, uint64_t* out_hist, uint64_t* out_hash,
                              uint64_t* out_tcount, uint32_t* out_rounds, cc_run_info* out_info);

/*
 * CUDA graphs (the paper relaunches its kernels from the host, Algorithm 4; here a whole
 * call is one replayable unit).  Without out_cycles and without CC_FLAG_NO_GRAPH, the
 * second cc_enumerate of a graph with the same max_len and launch configuration captures
 * its device work (result resets, labelling, seeding, the expansion launches and the
 * result copies) into a CUDA graph kept with the cc_graph, and that call and later ones
 * with the same configuration replay it with one launch (cc_run_info.replayed).  If
 * capture is not possible the kernels are launched directly; the results are the same
 * either way.
 */

/*
 * Autotuner (the paper sets its work sizes by hand, globalSize = |SM| x MaxSMSize in
 * Section 4.4; here they are measured).  Times candidate launch configurations of
 * cc_enumerate on graph g (all lengths up to max_len) and returns the fastest:
 *   bitset or CSR adjacency (when n <= 256), threads_per_block x blocks_per_sm,
 *   paths_per_thread (bitset), the cluster phase (off, or small_phase_paths) and
 *   two-level steps (CC_FLAG_NO_FUSE).
 * Every candidate must give the same histogram and hash as the context's current options;
 * a mismatch returns CC_ERR_CUDA.  The context's options are restored before returning;
 * apply the result with cc_context_set_options(ctx, &out->best).
 *   cache_path  a JSON-lines file (one object per line: device name, graph class, the
 *               chosen knobs, time), or NULL for no cache.  A line for this device and the
 *               graph's class (adjacency kind, n and mean degree bucket, L') is returned
 *               without timing (from_cache = 1); otherwise the search runs and a line is
 *               appended.
 *   out->best   the context's options with the tuned knobs set
 */
typedef struct cc_tune_result {
  cc_options best;
  double ms_best;        /* device time (ms_proc) of the chosen configuration      */
  double ms_default;     /* of the context's options on entry                      */
  uint32_t candidates;   /* configurations timed (0 when read from the cache)      */
  uint32_t from_cache;   /* 1 if read from cache_path                              */
  char graph_class[64];  /* the cache key's class string                           */
} cc_tune_result;
cc_status cc_tune(cc_graph* g, uint32_t max_len, const char* cache_path, cc_tune_result* out);

/*
 * The same search for cc_batch_submit on the given batch (arguments as there): launch
 * shape and paths_per_thread, each candidate one whole batch, results compared graph by
 * graph.  Needs no batch outstanding on the context.
 */
cc_status cc_tune_batch(cc_context* ctx, uint32_t count, const uint32_t* n, const uint64_t* row_off,
                        const uint32_t* row_ptr, const uint64_t* col_off, const uint32_t* col_idx,
                        uint32_t max_len, const char* cache_path, cc_tune_result* out);

/*
 * Per-step trace of the last cc_enumerate on this context (Section 5, Fig. 4 of the paper
 * plots the size of T per step).  Step i expands a set of stored paths of one length (a
 * whole level, or a chunk of one when the frontier budget forces depth-first chunks).
 *   cap       entries available in t_ns and expanded (0: only *n_steps is filled)
 *   t_ns      device time (ns) from the start of the expansion to the end of step i
 *   expanded  paths expanded in step i
 *   n_steps   steps of the last call (at most 65536 are recorded)
 */
cc_status cc_get_trace(cc_context* ctx, uint32_t cap, uint64_t* t_ns, uint64_t* expanded, uint64_t* n_steps);

/*
 * Batched enumeration: `count` graphs packed back to back, all enumerated by one
 * persistent launch whose frontier mixes paths of every graph.
 *   n[g]        vertices of graph g (each <= cc_limits.max_n_batch)
 *   row_off[g]  index of graph g's first row offset in row_ptr (count+1 entries; graph g
 *               owns row_ptr[row_off[g] .. row_off[g] + n[g]], its own offsets from 0)
 *   col_off[g]  index of graph g's first neighbour in col_idx (count+1 entries)
 * The inputs are validated and copied before the call returns; the work runs
 * asynchronously on the context's stream.  One batch may be outstanding per context.
 * Errors: CC_ERR_ARG, CC_ERR_INVALID_GRAPH (the index of the first bad graph is stored
 * in *out_batch), CC_ERR_UNSUPPORTED, CC_ERR_CUDA.
 */
typedef uint64_t cc_batch_id;
cc_status cc_batch_submit(cc_context* ctx, uint32_t count, const uint32_t* n,
                          const uint64_t* row_off, const uint32_t* row_ptr,
                          const uint64_t* col_off, const uint32_t* col_idx, uint32_t max_len,
                          cc_batch_id* out_batch);

/*
 * Device-resident batches (the same work as cc_batch_submit, split so that repeated runs
 * over one set of graphs copy nothing to the device).  cc_batch_load validates and copies
 * `count` graphs (arguments as for cc_batch_submit) into device memory owned by the set
 * and returns when the copies are done (the caller may free its arrays).  cc_batch_run
 * enumerates every graph of the set with at most max_len vertices per cycle, like
 * cc_batch_submit (asynchronous; collect with cc_batch_poll on the set's context; one
 * batch in flight per context).  cc_batch_free waits for a batch of the set still in
 * flight (its results are then dropped) and frees the set.  The set belongs to the
 * context it was loaded on and must be freed before that context is destroyed.
 * Errors of cc_batch_load: CC_ERR_ARG, CC_ERR_INVALID_GRAPH and CC_ERR_UNSUPPORTED (the
 * index of the first bad graph in *bad_graph when bad_graph is not NULL), CC_ERR_OOM,
 * CC_ERR_CUDA.  Errors of cc_batch_run: CC_ERR_ARG (NULL, or a batch already in flight on
 * the context), CC_ERR_CAPACITY (the initial triplets need more than half the frontier
 * memory), CC_ERR_OOM, CC_ERR_CUDA.
 */
typedef struct cc_batch_set cc_batch_set;
cc_status cc_batch_load(cc_context* ctx, uint32_t count, const uint32_t* n, const uint64_t* row_off,
                        const uint32_t* row_ptr, const uint64_t* col_off, const uint32_t* col_idx,
                        cc_batch_set** out, uint32_t* bad_graph);
cc_status cc_batch_run(cc_batch_set* set, uint32_t max_len, cc_batch_id* out_batch);
void cc_batch_free(cc_batch_set* set);

/*
 * Wait up to timeout_us microseconds for a batch.  CC_PENDING if it is still running
 * (call again), otherwise its final status; on CC_OK the outputs are filled:
 *   hist        count * hist_stride entries; graph g's histogram at hist[g * hist_stride],
 *               entries 0..min(L'_g, hist_stride - 1); hist_stride >= 65 holds every length
 *   hash        count entries
 *   paths       count entries (stored paths per graph), or NULL
 *   done_us     count entries: microseconds from the start of the batch's expansion until
 *               the step that finished the graph's last path, or NULL
 *   info        whole-batch timings, or NULL: ms_proc = device time of labelling, seeding
 *               and expansion (from the start of the batch's device work; the input copies
 *               of cc_batch_submit are not included), ms_engine = the expansion launch,
 *               ms_total = ms_proc plus the result copies of this call
 */
cc_status cc_batch_poll(cc_context* ctx, cc_batch_id batch, uint32_t timeout_us, uint64_t* hist,
                        uint32_t hist_stride, uint64_t* hash, uint64_t* paths, double* done_us,
                        cc_run_info* info);

/*
 * Serving: a request loop with continuous batching (the paper has no counterpart; it
 * serves many graphs with the same level-synchronous expansion).
 *
 * Requests (graphs with n <= 64) are queued by cc_serve_submit.  Each cc_serve_step
 *   1. collects every in-flight request whose last path has been expanded (its result is
 *      copied to the host and its slot freed),
 *   2. admits queued requests in arrival order while a slot is free, the sum of the
 *      admitted requests' predicted frontier bytes stays within admit_bytes, and their
 *      initial triplets fit the space reserved in the live frontier; their triplets join
 *      the frontier that the running requests' paths are in,
 *   3. runs up to steps_per_round expansion steps over that shared frontier (paths of
 *      every admitted request, whatever their length), then returns.
 * Results are bit-identical to cc_enumerate on the same graph; only the timing depends on
 * the mix.  A request's predicted bytes come from the caller or, when 0, from a
 * predictor built into the library (a fit of peak stored paths against n, m and the
 * maximum degree on seeded random, grid and complete bipartite graphs).  A
 * misprediction costs only memory: a frontier that would not fit is expanded in
 * depth-first chunks.  One server per context; not thread safe.
 */
typedef struct cc_server cc_server;
typedef struct cc_serve_options {
  uint32_t slots;            /* requests in flight at most (<= 16384; 0 = 4096)            */
  uint32_t max_len;          /* cycle length bound for every request (0 = none)            */
  uint64_t admit_bytes;      /* admission budget of predicted frontier bytes (0 = 64 GiB)  */
  uint32_t steps_per_round;  /* expansion steps per cc_serve_step (0 = 8)                  */
  uint32_t pad;
  uint64_t reserve_paths;    /* frontier capacity kept free per step for admissions (0 = 2^18) */
} cc_serve_options;

typedef struct cc_completion {
  uint64_t id;           /* as returned by cc_serve_submit                           */
  uint64_t hash;         /* cycle hash (as cc_enumerate)                             */
  uint64_t total;        /* chordless cycles                                         */
  uint64_t paths;        /* stored chordless paths                                   */
  uint64_t hist[65];     /* hist[k], k <= min(L', 64)                                */
  double wait_us;        /* submit -> admission                                      */
  double latency_us;     /* submit -> result on the host                             */
} cc_completion;

/* Create a server on a context (its frontier arena is shared with cc_enumerate calls on
 * the same context, which must not run while the server has requests in flight). */
cc_status cc_serve_create(cc_context* ctx, const cc_serve_options* opts, cc_server** out);
void cc_serve_destroy(cc_server* srv);
/* Queue a request (host CSR as for cc_graph_load, n <= 64; copied).  predicted_bytes = 0
 * uses the built-in predictor.  *out_id receives the request id. */
cc_status cc_serve_submit(cc_server* srv, uint32_t n, const uint32_t* row_ptr, const uint32_t* col_idx,
                          uint64_t predicted_bytes, uint64_t* out_id);
/* One scheduling round (see above).  Up to cap completions are written to out and their
 * number to *n_out (completions beyond cap are kept for the next call).  *in_flight and
 * *queued (may be NULL) receive the requests on the GPU and still waiting. */
cc_status cc_serve_step(cc_server* srv, cc_completion* out, uint32_t cap, uint32_t* n_out, uint32_t* in_flight,
                        uint32_t* queued);
/* The built-in frontier-memory prediction for a graph with n vertices, m edges and maximum
 * degree max_degree (bytes of two consecutive stored levels at the predicted peak). */
uint64_t cc_serve_predict_bytes(uint32_t n, uint64_t m, uint32_t max_degree);

/*
 * Niche overlap graph of a food web (Section 5: the paper's food-web graphs are turned into
 * undirected niche overlap graphs, after Wilson and Watkins, before their chordless cycles
 * are enumerated).  The food web is a directed graph on n species in CSR form: prey_idx[
 * prey_ptr[x] .. prey_ptr[x+1]) are the species x feeds on (an arc x -> z; duplicates and
 * cannibalism x -> x are allowed).  Two distinct species are adjacent in the niche overlap
 * graph when they have a prey in common.  The result is a simple undirected graph in CSR
 * form with sorted rows, ready for cc_graph_load:
 *   out_row_ptr  host array of n + 1 entries, always filled
 *   out_col      host array of col_capacity entries
 *   out_nnz      receives row_ptr[n] (twice the number of edges)
 * Runs on the context's stream and device.  Errors: CC_ERR_ARG, CC_ERR_INVALID_GRAPH (offsets
 * not monotone, a prey id >= n), CC_ERR_UNSUPPORTED (n > cc_limits.max_n_csr),
 * CC_ERR_TRUNCATED (col_capacity < *out_nnz: call again with a larger array), CC_ERR_OOM,
 * CC_ERR_CUDA.
 */
cc_status cc_niche_overlap(cc_context* ctx, uint32_t n, const uint32_t* prey_ptr, const uint32_t* prey_idx,
                           uint32_t* out_row_ptr, uint32_t* out_col, uint64_t col_capacity, uint64_t* out_nnz);

/*
 * Allocation-free enumeration (the paper has no counterpart; this is a deployment aid).
 *
 * For callers that cannot allocate memory while they run: a plugin or real-time loop whose
 * host application forbids device allocations after start-up, a process whose device
 * memory is owned by another pool allocator, or a latency-critical path where
 * cudaMalloc's implicit device-wide synchronisation would stall other streams.  It does
 * what cc_enumerate does for one graph with n <= CC_NOALLOC_MAX_N, but allocates nothing
 * (no cudaMalloc/cudaFree of any kind, no host heap): all device memory it uses is one
 * fixed device array of CC_NOALLOC_SCRATCH_BYTES inside this library, which every GPU that
 * loads the library holds until the process exits.  The frontier gets what the array's
 * fixed layout leaves (about 63 MiB); larger levels are expanded in depth-first chunks.
 *
 *   n, row_ptr, col_idx  host CSR as for cc_graph_load, except that every row must already
 *                        be sorted ascending (nothing is copied to sort it); otherwise
 *                        CC_ERR_INVALID_GRAPH
 *   max_len              as for cc_enumerate
 *   stream               cudaStream_t to run on (NULL = default stream); the call returns
 *                        after the stream has finished its work
 *   out_hist, out_hash, out_tcount   host outputs as for cc_enumerate (out_tcount may be NULL)
 * Errors: CC_ERR_UNSUPPORTED if n > CC_NOALLOC_MAX_N, CC_ERR_CAPACITY if the initial triplets
 * cannot fit the array, CC_ERR_INVALID_GRAPH (also for row_ptr[n] > n (n - 1), checked before
 * col_idx is read), CC_ERR_ARG, CC_ERR_CUDA, CC_ERR_TIMEOUT.
 * The array's device address is looked up (cudaGetSymbolAddress) on the first call on each
 * device, so make that first call before any stream capture.  That address lasts as long
 * as the device's primary context: after a cudaDeviceReset (or any other reset of that
 * context) the array may move, so do not call this function on a device that was reset.  All calls share the array and
 * each call clears the parts that must start at zero; calls whose GPU work overlaps (other
 * streams or host threads) race on it and must be serialised by the caller.
 */
#define CC_NOALLOC_MAX_N 256
#define CC_NOALLOC_SCRATCH_BYTES (64ull << 20)
cc_status cc_enumerate_noalloc(uint32_t n, const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t max_len,
                               void* stream, uint64_t* out_hist, uint64_t* out_hash, uint64_t* out_tcount);

#ifdef __cplusplus
}
#endif
#endif /* CC_H_ */
