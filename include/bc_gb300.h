/*
 * bc_gb300.h -- C ABI of the exact betweenness-centrality library for one
 * NVIDIA GB300 (sm_103a).
 *
 * Problem (Kintali, "Betweenness Centrality: Algorithms and Lower Bounds",
 * Section 1.1): an undirected graph G(V,E), vertices 0..n-1, each edge with a
 * positive integer weight (unweighted = all 1). For a source s, d(s,v) is the
 * shortest-path length, sigma_s(v) (lambda_sv in the paper) the number of
 * shortest s-v paths, P_s(v) = {u : (u,v) in E, d(s,v) = d(s,u) + w(u,v)} the
 * predecessors, and delta_s*(v) the dependency given by Theorem 1.1:
 *     delta_s*(v) = sum_{w : v in P_s(w)} sigma_s(v)/sigma_s(w) * (1 + delta_s*(w)).
 * The library returns BC(v) = sum_{s in S, s != v} delta_s*(v) over a source
 * set S (all vertices by default), i.e. the sum over ORDERED pairs of the
 * paper's definition; flag BC_HALVE divides by two (unordered pairs, as the
 * paper does for undirected graphs at the end of Section 1.1).
 *
 * Arithmetic: sigma is exact uint64 (wrapping mod 2^64, with a status flag
 * when any count reaches 2^64); distances are int32; dependencies are FP32 per
 * (source, vertex); BC is summed in FP64 in a fixed order, so a run is
 * deterministic. Vertices unreachable from s contribute nothing.
 *
 * Conventions for every call:
 *   - Returns a status: 0 (BC_OK), a positive warning, or a negative error.
 *     No call throws or aborts; bc_last_error() gives a message for the last
 *     failing call on the calling thread.
 *   - Pointer arguments marked "host or device" may be either: copies use
 *     unified addressing (cudaMemcpyDefault).
 *   - cuda_stream: a cudaStream_t passed as void* (NULL = legacy default
 *     stream). A call's work starts after the work already on it and ends
 *     before anything enqueued on it later: bc_run spreads the batches over
 *     internal streams (lanes) that fork from cuda_stream when it starts and
 *     join it before it returns.
 *   - The library allocates the device memory it needs (cudaMalloc). When
 *     bc_destroy_graph frees a handle (after the device has finished its
 *     work), its device blocks, up to 24 GiB in all, and the lanes' streams and
 *     buffers are kept for the next graphs created on the same device;
 *     bc_release_cached_memory frees the cached blocks, and an allocation that
 *     fails frees them and retries. Caller buffers stay owned by the caller.
 *   - A graph handle may be used by one thread at a time. It lives on the
 *     device that is current when it is created, and every call on it
 *     (bc_destroy_graph included) must be made with that device current.
 *   - With the environment variable BC_LOG=1, bc_result writes one JSON line
 *     per completed run to stderr (sizes, options, launches, host wall time
 *     from bc_run to bc_result, edges/s, status bits).
 */
#ifndef BC_GB300_H
#define BC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define BC_OK 0
#define BC_WARN_SIGMA_OVERFLOW 1 /* results returned; some sigma reached 2^64 */
#define BC_ERR_ARG (-1)          /* bad argument (NULL, size, id out of range) */
#define BC_ERR_NOT_SYMMETRIC (-2)/* CSR is not an undirected graph (missing reverse arc, self-loop, duplicate) */
#define BC_ERR_WEIGHT (-3)       /* weight <= 0, or n * max weight >= 2^31 */
#define BC_ERR_OOM (-4)          /* device or host allocation failed */
#define BC_ERR_CUDA (-5)         /* a CUDA runtime call failed */
#define BC_ERR_TIMEOUT (-6)      /* a bounded wait gave up (see bc_options.wait_limit_ms) */
#define BC_ERR_BOUNDS (-7)       /* a device-side bounds check fired */
#define BC_ERR_UNSUPPORTED (-8)  /* option combination not supported for this graph */
#define BC_ERR_STATE (-9)        /* call out of order (e.g. bc_result before bc_run) */

/* ---- bits of the status_flags word returned by bc_result -------------- */
#define BC_STATUS_SIGMA_OVERFLOW 0x1u
#define BC_STATUS_BOUNDS 0x2u
#define BC_STATUS_LEVEL_CAP 0x4u /* internal: a batch needed more BFS levels (re-run automatically) */
#define BC_STATUS_DENSE_TIMEOUT 0x8u /* a tensor-core pipeline wait gave up (bc_result returns BC_ERR_TIMEOUT) */
#define BC_STATUS_COPY_TIMEOUT 0x10u /* a wait for staged row copies gave up (bc_result returns BC_ERR_TIMEOUT) */

/* ---- bc_create_graph flags --------------------------------------------- */
#define BC_GRAPH_TRUST_INPUT 0x1u /* skip the host-side symmetry/duplicate check */
#define BC_GRAPH_DIRECTED 0x2u    /* row_ptr/col list out-arcs of a directed graph (Section 2's model):
                                     P_s(v) takes v's in-arcs, built here as the transpose. No symmetry
                                     check (self-loops, duplicates and weights are still checked).
                                     bc_run supports it on the batched unweighted path, BC_PLAIN,
                                     the weighted path, BC_PAIRS and BC_DENSE on weighted graphs;
                                     BC_DENSE on unweighted graphs and bc_many_create return
                                     BC_ERR_UNSUPPORTED. BC is the ordered-pair sum (BC_HALVE is not
                                     meaningful for directed graphs). */

/* ---- bc_options.flags ---------------------------------------------------- */
#define BC_HALVE 0x1u        /* divide BC by 2 (unordered pairs, Section 1.1) */
#define BC_ACCUMULATE 0x2u   /* add to the previous run's BC instead of starting from 0 */
#define BC_PLAIN 0x4u        /* one source per launch sequence (the unbatched GPU Brandes) */
#define BC_TIMING 0x8u       /* record CUDA events around every kernel launch (bc_kernel_time); the run
                                uses one lane so that each launch's event time is its own */
#define BC_NO_HASH 0x10u     /* skip the per-source summary values */
#define BC_DENSE 0x20u       /* the algebraic forms of Section 3. Unweighted graphs: levels >= 1 as
                                tensor-core products with the 0/1 adjacency matrix, forward
                                (ComputePathCount) and backward (ComputeDependency), Section 3.1;
                                n <= 65536, batch 128. Weighted graphs: distance products with path
                                counts on the dense weight matrix until a step changes nothing
                                (Section 3.2), then BC by Algorithm 2's pair formula; every vertex a
                                source, n <= 16384 (bc_forward_rows: n <= 32768), n * max weight < 2^30 - 1;
                                directed or not (the unweighted tensor-core form is undirected only). */
#define BC_SPARSE_BACKWARD 0x40u /* with BC_DENSE: run the backward pass on the sparse kernel instead */
#define BC_PAIRS 0x100u      /* BC from all-pairs distances and path counts with Algorithm 2's pair formula
                                (Section 4.2.1): BC(v) = sum over ordered (s,t), d(s,v)+d(v,t)=d(s,t),
                                of lambda_sv lambda_vt / lambda_st. Needs sources = NULL, n <= 16384
                                (12 n^2 bytes of rows plus 8 n^2 of scratch); unweighted or weighted,
                                directed or not; not with BC_PLAIN / BC_DENSE. */
#define BC_KEEP_ORDER 0x80u  /* run in the caller's source order and vertex numbering. By default
                                (unweighted, batched, more than 32 sources) batches are formed from
                                the sources sorted by their BFS distances to 32 landmark vertices, so
                                the sources of one 32-source word have similar distance profiles and
                                the level sweep fetches fewer rows; and the weighted sweep runs on
                                a copy of the graph renumbered by bc_vertex_order (built on first
                                use, kept with the handle; a directed graph by its out-arcs), so that
                                neighbouring vertices share memory sectors. Either way BC differs
                                only by floating-point summation order; distances, path counts,
                                forward rows and per-source summaries are the same, in the caller's
                                order and ids. */

/* Test hook for the device-side timeout path (not for production runs):
   every staged-row wait of the level sweeps also expects 16 bytes that no
   copy delivers, so the bounded device wait (bc_options.device_wait_us)
   runs out; the warp then releases those bytes, waits for its own copies to
   land, stops staging, and bc_result returns BC_ERR_TIMEOUT. Nothing faults
   or hangs: the wait is bounded and the context stays usable. */
#define BC_TEST_WAIT_EXPIRY 0x200u
#define BC_FORCE_BOTTOMUP 0x400u /* level 0 -> 1 also by the bottom-up pull over every vertex instead of
                                    the top-down push from the sources' arcs */

/*
 * Run options. Zero-initialise and set what you need; bc_run(..., NULL, ...)
 * uses the same defaults.
 *   batch          sources per batch for the unweighted multi-source path:
 *                  32, 64, 128 or 256 (0 = 256; BC_DENSE uses 128). For
 *                  weighted graphs: sources per wave (0 = 8 per SM below
 *                  131072 vertices, else 3 per SM).
 *   flags          BC_* option bits above.
 *   chunk          arcs per work item for high-degree vertices (0 = 256 in both
 *                  sweeps; a given value applies to both).
 *   delta          bucket width of the weighted path: 0 or 1 (exact distances
 *                  settle one value at a time, which the tie-aware path counts
 *                  need); any other value returns BC_ERR_UNSUPPORTED.
 *   wait_limit_ms  bound on every host-side wait for device progress
 *                  (0 = 600000). Expiry returns BC_ERR_TIMEOUT.
 *   alpha          direction of the unweighted forward sweep at level 0 -> 1,
 *                  the level whose frontier (the batch's sources) is known before
 *                  it runs: top-down (a push over the sources' arcs) while those
 *                  arcs number fewer than 2m / alpha, the arcs a bottom-up pull
 *                  reads; else bottom-up (every vertex sums over its neighbours
 *                  in the frontier), as every later level runs. 0 = 1.
 *                  BC_FORCE_BOTTOMUP pulls regardless.
 *   beta           tail of the forward pass: the host launches levels three
 *                  ahead of the device, and one at a time once the newest
 *                  frontier holds at most beta x n vertices and under half of
 *                  the one before it (a launch past the last level still costs
 *                  a grid's start-up). 0 = 1/64.
 *   device_wait_us bound on each device-side wait for staged row copies
 *                  (0 = 2 s). Expiry sets BC_STATUS_COPY_TIMEOUT.
 */
typedef struct bc_options {
    int32_t batch;
    uint32_t flags;
    int32_t chunk;
    int32_t delta;
    int64_t wait_limit_ms;
    float alpha;
    float beta;
    int32_t device_wait_us;
    int32_t reserved0;
    int64_t reserved1[2];
} bc_options;

typedef struct bc_graph bc_graph;

/*
 * Copy a CSR graph to the device (Section 1.1's graph model).
 *   n        vertex count, 0 <= n < 2^31.
 *   row_ptr  int32[n+1] (host or device), row_ptr[0] = 0, non-decreasing.
 *   col      int32[row_ptr[n]] (host or device): neighbours of each vertex.
 *            Every undirected edge appears as both arcs.
 *   weights  int32[row_ptr[n]] arc weights (host or device), NULL = unweighted.
 *            Both arcs of an edge carry the same weight.
 *   flags    BC_GRAPH_* bits.
 *   out      receives the handle (NULL on failure).
 * Errors: BC_ERR_ARG (sizes, ids), BC_ERR_NOT_SYMMETRIC (missing reverse arc,
 * mismatched weight, self-loop, duplicate arc), BC_ERR_WEIGHT, BC_ERR_OOM,
 * BC_ERR_CUDA. The caller's arrays are not kept.
 */
int bc_create_graph(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *weights,
                    uint32_t flags, bc_graph **out);

/*
 * Betweenness over a source set: the forward pass (distances and exact path
 * counts over P_s, Section 1.1), the backward pass (Theorem 1.1) and the sum
 * over sources, all on the device.
 *   sources      int32[num_sources] (host or device), NULL = all n vertices.
 *                Ids in [0, n); repeats are allowed and counted each time.
 *   num_sources  >= 0 (ignored when sources == NULL).
 *   opt          NULL = the handle's default options (bc_autotune,
 *                bc_set_default_options), else the built-in defaults.
 * Without BC_ACCUMULATE the result starts from zero. Returns when all work is
 * enqueued on cuda_stream, except for the bounded host waits the level loop
 * needs to learn each batch's depth. Unweighted batches run on up to eight
 * concurrent lanes (batch i on lane i mod lanes, each lane with its own state
 * and BC accumulator, added in lane order at the end); weighted waves on two.
 * The assignment is fixed, so repeated runs give identical results. Errors:
 * BC_ERR_ARG, BC_ERR_OOM, BC_ERR_CUDA, BC_ERR_TIMEOUT, BC_ERR_UNSUPPORTED.
 */
int bc_run(bc_graph *g, const int32_t *sources, int32_t num_sources, const bc_options *opt,
           void *cuda_stream);

/*
 * Copy the result of the last bc_run.
 *   bc            double[n] (host or device), may be NULL.
 *   status_flags  receives BC_STATUS_* bits (may be NULL).
 * Synchronises the run's stream. Returns BC_OK, BC_WARN_SIGMA_OVERFLOW when
 * some path count reached 2^64 (BC is then not trustworthy), or an error
 * (BC_ERR_STATE before any run, BC_ERR_BOUNDS, BC_ERR_CUDA).
 */
int bc_result(bc_graph *g, double *bc, uint32_t *status_flags);

/*
 * Per-source summary values of the last bc_run, in source-list order
 * (length = number of sources run). Any pointer may be NULL; all are host or
 * device. For source s:
 *   h_sigma[i]  = sum_v (sigma_s(v) mod 2^64) * (v+1)            mod 2^64
 *   h_dist[i]   = sum_{v reachable} (d(s,v) + 1) * (v+1)         mod 2^64
 *   dist_sum[i] = sum_{v reachable} d(s,v)
 *   reach[i]    = number of vertices reachable from s (s included)
 * Errors: BC_ERR_STATE if the run used BC_NO_HASH or no run happened.
 */
int bc_source_hashes(bc_graph *g, uint64_t *h_sigma, uint64_t *h_dist, int64_t *dist_sum,
                     int64_t *reach);

/*
 * Forward-pass rows for k sources (Section 3's D and Lambda rows), computed by
 * the same kernels bc_run uses.
 *   sources  int32[k] (host or device), 0 <= k.
 *   sigma    uint64[k*n] (host or device): row i = sigma_{sources[i]}(.), 0 where unreachable.
 *   dist     int32[k*n] (host or device): d(sources[i], .), -1 where unreachable.
 * Either output may be NULL. Synchronises cuda_stream. Returns BC_OK or
 * BC_WARN_SIGMA_OVERFLOW, or an error.
 */
int bc_forward_rows(bc_graph *g, const int32_t *sources, int32_t k, uint64_t *sigma, int32_t *dist,
                    const bc_options *opt, void *cuda_stream);

/*
 * Kernel timing of the last run made with BC_TIMING: for kernel class `kind`
 * (BC_KERNEL_*), the number of launches and their summed CUDA-event durations
 * in milliseconds (events recorded on the run's stream around each launch).
 * Synchronises the stream. Errors: BC_ERR_ARG, BC_ERR_STATE.
 */
#define BC_KERNEL_INIT 0
#define BC_KERNEL_FORWARD 1
#define BC_KERNEL_BACKWARD 2
#define BC_KERNEL_HASH 3
#define BC_KERNEL_PLAIN 4
#define BC_KERNEL_DENSE 5
#define BC_KERNEL_KINDS 6
int bc_kernel_time(bc_graph *g, int32_t kind, int64_t *launches, double *total_ms);

/*
 * Per-launch trace of the last run made with BC_TIMING, in launch order:
 * kind[i] (BC_KERNEL_*), level[i] (the sweep level of a forward or backward
 * launch, -1 otherwise) and ms[i] (its CUDA-event duration). Fills at most
 * cap entries (kind, level, ms: host arrays of cap entries) and sets *count
 * (may be NULL) to the number of traced launches. Synchronises the stream.
 * Errors: BC_ERR_ARG, BC_ERR_STATE.
 */
int bc_kernel_trace(bc_graph *g, int64_t cap, int32_t *kind, int32_t *level, float *ms, int64_t *count);

/*
 * Work counters of the last bc_run (synchronises its stream):
 *   dag_arcs   sum over the run's sources s of the number of arcs (u,v) with
 *              u in P_s(v), i.e. the size of each shortest-path DAG (Section 1.1)
 *   depth_sum  sum over batches (one-source path: over sources) of the BFS depth
 *   tensor_flops  multiply-add work issued to the tensor cores by BC_DENSE in
 *              bf16 (2 * M * N * K summed over the level products), 0 otherwise
 *   tensor_flops_f8  the same for the products in e4m3 (forward levels whose
 *              counts fit four 4-bit limbs)
 * Any pointer may be NULL (host pointers). Errors: BC_ERR_ARG, BC_ERR_STATE.
 */
int bc_run_stats(bc_graph *g, int64_t *dag_arcs, int64_t *depth_sum, double *tensor_flops,
                 double *tensor_flops_f8);

/*
 * Launch parameters (the paper has no counterpart: these choose how the
 * kernels are shaped, never what they compute).
 * bc_autotune  times bc_run on `sample` sources spread over the vertex ids
 *              (0 = 2048) with CUDA events on cuda_stream, for every
 *              candidate: unweighted graphs, batch 64/128/256 x chunk
 *              128/256/512, then beta 1/256, 1/64, 1/16; weighted graphs,
 *              1/2/3/4/8 sources per SM per wave. The fastest becomes the
 *              handle's default (bc_run with opt = NULL uses it) and is copied
 *              to *out (may be NULL). The handle's previous result is
 *              overwritten. Errors: those of bc_run.
 * bc_set_default_options  installs *opt as what bc_run uses for opt = NULL
 *              (a tuned choice kept from an earlier process); NULL restores
 *              the built-in defaults.
 * bc_last_options  the options the last bc_run ran with, after that
 *              substitution (all zero for the built-in defaults).
 */
int bc_autotune(bc_graph *g, int32_t sample, bc_options *out, void *cuda_stream);
int bc_set_default_options(bc_graph *g, const bc_options *opt);
int bc_last_options(const bc_graph *g, bc_options *out);

/* Number of kernel launches the last bc_run issued (all kinds). */
int64_t bc_launch_count(const bc_graph *g);

/* Vertex and undirected edge counts of a graph handle. */
int bc_graph_size(const bc_graph *g, int32_t *n, int64_t *m, int32_t *weighted);

/*
 * bc_run_noalloc -- betweenness for callers that cannot allocate.
 * The paper has no counterpart: this is a deployment variant of bc_run for
 * callers that may not call cudaMalloc (a custom allocator or memory pool owns
 * the device, a host process forbids allocation after start-up, a fixed
 * memory footprint is required). It allocates nothing: its scratch is one
 * file-scope __device__ array of BC_NOALLOC_SCRATCH_BYTES that every GPU on
 * which the library is loaded holds until the process exits.
 *   n            vertex count, 0 <= n <= BC_NOALLOC_MAX_N.
 *   row_ptr      int32[n+1], col int32[row_ptr[n]]: DEVICE pointers to an
 *                undirected CSR (both arcs of each edge; symmetry is not
 *                checked here, as with BC_GRAPH_TRUST_INPUT). Unweighted.
 *   sources      DEVICE int32[num_sources] (ids in [0, n), at most
 *                BC_NOALLOC_MAX_N of them), or NULL for all vertices.
 *   bc           DEVICE double[n]: receives the ordered-pair betweenness.
 * Runs on cuda_stream and synchronises it several times (it checks the
 * inputs and reads each batch's depth back to the host).
 * Returns BC_OK, BC_WARN_SIGMA_OVERFLOW, BC_ERR_ARG (sizes beyond the limits,
 * NULL pointers, ids out of range), BC_ERR_UNSUPPORTED (a BFS deeper than
 * BC_NOALLOC_MAX_LEVELS levels), BC_ERR_TIMEOUT (a bounded device wait for
 * staged row copies gave up: the result is incomplete), BC_ERR_CUDA. No
 * message is recorded for bc_last_error (that would allocate); use
 * bc_status_string.
 * The first call on a device looks up the array's device address for that
 * device (cudaGetSymbolAddress); make that first call before any stream
 * capture begins. Every call on a device shares the one array and leaves its
 * contents behind (each call clears what must start at zero): calls that
 * overlap on the GPU race and must not be issued concurrently.
 */
#define BC_NOALLOC_MAX_N 16384
#define BC_NOALLOC_MAX_LEVELS 62
#define BC_NOALLOC_SCRATCH_BYTES (24u << 20)
int bc_run_noalloc(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *sources,
                   int32_t num_sources, double *bc, void *cuda_stream);

/*
 * Many graphs in one persistent launch: exact all-sources betweenness of k
 * independent unweighted graphs (the paper's definitions, every vertex of
 * every graph a source).
 *
 * bc_many_create  builds the plan: work items (graph, range of source
 *                 batches), ordered longest first and taken by CTAs from an
 *                 atomic queue; per-CTA workspaces; the reset and the
 *                 persistent kernel captured once into a CUDA graph.
 *                 graphs: k unweighted handles from bc_create_graph, owned by
 *                 the caller and kept alive while the plan exists.
 *                 opt->batch: sources per batch, 32, 64, 128 or 256 (0 = 32).
 *                 opt->flags: BC_NO_HASH skips the per-source summaries.
 * bc_many_run     replays the captured graph on cuda_stream (asynchronous).
 *                 Each graph's BC lands in its own handle: read it with
 *                 bc_result(graphs[i], ...) after bc_many_result, and its
 *                 per-source summaries (every vertex a source, in vertex
 *                 order) with bc_source_hashes(graphs[i], ...).
 * bc_many_result  synchronises; a graph deeper than the launch's level
 *                 capacity (64 levels) is re-run with bc_run on the same
 *                 stream; *rerun (may be NULL) receives how many were.
 *                 Returns BC_OK or BC_WARN_SIGMA_OVERFLOW, or an error.
 * bc_many_stats   after bc_many_result: the shortest-path DAG arcs (Section
 *                 1.1's P_s(v) relations) summed over every source of every
 *                 graph the persistent launch completed (re-run graphs not
 *                 included).
 * bc_run_many     create + run + result + destroy in one call.
 * Errors: BC_ERR_ARG, BC_ERR_UNSUPPORTED (a weighted handle), BC_ERR_OOM,
 * BC_ERR_CUDA, BC_ERR_STATE.
 */
typedef struct bc_many bc_many;
int bc_many_create(bc_graph *const *graphs, int32_t k, const bc_options *opt, bc_many **out);
int bc_many_run(bc_many *plan, void *cuda_stream);
int bc_many_result(bc_many *plan, uint32_t *status_flags, int32_t *rerun);
int bc_many_stats(const bc_many *plan, int64_t *dag_arcs);
void bc_many_destroy(bc_many *plan);
int bc_run_many(bc_graph *const *graphs, int32_t k, const bc_options *opt, void *cuda_stream);

/* Free the handle and its device memory (its device blocks go to the cache
 * described at the top). Synchronises the device first. NULL is ignored. */
void bc_destroy_graph(bc_graph *g);

/* Free the device blocks cached from destroyed handles (every device). Call
 * it with no library call in flight. */
void bc_release_cached_memory(void);

/* A vertex numbering with locality, from the CSR alone (host code; no GPU
 * needed). Not part of the paper's method: it is the memory layout the
 * weighted sweep runs on (see BC_KEEP_ORDER). Multilevel
 * heavy-edge matching: each level matches every node, in id order, with the
 * unmatched neighbour joined to it by the most edges; matched pairs become the
 * next level's nodes. Vertices are then numbered by their ancestors, top level
 * first, so each run of consecutive new ids is a connected cluster as a rule.
 *   n                 vertices (>= 0)
 *   row_ptr [n+1]     host, CSR row offsets (row_ptr[0] = 0, non-decreasing)
 *   col [row_ptr[n]]  host, arc heads in [0, n)
 *   perm [n]          host, written: perm[v] = the new id of v (a permutation)
 * Deterministic. Returns BC_OK, or BC_ERR_ARG for a NULL pointer, n < 0, a
 * malformed row_ptr or a head out of range (perm untouched). */
int bc_vertex_order(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t *perm);

/* Static text for a status code. */
const char *bc_status_string(int status);

/* Message of the last failing call on this thread ("" if none). */
const char *bc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BC_GB300_H */
