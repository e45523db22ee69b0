/*
 * ldl.h -- C ABI of the GB300 LD-Leiden batch-update library.
 *
 * The library keeps a weighted graph, its community partition and its Leiden
 * hierarchy resident on one GPU and updates them batch by batch, following the
 * paper's Algorithm 1 (LD-Leiden batch update): apply the edge batch, repair
 * the statistics along the parent chain, then run frontier-restricted move,
 * refine and aggregate-repair stages level by level.  The partition quality is
 * the directed weighted modularity of Eq. 1; moves are ranked by the exact
 * one-step gain of Eq. 2; accepted moves pass the decoupling filter of
 * Sec. III-E; aggregate levels are repaired by the subtract-add rule of Eq. 3.
 *
 * All arithmetic that decides anything is integer (int64 weights and totals,
 * int128 gains), so results are bit-reproducible and independent of launch
 * configuration.
 *
 * Conventions
 *   - Vertex ids are int32 in [0, n); n is fixed at creation.
 *   - Undirected graphs are symmetric weight matrices: an edge {i, j} is the
 *     two arcs (i, j) and (j, i); a self-loop is one arc.  m = sum_ij w_ij.
 *   - Level-0 weights are int32 >= 1; aggregate weights and all totals int64.
 *   - Every entry point returns an ldl_status; LDL_OK is 0, and
 *     ldl_last_error() describes a failure.  A batch is atomic: a batch
 *     rejected by validation (RANGE, INVALID, NEG_WEIGHT, NO_EDGE, OVERFLOW)
 *     changes nothing, and an error in the middle of a batch (NOMEM, TIMEOUT,
 *     an internal INVALID) is rolled back, leaving the state exactly as it
 *     was before the call (see ldl_params.no_rollback).  A CUDA error that
 *     leaves the device context broken can prevent the rollback; the context
 *     then reports LDL_E_CUDA on every later call and must be destroyed.
 *   - Pointers marked "host" are read or written with ordinary host access;
 *     "device" pointers are GPU global memory of the context's device.
 *   - The context owns all device state.  Pointers it returns stay valid until
 *     the next ldl_apply_batch() or ldl_destroy() on that context.
 *   - A context lives on the device that was current at ldl_create(); every
 *     entry point makes that device current for its duration and restores the
 *     caller's current device before it returns.
 *   - A context is not thread safe; distinct contexts are independent.
 */
#ifndef LDL_H
#define LDL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ldl_ctx ldl_ctx;

typedef enum {
  LDL_OK = 0,
  LDL_E_INVALID = 1,    /* malformed argument, op code or CSR */
  LDL_E_RANGE = 2,      /* vertex id outside [0, n) */
  LDL_E_NO_EDGE = 3,    /* delete or reweight of an absent edge */
  LDL_E_NEG_WEIGHT = 4, /* reweight to a negative weight */
  LDL_E_NOMEM = 5,      /* device allocation failed */
  LDL_E_CUDA = 6,       /* CUDA runtime error */
  LDL_E_TIMEOUT = 7,    /* a bounded device wait gave up */
  LDL_E_OVERFLOW = 8    /* weight above INT32_MAX or m >= 2^50 */
} ldl_status;

/* Edge-update op codes (Sec. II: every op is a signed weight increment). */
enum { LDL_INSERT = 0, LDL_DELETE = 1, LDL_REWEIGHT = 2 };

/*
 * Parameters.  N, L, M, alpha = 1/alpha_inv and beta = 1/beta_inv are the
 * budgets and thresholds of Algorithm 1; the paper's defaults (Sec. IV-D) are
 * N=2, L=4, M=5, alpha=0.001, beta=0.01.  gamma = gamma_num/gamma_den is the
 * Eq. 1 resolution (1 in all of the paper's experiments); both parts must be
 * in [1, 1024].  M_static is the round budget of the static Leiden run that
 * builds the initial hierarchy in ldl_create (default 20).  cuda_stream is a
 * cudaStream_t (NULL: the legacy default stream).
 */
typedef struct {
  int32_t directed;
  int32_t gamma_num, gamma_den;
  int32_t N, L, M, M_static;
  int32_t alpha_inv, beta_inv;
  /* Sweep scheduling (no effect on results): rows of 2049 .. cluster_max_deg
   * entries (at most 32768) are swept by one 8-block cluster with a
   * distributed shared-memory hash instead of the whole-GPU hub path;
   * 0 (the default) keeps every row above 2048 entries on the hub path. */
  int32_t cluster_max_deg;
  /* 1: collect the sweep kernel statistics (ldl_get_kernel_stats) from the
   * start, so that they cover the static build inside ldl_create; 0 (the
   * default): off until ldl_set_kernel_stats. */
  int32_t kernel_stats;
  /* Degree bins of the sweeps (no effect on results): a node with d
   * adjacency entries (out + in) goes to 8-lane groups if d <= bin_deg[0],
   * one warp if d <= bin_deg[1], a 128-thread block if d <= bin_deg[2], a
   * 256-thread block if d <= bin_deg[3], else to the cluster / hub paths.
   * 0 keeps an entry's default (24, 96, 1024, 2048); the bounds must not
   * decrease and must not exceed (32, 128, 1024, 2048), the largest degrees
   * whose hash tables stay at most half full (LDL_E_INVALID otherwise). */
  int32_t bin_deg[4];
  /* 0 (the default): every ldl_apply_batch is atomic.  Before the batch
   * changes anything the library copies the per-level node arrays and the
   * community totals (about 21 bytes per node and level, 29 when directed,
   * into a buffer kept by the context), and every adjacency update of the
   * batch logs the old row tables, row contents and weights it overwrites,
   * so that an error in the middle of the batch (NOMEM, TIMEOUT, an internal
   * error) restores the state exactly as it was.  1: no copy and no log
   * (saves that memory and time; an error in the middle of a batch then
   * leaves the context unusable). */
  int32_t no_rollback;
  void* cuda_stream;
} ldl_params;

/* Fills p with the defaults above (undirected, gamma = 1). */
void ldl_default_params(ldl_params* p);

/*
 * One edge update (Sec. II batch Delta_t): INSERT adds w >= 1 to the weight of
 * (src, dst) (creating the edge if absent), DELETE removes the edge (w is
 * ignored), REWEIGHT sets the weight to w >= 0 (0 removes the edge).  Several
 * updates of one edge in a batch apply in array order.  For undirected graphs
 * (src, dst) and (dst, src) name the same edge and both arcs change.
 */
typedef struct {
  int32_t src, dst, op, w;
} ldl_update;

/*
 * Result of the last batch: the pair (H_t, P_t) that Algorithm 1 returns.
 * labels is the level-0 partition P_t (device, int32[n], owned by the
 * context).  changed lists the vertices whose label differs from before the
 * batch (device, int32[n_changed]).  levels is the hierarchy height T+1, and
 * the hierarchy H_t itself is given per level r < levels as host arrays of
 * device pointers (all owned by the context): parent[r] is pi_r (int32[n]; -1
 * for nodes absent at level r and at the top level), comm[r] is the level-r
 * community labels P^r (int32[n]), refined[r] is the refined community of
 * every level-r node (int32[n]; refined communities are named by their
 * level-(r+1) node, so refined[r] and parent[r] are the same array), and
 * alive[r] marks the nodes that exist at level r (uint8[n]).  Node ids are in
 * [0, n) at every level.  The counters describe the work done.
 */
typedef struct {
  const int32_t* labels;
  int64_t n;
  const int32_t* changed;
  int64_t n_changed;
  int32_t levels;
  const int32_t* const* parent;
  const int32_t* const* comm;
  const int32_t* const* refined;
  const uint8_t* const* alive;
  int64_t frontier_nodes[8]; /* |A^r| summed over passes, per level */
  int64_t edges_scanned;     /* adjacency entries read by BestMove / BestRef */
  int64_t moves, refine_moves, rejected, rollbacks, rounds, agg_records;
  int64_t decouple_rounds;   /* parallel resolution rounds of the decoupling filter */
  int64_t host_syncs;        /* counter reads that waited for the device */
  int64_t pending_records;   /* weight records queued for levels >= 1 (before summing) */
  int64_t pending_applied;   /* distinct arcs those records changed when applied */
  int64_t split_members;     /* members of refined communities re-checked for connectivity */
} ldl_result;

/*
 * ldl_create -- upload a CSR snapshot and build the initial hierarchy with the
 * deterministic static Leiden run (every node active, move / refine /
 * aggregate from singletons, up to level L).
 *   n        vertices (1 .. 2^31-1)
 *   nnz      stored entries; row_ptr int64[n+1] with row_ptr[0]=0,
 *            row_ptr[n]=nnz; col int32[nnz] in [0,n); w int32[nnz] >= 1
 *            (host).  Repeated (row, col) entries are summed.  Undirected
 *            CSR must be symmetric.
 *   out      receives the context on LDL_OK.
 * Errors: INVALID (bad sizes, params, asymmetric undirected input, w < 1),
 * RANGE (col outside [0,n)), OVERFLOW (summed weight > INT32_MAX or
 * m >= 2^50), NOMEM, CUDA.
 */
ldl_status ldl_create(const ldl_params* params, int64_t n, int64_t nnz, const int64_t* row_ptr,
                      const int32_t* col, const int32_t* w, ldl_ctx** out);

/*
 * ldl_apply_batch -- Algorithm 1 for one batch of `count` updates.
 *   updates  host array (updates_on_device = 0) or device array (= 1) of
 *            ldl_update; read only, may be freed after the call.
 *   out      optional (may be NULL); filled on LDL_OK.
 * Errors: RANGE, INVALID, NEG_WEIGHT, NO_EDGE, OVERFLOW (validation: the
 * lowest-index failing update decides; single-update checks come before
 * sequence checks), NOMEM, TIMEOUT (a bounded wait inside a device scan gave
 * up), CUDA.  On every error the state is as it was before the call (unless
 * no_rollback is set, or the CUDA context itself broke).
 */
ldl_status ldl_apply_batch(ldl_ctx* ctx, const ldl_update* updates, int64_t count,
                           int32_t updates_on_device, ldl_result* out);

/* Eq. 1 modularity of the current partition, from the maintained integer
 * numerator (no graph scan): q = Qnum / (gamma_den * m^2). */
ldl_status ldl_modularity(const ldl_ctx* ctx, double* q);

/* The exact numerator gamma_den*m^2*Q as two's-complement (hi, lo) halves, and m. */
ldl_status ldl_modularity_num(const ldl_ctx* ctx, int64_t* q_hi, uint64_t* q_lo, int64_t* m);

/* Frees every device allocation of the context.  NULL is ignored. */
void ldl_destroy(ldl_ctx* ctx);

/* Text of the last error on ctx (or of the last failed ldl_create when ctx is
 * NULL); never NULL. */
const char* ldl_last_error(const ldl_ctx* ctx);

/* ----------------------------------------------------------------------------
 * Execution forms (the arithmetic of every context is that of ldl_apply_batch)
 * -------------------------------------------------------------------------- */

/*
 * Batched form: applies updates[i] (counts[i] entries) to ctxs[i] for i < g,
 * concurrently from `threads` host threads (0: up to 16).  Contexts created
 * with distinct cuda_stream values overlap on the device; contexts must be
 * distinct.  statuses / results (optional, length g) receive each context's
 * outcome; the return value is LDL_OK or the first failing status.
 */
ldl_status ldl_apply_batches(ldl_ctx* const* ctxs, const ldl_update* const* updates, const int64_t* counts,
                             int32_t g, int32_t updates_on_device, int32_t threads, ldl_status* statuses,
                             ldl_result* results);

/* Estimated device bytes of a context with n vertices and nnz stored entries. */
ldl_status ldl_estimate_bytes(const ldl_params* params, int64_t n, int64_t nnz, int64_t* bytes);

/* Estimated new device bytes one batch of `count` updates may allocate on ctx:
 * the rollback snapshot (first batch), record buffers beyond their current
 * capacity, and pool compactions of levels whose slack headroom is short, and
 * at least `count` times the most device memory per update that any earlier
 * batch of this context asked for (a batch whose frontier reaches hubs can
 * touch most of the graph).  A planning figure for admission, not a bound: a
 * batch that runs out of memory anyway is rolled back (LDL_E_NOMEM, state
 * unchanged). */
ldl_status ldl_batch_estimate_bytes(const ldl_ctx* ctx, int64_t count, int64_t* bytes);

/*
 * Served form: a request server with `workers` host threads.  Requests
 * (batches) on one context run in submission order; requests on different
 * contexts overlap on the device (give each context its own stream).
 * ldl_server_admit creates a context only when the device's free memory,
 * less what running requests have reserved, covers its estimated footprint
 * (LDL_E_NOMEM otherwise, nothing allocated); admissions are serialised.
 * ldl_server_submit copies the host updates and returns a ticket.  Each
 * request is admitted to the device by memory too: a worker starts the oldest
 * request whose context is idle and whose estimated growth
 * (ldl_batch_estimate_bytes) fits the free memory less the reservations of
 * running requests; a request that does not fit waits (deferred, keeping its
 * context's order) until a running request finishes, and one that runs out of
 * memory while others run is rolled back and queued again.  ldl_server_wait
 * blocks until the ticket's batch is done (timeout_ms < 0: no limit;
 * LDL_E_TIMEOUT when it runs out) and reports its status, result, time queued
 * (submission to first start) and time in service (microseconds).  The
 * result's counters belong to that batch; its device pointers (labels,
 * changed, the hierarchy) point at the context's live state, which later
 * requests on the same context may already have changed by the time the wait
 * returns.  A ticket can be waited once.  ldl_server_destroy runs the queue
 * dry and joins the workers.
 */
typedef struct ldl_server ldl_server;
ldl_status ldl_server_create(int32_t workers, ldl_server** out);
ldl_status ldl_server_admit(ldl_server* server, const ldl_params* params, int64_t n, int64_t nnz,
                            const int64_t* row_ptr, const int32_t* col, const int32_t* w, ldl_ctx** out);
ldl_status ldl_server_submit(ldl_server* server, ldl_ctx* ctx, const ldl_update* updates, int64_t count,
                             int64_t* ticket);
ldl_status ldl_server_wait(ldl_server* server, int64_t ticket, int32_t timeout_ms, ldl_status* status,
                           ldl_result* result, double* queue_us, double* service_us);
void ldl_server_destroy(ldl_server* server);

/* Requests deferred for memory at least once, and requests rolled back and
 * queued again after running out of memory, since the server started. */
ldl_status ldl_server_stats(ldl_server* server, int64_t* deferred, int64_t* retried);

/* Test hook: admission decisions use `bytes` as the device's free memory
 * (-1: ask the device again). */
ldl_status ldl_server_debug_free_bytes(ldl_server* server, int64_t bytes);

/* ----------------------------------------------------------------------------
 * Checkpoint / resume and vertex-set growth.  The hierarchy H_t is the state
 * a batch update resumes from (Sec. III-A); the vertex set V_t may change
 * between batches (Sec. II).
 * -------------------------------------------------------------------------- */

/* Writes the context's whole state (parameters, every level's graph, parent
 * map, labels, strengths and node existence, the community totals and the
 * exact modularity numerator) to a file.  LDL_E_INVALID if the file cannot
 * be written; the context is unchanged. */
ldl_status ldl_save(const ldl_ctx* ctx, const char* path);

/* Creates a context from a file written by ldl_save, on the current device,
 * without rerunning the static build: it continues exactly where the saved
 * context stood.  params may be NULL; otherwise only its cuda_stream,
 * kernel_stats, cluster_max_deg, bin_deg and no_rollback are taken (the
 * method's parameters N, L, M, alpha, beta, gamma are those saved).
 * LDL_E_INVALID for a missing, truncated or inconsistent file (the reason is
 * in ldl_last_error(NULL)); NOMEM, CUDA. */
ldl_status ldl_load(const char* path, const ldl_params* params, ldl_ctx** out);

/* Grows the vertex set to n_new >= n: the new vertices n .. n_new-1 are
 * isolated, each its own community and, at every level, its own node whose
 * parent is the node of the same id one level up (so later batches may
 * connect them like any vertex).  The modularity is unchanged.  The context
 * keeps its handle; device pointers it returned before are invalid after
 * the call.  On an error the context is unchanged (INVALID for n_new < n or
 * above 2^31-2, NOMEM, CUDA). */
ldl_status ldl_grow(ldl_ctx* ctx, int64_t n_new);

/* ----------------------------------------------------------------------------
 * Introspection (copies device state to host; for tests and tooling).
 * -------------------------------------------------------------------------- */

/* Hierarchy height T+1. */
int32_t ldl_levels(const ldl_ctx* ctx);

/* Vertex count n, and 1 for a directed graph (0 undirected); 0 for NULL. */
int64_t ldl_num_vertices(const ldl_ctx* ctx);
int32_t ldl_is_directed(const ldl_ctx* ctx);

/*
 * Per-node arrays of level r (0 <= r <= T), each of length n (host, caller
 * allocated; any may be NULL): lab = P^r, par = pi_r (-1 at the top level or
 * for absent nodes), kout / kin = strengths, cnt = number of level r-1
 * children (1 at level 0), alive = 1 when the node exists at level r.
 */
ldl_status ldl_get_level(const ldl_ctx* ctx, int32_t r, int32_t* lab, int32_t* par,
                         int64_t* kout, int64_t* kin, int32_t* cnt, uint8_t* alive);

/* Number of stored out-arcs at level r. */
ldl_status ldl_level_nnz(const ldl_ctx* ctx, int32_t r, int64_t* nnz);

/* Out-adjacency of level r as CSR sorted by (row, col) (host, caller
 * allocated: row_ptr int64[n+1], col int32[nnz], w int64[nnz]). */
ldl_status ldl_get_adjacency(const ldl_ctx* ctx, int32_t r, int64_t* row_ptr, int32_t* col,
                             int64_t* w);

/* Community totals K^out, K^in and internal weight e, int64[n] each (host). */
ldl_status ldl_get_communities(const ldl_ctx* ctx, int64_t* kout, int64_t* kin, int64_t* e);

/* Device time in milliseconds spent in each stage since timing was last
 * enabled: [ingest, repair, expand, bestmove, decouple, commit, refine,
 * aggregate, pushdown]; `times` has room for 16.  ldl_set_timing(ctx, 1)
 * enables the events (one synchronisation per stage) and resets the sums. */
ldl_status ldl_stage_times(const ldl_ctx* ctx, double* times);
ldl_status ldl_set_timing(ldl_ctx* ctx, int32_t on);

/* Copies the last batch's changed vertices (ids) and their new labels to host
 * arrays of length n_changed (labels may be NULL). */
ldl_status ldl_copy_changed(const ldl_ctx* ctx, int32_t* ids, int32_t* labels);

/*
 * Same result as ldl_copy_changed, without any device allocation, for callers
 * that cannot allocate device memory while they run (a serving loop that
 * reserved its memory at start-up, a process whose device memory is held by
 * another framework's caching allocator, a real-time path that forbids
 * allocator calls).  The paper has no counterpart; this is an interface
 * convenience.  The labels are gathered into a static device array of
 * 2^20 int32 (4 MiB per device, held until the process exits); a batch with
 * more than 2^20 changed vertices is rejected with LDL_E_INVALID (use
 * ldl_copy_changed).  The first call on a device looks up the array's device
 * address, so make that first call before any stream capture.  All calls share
 * the array: calls whose GPU work overlaps (different streams or contexts at
 * the same time) race and must be serialised by the caller.  ids and labels
 * are host arrays of length n_changed.
 */
ldl_status ldl_copy_changed_noalloc(const ldl_ctx* ctx, int32_t* ids, int32_t* labels);

/* Number of CUDA kernels this library has launched in this process. */
int64_t ldl_launch_count(void);

/*
 * Per-kernel statistics of the BestMove / BestRef sweep kernels, measured
 * with CUDA events on the context's stream while enabled (enabling resets
 * them).  out[28] = {launches, ms, algorithmic bytes, entries} for, in this
 * order, k_sweep_group with 8-lane groups (one group per node of at most
 * bin_deg[0] entries), k_sweep_group with whole warps (<= bin_deg[1]),
 * k_sweep_block with 128 threads (<= bin_deg[2]), k_sweep_block with 256
 * threads (<= bin_deg[3]), k_sweep_cluster (a cluster of 8 blocks with a distributed
 * shared-memory hash, <= cluster_max_deg entries), k_hub_acc (the hub rows
 * spread over the GPU into global hash tables) and the rest of the hub path
 * (table set-up, evaluation and final reduction kernels).
 * Algorithmic bytes count, per adjacency entry, the neighbour id, its weight
 * and its label (refinement: also its parent); per swept node its offsets,
 * lengths, label and strengths; per evaluated (node, target) pair the
 * target's totals.  Collection adds no host synchronisation: events and
 * device counters are resolved by ldl_get_kernel_stats, which waits for the
 * context's stream.  Both return LDL_E_INVALID on a null pointer and
 * LDL_E_CUDA on a CUDA error.
 */
ldl_status ldl_set_kernel_stats(ldl_ctx* ctx, int32_t on);
ldl_status ldl_get_kernel_stats(const ldl_ctx* ctx, double* out);

/* Test hook: make the k-th device allocation from now on fail (k >= 1);
 * k = 0 disables.  Lets a test check that NOMEM leaves the state intact. */
void ldl_debug_fail_alloc_after(int64_t k);

/* Test hook: device allocations attempted by this library so far, in total
 * and while a batch was in the middle of changing a context's state (after
 * its snapshot); either pointer may be NULL. */
void ldl_debug_alloc_counts(int64_t* all, int64_t* in_batch);

/*
 * Test hook for the decoupling filter of Sec. III-E: runs the library's
 * device filter (the one-block rounds for up to 8192 candidates, the
 * cooperative multi-block rounds above) on `count` explicit candidates
 * (host arrays): node v[k] moving from community src[k] to dst[k] with the
 * exact gain (g_hi[k], g_lo[k]) (two's-complement halves of an int128).
 * accepted[k] receives 1 for an accepted candidate, 0 otherwise.  Ids lie in
 * [0, n) of the context, nodes are distinct, src != dst and count <= n
 * (LDL_E_INVALID otherwise).  Uses the context's scratch buffers only: its
 * graph, hierarchy and result are unchanged.
 */
ldl_status ldl_debug_decouple(ldl_ctx* ctx, int64_t count, const int32_t* v, const int32_t* src, const int32_t* dst,
                              const int64_t* g_hi, const uint64_t* g_lo, uint8_t* accepted);

/* Test hook for the device radix sort that orders every record set (batch
 * updates, aggregate records, pending records, children records) before it
 * is reduced or applied: sorts `count` (key, value) pairs (host arrays,
 * replaced by their sorted order) stably by the low `bits` bits of the key
 * (1 <= bits <= 64; higher key bits must be zero).  The library picks the
 * one-block, single cooperative launch or multi-launch form by count, as it
 * does for its own sorts.  Uses the context's scratch buffers and stream
 * only.  Returns LDL_E_INVALID on bad arguments. */
ldl_status ldl_debug_sort_pairs(ldl_ctx* ctx, int64_t count, uint64_t* keys, uint64_t* vals, int32_t bits);

/* Test hook: the number of hub hash-table slots a sweep holds at once
 * (default 2^28, 3 GB; slots <= 0 restores it).  Hubs whose tables exceed it
 * together are swept in consecutive groups; a small value makes ordinary
 * graphs take that path.  Process-wide. */
void ldl_debug_hub_table_slots(int64_t slots);

/* Test hook for the bounded waits: runs a two-tile device scan in which the
 * first tile never publishes its sum, so the second tile's look-back wait
 * runs out (after about 2^20 polls).  Returns LDL_E_TIMEOUT when the wait gave
 * up and reported it (the expected outcome), LDL_OK if it did not, or
 * LDL_E_NOMEM / LDL_E_CUDA.  Touches no context. */
ldl_status ldl_debug_scan_wait_timeout(void);

#ifdef __cplusplus
}
#endif

#endif /* LDL_H */
