// Host-side launchers of the algorithm kernels (sweep.cu, hier.cu).
#pragma once
#include "ctx.cuh"

struct CommitOut {
  i128 dq;     // exact change of the Eq. 1 numerator
  i128 dp;     // change of sum_C K_out K_in
  int64_t de;  // change of sum_C e_C
  int32_t ntc; // touched communities
};

// Degree bins of the sweeps: a node with d adjacency entries goes to the
// first bin whose bound is >= d (8-lane groups, warps, 128-thread blocks,
// 256-thread blocks; beyond: clusters / hub path).  Default bounds, and the
// largest bound each bin's hash table allows while staying at most half full.
constexpr int32_t BIN_DEFAULT[4] = {24, 96, 1024, 2048};
constexpr int32_t BIN_MAX[4] = {32, 128, 1024, 2048};

// ---- sweep.cu
void expand_set(ldl_ctx& c, int r, const int32_t* list, int idx_n, int32_t* stamp, int32_t ep, int32_t* olist,
                int idx_out, int64_t n_hint);
void filter_alive(ldl_ctx& c, int r, const int32_t* list, int idx_n, int32_t* olist, int idx_out, int64_t n_hint);
void union_into(ldl_ctx& c, const int32_t* list, int idx_n, int32_t* stamp, int32_t ep, int32_t* olist, int idx_out,
                int64_t n_hint);
// BestMove (mode 0) / BestRef (mode 1) over the listed nodes; the candidates
// and their count (counter K_CAND) stay on the device.  Returns the list's
// length (dcnt[idx_n]), read with the sweep's bin counts.
int32_t sweep(ldl_ctx& c, int r, int mode, const int32_t* list, int idx_n, int64_t n_hint);
// Decoupling filter over the last sweep's candidates: returns their number
// and the number accepted (the accepted moves are in bv / bsrc / bdst), and
// counter `extra` (when >= 0) read in the same host wait.
struct DecoupleOut {
  int32_t nc, nb, extra;
};
DecoupleOut decouple(ldl_ctx& c, int extra = -1);
// Launches the commit of a mini-batch; commit_read then reads its outcome
// (with the counter dcnt[extra_idx] in the same read when extra is given).
void commit_move(ldl_ctx& c, int r, int32_t nb, int32_t epB, int32_t epT, int32_t epCh);
CommitOut commit_read(ldl_ctx& c, int extra_idx, int32_t* extra);
void rollback_move(ldl_ctx& c, int r, int32_t nb, int32_t ntc);
void mark_moved(ldl_ctx& c, int r, int32_t nb, int32_t epMv, int32_t epM0);
void commit_ref(ldl_ctx& c, int r, int32_t nb);
void spexpand(ldl_ctx& c, int r, int32_t nb, int32_t epD, int32_t epR, int32_t* lR, int idx_R);

// ---- hier.cu
// Batch validation and net deltas; leaves the sorted arcs in (c.rk, c.rv)
// and returns their count.  Throws (state untouched) on a bad batch.
int64_t ingest(ldl_ctx& c, const ldl_update* upd, int64_t count, int on_device, int64_t* dm);
// Apply the level-0 arcs to the adjacency and repair every statistic along
// the parent chain; marks InitFrontier in the A lists (epA per level).
void repair_batch(ldl_ctx& c, int64_t na, const int32_t* epA, int32_t epT, int64_t dm);
void pending_reset(ldl_ctx& c);
// known: the level's pending record count when the caller has read it, else -1
void flush_level(ldl_ctx& c, int q, int64_t known = -1);
// moved_ub: an upper bound of the level's moved nodes (0 when none moved)
void pushdown(ldl_ctx& c, int r, int32_t epCh, int64_t moved_ub);
int32_t dissolve_all(ldl_ctx& c, int r, int32_t epD);
int32_t split(ldl_ctx& c, int r, int32_t epD, int32_t epX);
// the listed level-r nodes that are singleton refined communities -> out
// (their count stays on the device, at dcnt[idx_out])
void singletons_of(ldl_ctx& c, int r, const int32_t* list, int idx_n, int64_t n_hint, int32_t* out, int idx_out);
// nD = |D| (list lD), the nodes whose refined community changed.
void aggregate(ldl_ctx& c, int r, int32_t epD, int32_t epC, int32_t epA_next, bool build, int32_t nD);
// context set-up and tear-down (ldl.cu)
void alloc_globals(ldl_ctx& c);
void free_all(ldl_ctx& c);
ldl_status ctx_new(const ldl_params& p, int64_t n, ldl_ctx** out);
void set_create_error(const std::string& msg);
// static set-up of level 0 from a host CSR
void upload_graph(ldl_ctx& c, int64_t nnz, const int64_t* row_ptr, const int32_t* col, const int32_t* w);
void level_alloc(ldl_ctx& c, int r);
void level_free(ldl_ctx& c, int r);
int32_t alive_list(ldl_ctx& c, int r, int32_t* list, int idx);
void reset_par(ldl_ctx& c, int r, int32_t nD);
// the level-0 nodes whose label differs from the batch's start -> lChg
// (count at dcnt[K_CHG], read by the caller)
void changed_labels_launch(ldl_ctx& c);
void gather_labels(ldl_ctx& c, const int32_t* ids, int32_t k, int32_t* out);
