// The library context: device-resident hierarchy, community statistics and
// the scratch of one LD-Leiden instance.
#pragma once
#include <vector>

#include "common.cuh"
#include "csr.cuh"
#include "prims.cuh"

// Adjacency view of one level: level 0 stores int32 weights, aggregate levels
// int64.  For undirected graphs the in-view aliases the out-view.
template <class WT>
struct Adj {
  const int64_t* off;
  const int32_t* len;
  const int32_t* col;
  const WT* w;
};

struct LevelState {
  SlackCSR<int32_t> out0, in0;   // level 0 (directed: in-rows at rows n..2n-1 of out0)
  SlackCSR<int64_t> out, in;     // levels >= 1 (same layout)
  SlackCSR<int32_t> children;    // keyed by level r+1 node: its level-r members (r < T)
  DBuf<int32_t> lab, par, cnt;   // P^r, pi_r (NONE = -1), number of level r-1 children
  DBuf<int64_t> kout, kin;       // strengths (kin aliases kout when undirected)
  DBuf<uint8_t> alive;
  DBuf<int32_t> stA, lA;         // frontier A^r (dedup stamp + list)
  DBuf<int32_t> stK, lK;         // endpoints of arcs deleted since the level was last refined
  int32_t brk_ep = 0;            // epoch of stK
  // weight records of this level not yet applied to its adjacency (levels >= 1
  // of a batch update: unsorted, unreduced; count in dcnt[K_PEND0 + r])
  DBuf<u64> pk, pv;
  int64_t pend_ub = 0;           // host bound on the pending count
  bool allocated = false;
  void release() {
    out0.release(); in0.release(); out.release(); in.release(); children.release();
    lab.release(); par.release(); cnt.release(); kout.release(); kin.release(); alive.release();
    stA.release(); lA.release(); stK.release(); lK.release(); pk.release(); pv.release();
    pend_ub = 0;
    allocated = false;
  }
};

// Device counters (indices into ldl_ctx::dcnt).
enum {
  K_U = 0, K_S, K_USTAR, K_MV, K_M0, K_D, K_C, K_R, K_R2, K_X, K_T, K_E, K_E2, K_CH, K_CAND, K_B,
  K_UNDEC, K_SMALL, K_MID, K_LARGE, K_REC, K_CREC, K_NREC, K_ERR, K_TMP, K_TMP2, K_CHG, K_MID2, K_TINY, K_CLU,
  K_G,
  K_HUBG,      // hubs of the current hub group
  K_A0 = 32,   // K_A0 + r: |A^r|
  K_BRK0 = 48, // K_BRK0 + r: endpoints of deleted level-r arcs
  K_PEND0 = 56, // K_PEND0 + r: pending weight records of level r
  K_COUNT = 64
};

struct ldl_ctx {
  ldl_params prm{};
  int dev = 0;           // the CUDA device the context lives on
  int64_t n = 0;
  int directed = 0;
  int32_t bin_deg[4] = {0, 0, 0, 0};  // resolved sweep degree bins
  int bits = 1;          // bits to hold a node id
  int T = 0;             // top level
  cudaStream_t s = 0;
  std::vector<LevelState> lv;

  DBuf<int64_t> Kout, Kin, e;  // community totals (Kin aliases Kout when undirected)
  int64_t m = 0;               // total weight
  int64_t E = 0;               // sum_C e_C
  i128 Psum = 0;               // sum_C K_out K_in

  DevScalars* d_sc = nullptr;
  int32_t* dcnt = nullptr;
  int32_t epoch = 0;

  // dedup stamps (one int32 per node id) and lists
  DBuf<int32_t> stS, stU, stMv, stB, stM0, stD, stC, stR, stX, stT, stE, stCh, stL;
  DBuf<int32_t> lU, lS, lUstar, lMv, lM0, lD, lC, lR, lR2, lX, lT, lE, lE2, lCh, lChg, lTmp, lG;
  DBuf<int32_t> comp;  // connected-component labels of the refinement's re-check
  DBuf<int32_t> nbr;   // per leaving node: its neighbours in its old refined community
  DBuf<int32_t> ckf;   // per refined community: stamp when its connectivity must be computed
  // candidates and accepted moves
  DBuf<int32_t> cv, csrc, cdst, cst, bv, bsrc, bdst, best, role;
  DBuf<int64_t> cghi;
  DBuf<uint64_t> cglo;
  // commit / refine scratch
  DBuf<int32_t> oldlab, par_old, lab_before;
  DBuf<int64_t> snapKo, snapKi, snapE;
  // sweep binning
  DBuf<int32_t> binT, binS, binM, binM2, binC, binL;
  DBuf<int64_t> binLoff, binLsz;
  DBuf<int32_t> gkeys;   // hub hash tables (kept clean: all -1 / 0 between sweeps)
  DBuf<int64_t> gvals;
  int64_t gtab_clean = 0;  // capacity of gkeys / gvals known to be clean
  DBuf<int32_t> glist;   // per hub: the table slots its sweep occupied
  DBuf<int32_t> hcnt;    // per hub: number of occupied slots
  // records
  DBuf<u64> rk, rv, tk, tv, rk2, rv2;
  DBuf<int64_t> rsum, rsum2;
  DBuf<int32_t> ndx;
  DBuf<int64_t> ndko, ndki;
  DBuf<u64> crk, crv, fk, trk, trv;
  DBuf<u64> flk;      // a pending list's summed records (keys) ...
  DBuf<int64_t> flv;  // ... and their weight changes
  DBuf<int64_t> chunk_pre;
  DBuf<int64_t> hub_ecnt, hub_epre, pb_hi;
  DBuf<uint64_t> pb_lo;
  DBuf<int32_t> pb_c;
  DBuf<ldl_update> upd;
  Prims P;
  CsrScratch CS;

  // counters of the last batch
  ldl_result res{};
  // per-level device pointers handed out in ldl_result (host arrays)
  const int32_t* out_par[8] = {nullptr};
  const int32_t* out_lab[8] = {nullptr};
  const uint8_t* out_alive[8] = {nullptr};
  int64_t frontier[8] = {0};
  int timing = 0;
  double stage_ms[16] = {0};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
  // per-kernel statistics of the sweep kernels (enabled by ldl_set_kernel_stats)
  int kstats = 0;
  std::vector<cudaEvent_t> kev;  // KS_EVENTS events per sweep since enabling
  size_t kev_used = 0;
  double ks_launch[KS_GROUPS] = {0, 0, 0, 0, 0, 0, 0};
  int64_t syncs = 0;  // host synchronisations in the current batch
  int64_t grow_per_update = 0;  // most device bytes a batch of this context allocated per update
  // host reads of device values: a pinned, device-mapped page (word 0 is the
  // sequence number of the last read, the payload follows)
  volatile int64_t* h_pub = nullptr;
  int64_t* d_pub = nullptr;
  int64_t pub_seq = 0;
  std::string err;
  bool broken = false;  // a failed rollback left the state unknown

  // batch transaction (atomic batches): the snapshot of the node arrays and
  // community totals, and the host scalars (each CSR keeps its undo log)
  struct SnapSeg {
    void* p;
    size_t bytes, off;
  };
  DBuf<unsigned char> snap;
  std::vector<SnapSeg> snap_segs;
  int64_t snap_m = 0, snap_E = 0;
  i128 snap_P = 0;
  bool in_txn = false;

  int32_t next_epoch() { return ++epoch; }
};

// ---------------------------------------------------------------- helpers
inline Adj<int32_t> adj_out0(ldl_ctx& c) {
  auto& g = c.lv[0].out0;
  return Adj<int32_t>{g.off.p, g.len.p, g.col.p, g.w.p};
}
// Directed graphs keep the in-rows of a level in the same slack CSR as its
// out-rows, at rows n..2n-1.
inline Adj<int32_t> adj_in0(ldl_ctx& c) {
  auto& g = c.lv[0].out0;
  const int64_t o = c.directed ? c.n : 0;
  return Adj<int32_t>{g.off.p + o, g.len.p + o, g.col.p, g.w.p};
}
inline Adj<int64_t> adj_out(ldl_ctx& c, int r) {
  auto& g = c.lv[r].out;
  return Adj<int64_t>{g.off.p, g.len.p, g.col.p, g.w.p};
}
inline Adj<int64_t> adj_in(ldl_ctx& c, int r) {
  auto& g = c.lv[r].out;
  const int64_t o = c.directed ? c.n : 0;
  return Adj<int64_t>{g.off.p + o, g.len.p + o, g.col.p, g.w.p};
}
inline int64_t* kin_of(ldl_ctx& c, int r) { return c.directed ? c.lv[r].kin.p : c.lv[r].kout.p; }
inline int64_t* Kin_of(ldl_ctx& c) { return c.directed ? c.Kin.p : c.Kout.p; }

// host reads of device counters (synchronise)
// Copies device values to the host once the context's stream has reached
// this point: a one-block kernel writes them into the pinned page and then the
// sequence number, which the host polls (a stream error ends the wait).
void host_read(ldl_ctx& c, const HostRead* r, int n);
int32_t rd_cnt(ldl_ctx& c, int idx);
void zero_cnt(ldl_ctx& c, int idx);
// One launch that clears several counters (bit i of mask: dcnt[i]) and up to
// ZERO_SPANS spans of 64-bit device words (p[i], nw[i] <= K_COUNT words).
constexpr int ZERO_SPANS = 3;
struct ZeroSpans {
  uint64_t mask = 0;
  int64_t* p[ZERO_SPANS] = {nullptr, nullptr, nullptr};
  int32_t nw[ZERO_SPANS] = {0, 0, 0};
};
inline uint64_t cnt_bit(int idx) { return 1ull << idx; }
void zero_many(ldl_ctx& c, const ZeroSpans& z);
void set_cnt(ldl_ctx& c, int idx, int32_t v);

// stage timing
void stage_begin(ldl_ctx& c);
void stage_end(ldl_ctx& c, int stage);
enum { ST_INGEST = 0, ST_REPAIR, ST_EXPAND, ST_BEST, ST_DECOUPLE, ST_COMMIT, ST_REFINE, ST_AGG, ST_PUSH,
       SU_AGG_EMIT, SU_AGG_SORT, SU_AGG_APPLY, SU_AGG_UP, SU_AGG_EXIST, SU_REF_DISSOLVE, SU_REF_LOOP };
// nested sub-stage timers (their own events)
void sub_begin(ldl_ctx& c);
void sub_end(ldl_ctx& c, int stage);
