// C ABI and host control of the LD-Leiden batch update (Algorithm 1).
//
// The host only sequences kernels and reads back the few integers that
// decide control flow (list sizes, dQ(B), the pass gain); every step of the
// method runs in the kernels of sweep.cu, hier.cu, csr.cu and prims.cu.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "kern.cuh"

// ---------------------------------------------------------------- errors / memory
void ldl_throw(ldl_status st, const std::string& msg) { throw LdlError{st, msg}; }

void ldl_cuda_check(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return;
  char buf[512];
  snprintf(buf, sizeof buf, "%s: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  if (e == cudaErrorMemoryAllocation) ldl_throw(LDL_E_NOMEM, buf);
  ldl_throw(LDL_E_CUDA, buf);
}

static std::atomic<int64_t> g_fail_after{0};
std::atomic<int64_t> g_launches{0};
static std::atomic<int64_t> g_allocs{0}, g_txn_allocs{0};
static thread_local bool t_in_txn = false;  // this thread is inside a batch transaction
static thread_local bool t_count_batch = false;  // this thread is applying a batch
static thread_local int64_t t_batch_bytes = 0;   // device bytes it asked for meanwhile

void* dalloc(size_t bytes) {
  g_allocs.fetch_add(1, std::memory_order_relaxed);
  if (t_in_txn) g_txn_allocs.fetch_add(1, std::memory_order_relaxed);
  if (t_count_batch) t_batch_bytes += ((int64_t)bytes + (2 << 20) - 1) & ~(int64_t)((2 << 20) - 1);  // device pages
  int64_t k = g_fail_after.load();
  if (k > 0) {
    if (g_fail_after.fetch_sub(1) == 1) ldl_throw(LDL_E_NOMEM, "injected allocation failure");
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes ? bytes : 1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char buf[128];
    snprintf(buf, sizeof buf, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    ldl_throw(e == cudaErrorMemoryAllocation ? LDL_E_NOMEM : LDL_E_CUDA, buf);
  }
  return p;
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

namespace {
constexpr int kMaxDev = 64;
std::atomic<int> g_sms[kMaxDev];  // 0: not queried yet
}  // namespace

int device_sms() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) ldl_throw(LDL_E_CUDA, "device ordinal out of range");
  int v = g_sms[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  CK(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
  if (v <= 0) ldl_throw(LDL_E_CUDA, "device reports no multiprocessors");
  g_sms[dev].store(v, std::memory_order_relaxed);
  return v;
}

DeviceScope::DeviceScope(int d) : dev(d) {
  CK(cudaGetDevice(&prev));
  if (prev != dev) CK(cudaSetDevice(dev));
}

DeviceScope::~DeviceScope() {
  if (prev >= 0 && prev != dev) cudaSetDevice(prev);
}

namespace {
constexpr int PUB_MAX = 8;        // values per read
constexpr int PUB_BYTES = 4000;   // payload bytes per read
struct PubReq {
  const unsigned char* src[PUB_MAX];
  int32_t off[PUB_MAX], bytes[PUB_MAX];
  int32_t n;
};

__global__ void k_publish(PubReq q, unsigned char* payload, int64_t* seq_word, int64_t seq) {
  for (int i = 0; i < q.n; ++i)
    for (int b = threadIdx.x; b < q.bytes[i]; b += blockDim.x) payload[q.off[i] + b] = q.src[i][b];
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence_system();  // the payload is visible to the host before the sequence number
    *(volatile int64_t*)seq_word = seq;
  }
}

__global__ void k_set_i32(int32_t* p, int32_t v) { *p = v; }

// clears the counters named by the mask and up to ZERO_SPANS spans of 64-bit words
__global__ void k_zero(int32_t* dcnt, ZeroSpans z) {
  const int t = threadIdx.x;
  if (t < K_COUNT && ((z.mask >> t) & 1ull)) dcnt[t] = 0;
  for (int i = 0; i < ZERO_SPANS; ++i)
    if (z.p[i] && t < z.nw[i]) z.p[i][t] = 0;
}
}  // namespace

void host_read(ldl_ctx& c, const HostRead* r, int n) {
  ++c.syncs;
  PubReq q{};
  int32_t off = 0;
  if (n > PUB_MAX) ldl_throw(LDL_E_INVALID, "internal: host read of too many values");
  for (int i = 0; i < n; ++i) {
    q.src[i] = (const unsigned char*)r[i].src;
    q.off[i] = off;
    q.bytes[i] = r[i].bytes;
    off += (r[i].bytes + 7) & ~7;
  }
  if (off > PUB_BYTES) ldl_throw(LDL_E_INVALID, "internal: host read too large");
  q.n = n;
  const int64_t seq = ++c.pub_seq;
  k_publish<<<1, 64, 0, c.s>>>(q, (unsigned char*)(c.d_pub + 1), c.d_pub, seq);
  CKL("k_publish");
  // Poll the mapped sequence word.  Every so often ask the stream: an error
  // ends the wait with that error; an idle stream whose write is still not
  // seen falls back to a full synchronisation before failing.
  for (uint64_t spins = 1; c.h_pub[0] != seq; ++spins) {
    if ((spins & 4095) == 0) {
      const cudaError_t e = cudaStreamQuery(c.s);
      if (e == cudaErrorNotReady) continue;
      CK(e);
      CK(cudaStreamSynchronize(c.s));
      if (c.h_pub[0] != seq) ldl_throw(LDL_E_CUDA, "internal: a published value never reached the host");
    }
  }
  std::atomic_thread_fence(std::memory_order_acquire);
  const unsigned char* pay = (const unsigned char*)(c.h_pub + 1);
  for (int i = 0; i < n; ++i) memcpy(r[i].dst, pay + q.off[i], (size_t)r[i].bytes);
}

int32_t rd_cnt(ldl_ctx& c, int idx) {
  int32_t v = 0;
  const HostRead r{c.dcnt + idx, &v, sizeof(int32_t)};
  host_read(c, &r, 1);
  return v;
}

void zero_cnt(ldl_ctx& c, int idx) { CK(cudaMemsetAsync(c.dcnt + idx, 0, sizeof(int32_t), c.s)); }

void zero_many(ldl_ctx& c, const ZeroSpans& z) {
  for (int i = 0; i < ZERO_SPANS; ++i)
    if (z.nw[i] < 0 || z.nw[i] > K_COUNT) ldl_throw(LDL_E_INVALID, "internal: zero span too long");
  k_zero<<<1, K_COUNT, 0, c.s>>>(c.dcnt, z);
  CKL("k_zero");
}

void set_cnt(ldl_ctx& c, int idx, int32_t v) {
  k_set_i32<<<1, 1, 0, c.s>>>(c.dcnt + idx, v);
  CKL("k_set_i32");
}

void stage_begin(ldl_ctx& c) {
  if (c.timing) CK(cudaEventRecord(c.ev0, c.s));
}

void stage_end(ldl_ctx& c, int stage) {
  if (!c.timing) return;
  CK(cudaEventRecord(c.ev1, c.s));
  CK(cudaEventSynchronize(c.ev1));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, c.ev0, c.ev1));
  c.stage_ms[stage] += ms;
}

void sub_begin(ldl_ctx& c) {
  if (c.timing) CK(cudaEventRecord(c.ev2, c.s));
}

void sub_end(ldl_ctx& c, int stage) {
  if (!c.timing) return;
  CK(cudaEventRecord(c.ev3, c.s));
  CK(cudaEventSynchronize(c.ev3));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, c.ev2, c.ev3));
  c.stage_ms[stage] += ms;
}

static thread_local std::string g_create_err = "no error";

// ---------------------------------------------------------------- numerator
static i128 qnum(const ldl_ctx& c) {
  return (i128)c.prm.gamma_den * c.m * c.E - (i128)c.prm.gamma_num * c.Psum;
}

// ---------------------------------------------------------------- allocation
void alloc_globals(ldl_ctx& c) {
  const int64_t n = c.n;
  c.Kout.exact(n);
  if (c.directed) c.Kin.exact(n);
  c.e.exact(n);
  DBuf<int32_t>* st[] = {&c.stS, &c.stU, &c.stMv, &c.stB, &c.stM0, &c.stD, &c.stC, &c.stR, &c.stX, &c.stT, &c.stE,
                         &c.stCh, &c.stL, &c.ckf};
  for (auto* b : st) {
    b->exact(n);
    CK(cudaMemsetAsync(b->p, 0, sizeof(int32_t) * (size_t)n, c.s));
  }
  DBuf<int32_t>* ls[] = {&c.lU, &c.lS, &c.lUstar, &c.lMv, &c.lM0, &c.lD, &c.lC, &c.lR, &c.lR2, &c.lX, &c.lT,
                         &c.lE, &c.lE2, &c.lCh, &c.lChg, &c.lTmp, &c.lG, &c.comp, &c.nbr, &c.cv, &c.csrc, &c.cdst, &c.cst, &c.bv,
                         &c.bsrc, &c.bdst, &c.oldlab, &c.par_old, &c.lab_before, &c.binT, &c.binS, &c.binM, &c.binM2, &c.binC, &c.binL};
  for (auto* b : ls) b->exact(n);
  c.best.exact(n);
  CK(cudaMemsetAsync(c.best.p, 0xff, sizeof(int32_t) * (size_t)n, c.s));
  c.role.exact(n);
  CK(cudaMemsetAsync(c.role.p, 0, sizeof(int32_t) * (size_t)n, c.s));
  c.cghi.exact(n);
  c.cglo.exact(n);
  c.snapKo.exact(2 * n);
  c.snapKi.exact(2 * n);
  c.snapE.exact(2 * n);
  c.binLoff.exact(n + 1);
  c.binLsz.exact(n + 1);
  c.d_sc = (DevScalars*)dalloc(sizeof(DevScalars));
  CK(cudaMemsetAsync(c.d_sc, 0, sizeof(DevScalars), c.s));
  c.dcnt = (int32_t*)dalloc(sizeof(int32_t) * K_COUNT);
  CK(cudaMemsetAsync(c.dcnt, 0, sizeof(int32_t) * K_COUNT, c.s));
  c.P.rd = [](void* owner, const HostRead* r, int n) { host_read(*(ldl_ctx*)owner, r, n); };
  c.P.rd_owner = &c;
}

void free_all(ldl_ctx& c) {
  if (c.s) cudaStreamSynchronize(c.s);
  for (auto& L : c.lv) L.release();
  DBuf<int64_t>* b64[] = {&c.Kout, &c.Kin, &c.e, &c.cghi, &c.snapKo, &c.snapKi, &c.snapE, &c.binLoff, &c.binLsz,
                          &c.gvals, &c.rsum, &c.rsum2, &c.ndko, &c.ndki,
                          &c.chunk_pre, &c.hub_ecnt, &c.hub_epre, &c.pb_hi};
  for (auto* b : b64) b->release();
  DBuf<int32_t>* b32[] = {&c.stS, &c.stU, &c.stMv, &c.stB, &c.stM0, &c.stD, &c.stC, &c.stR, &c.stX, &c.stT,
                          &c.stE, &c.stCh, &c.stL, &c.lG, &c.comp, &c.nbr, &c.ckf, &c.lU, &c.lS, &c.lUstar, &c.lMv, &c.lM0, &c.lD, &c.lC, &c.lR,
                          &c.lR2, &c.lX, &c.lT, &c.lE, &c.lE2, &c.lCh, &c.lChg, &c.lTmp, &c.cv, &c.csrc,
                          &c.cdst, &c.cst, &c.bv, &c.bsrc, &c.bdst, &c.best, &c.role, &c.oldlab, &c.par_old,
                          &c.lab_before, &c.binT, &c.binS, &c.binM, &c.binM2, &c.binC, &c.binL, &c.gkeys, &c.ndx,
                          &c.glist, &c.hcnt};
  for (auto* b : b32) b->release();
  DBuf<u64>* bu[] = {&c.rk, &c.rv, &c.tk, &c.tv, &c.rk2, &c.rv2, &c.crk, &c.crv, &c.fk, &c.trk, &c.trv, &c.flk};
  for (auto* b : bu) b->release();
  c.flv.release();
  c.cglo.release();
  c.pb_lo.release();
  c.pb_c.release();
  c.gtab_clean = 0;
  c.upd.release();
  c.snap.release();
  c.P.release();
  c.CS.release();
  if (c.d_sc) dfree(c.d_sc);
  if (c.dcnt) dfree(c.dcnt);
  c.d_sc = nullptr;
  c.dcnt = nullptr;
  if (c.h_pub) cudaFreeHost((void*)c.h_pub);
  c.h_pub = nullptr;
  c.d_pub = nullptr;
  if (c.ev0) cudaEventDestroy(c.ev0);
  if (c.ev1) cudaEventDestroy(c.ev1);
  if (c.ev2) cudaEventDestroy(c.ev2);
  if (c.ev3) cudaEventDestroy(c.ev3);
  c.ev0 = c.ev1 = c.ev2 = c.ev3 = nullptr;
  for (auto& ev : c.kev) cudaEventDestroy(ev);
  c.kev.clear();
  c.kev_used = 0;
}

// ---------------------------------------------------------------- move loop
// The local-move loop of Algorithm 1 at level r.  Precondition: lU holds U = A^r, and
// lUstar / stU (epoch epU) hold U*.  Moved nodes go to lMv (epMv) and, at
// level 0, to lM0 (epM0).
static int64_t move_loop(ldl_ctx& c, int r, int rounds, int32_t epU, int32_t epMv, int32_t epM0, int32_t epCh,
                         int32_t nU) {
  // nU = |U| on entry; later rounds take it from the end of the previous one.
  // Returns the committed moves, an upper bound of the distinct moved nodes
  // (lMv), which is empty exactly when it is 0.
  int64_t committed = 0;
  const i128 Q0 = qnum(c);
  const int64_t ainv = c.prm.alpha_inv, binv = c.prm.beta_inv;
  for (int j = 0; j < rounds; ++j) {
    if (nU == 0) break;
    c.res.rounds++;
    stage_begin(c);
    const int32_t epS = c.next_epoch();
    zero_cnt(c, K_S);
    expand_set(c, r, c.lU.p, K_U, c.stS.p, epS, c.lS.p, K_S, nU);
    stage_end(c, ST_EXPAND);
    // |S| stays on the device: the sweep's kernels stride over it (n bounds
    // their grids) and it comes back with the sweep's bin counts (β test)
    stage_begin(c);
    const int32_t nS = sweep(c, r, 0, c.lS.p, K_S, c.n);
    stage_end(c, ST_BEST);
    stage_begin(c);
    const DecoupleOut dd = decouple(c);
    stage_end(c, ST_DECOUPLE);
    const int32_t nc = dd.nc, nb = dd.nb;
    if (nc == 0) break;
    c.res.rejected += nc - nb;
    if (nb == 0) break;
    stage_begin(c);
    const int32_t epB = c.next_epoch(), epT = c.next_epoch();
    commit_move(c, r, nb, epB, epT, epCh);
    // the next frontier U = V ∪ N(V) is expanded before the commit's outcome
    // comes back (it only marks neighbours), so one read returns both; a
    // rolled-back mini-batch ends the loop and its expansion is dropped
    const int32_t epS2 = c.next_epoch();
    zero_cnt(c, K_U);
    expand_set(c, r, c.bv.p, K_B, c.stS.p, epS2, c.lU.p, K_U, nb);
    int32_t nU2 = 0;
    const CommitOut co = commit_read(c, K_U, &nU2);
    if (co.dq < 0) {
      rollback_move(c, r, nb, co.ntc);
      c.res.rollbacks++;
      stage_end(c, ST_COMMIT);
      break;
    }
    c.E += co.de;
    c.Psum += co.dp;
    c.res.moves += nb;
    committed += nb;
    mark_moved(c, r, nb, epMv, epM0);
    stage_end(c, ST_COMMIT);
    stage_begin(c);
    union_into(c, c.lU.p, K_U, c.stU.p, epU, c.lUstar.p, K_USTAR, nU2);
    stage_end(c, ST_EXPAND);
    nU = nU2;
    if (co.dq * (i128)ainv < Q0) break;
    if ((int64_t)nb * binv < (int64_t)nS) break;
  }
  return committed;
}

// The refinement loop of Algorithm 1 at level r over the dissolved set lD (epoch epD).
static int64_t refine_loop(ldl_ctx& c, int r, int rounds, int32_t epD, int32_t nD) {
  if (nD == 0) return 0;
  // R starts as the singleton refined communities of D
  singletons_of(c, r, c.lD.p, K_D, nD, c.lR.p, K_R);
  int32_t* R = c.lR.p;
  int32_t* R2 = c.lR2.p;
  int iR = K_R, iR2 = K_R2;
  int64_t merges = 0;
  const int64_t binv = c.prm.beta_inv;
  for (int j = 0; j < rounds; ++j) {
    // R is a subset of D, so nD bounds the sweep's launch; |R| comes back with
    // the sweep's bin counts (an empty R ends the loop before any filter)
    c.res.rounds++;
    const int32_t nR = sweep(c, r, 1, R, iR, nD);
    if (nR == 0) {
      c.res.rounds--;
      break;
    }
    const DecoupleOut dd = decouple(c);
    const int32_t nc = dd.nc, nb = dd.nb;
    if (nc == 0) break;
    c.res.rejected += nc - nb;
    if (nb == 0) break;
    commit_ref(c, r, nb);
    merges += nb;
    c.res.refine_moves += nb;
    if ((int64_t)nb * binv < (int64_t)nR) break;
    const int32_t epR = c.next_epoch();
    zero_cnt(c, iR2);
    spexpand(c, r, nb, epD, epR, R2, iR2);
    std::swap(R, R2);
    std::swap(iR, iR2);
  }
  return merges;
}

static void check_scan_wait(ldl_ctx& c);

// ---------------------------------------------------------------- static build
static void static_build(ldl_ctx& c) {
  const int L = c.prm.L;
  c.T = 0;
  zero_cnt(c, K_ERR);
  for (int r = 0; r <= L; ++r) {
    const int32_t nU = alive_list(c, r, c.lU.p, K_U);
    const int32_t epU = c.next_epoch();
    zero_cnt(c, K_USTAR);
    union_into(c, c.lU.p, K_U, c.stU.p, epU, c.lUstar.p, K_USTAR, nU);
    const int32_t epMv = c.next_epoch(), epM0 = c.next_epoch(), epCh = c.next_epoch();
    zero_cnt(c, K_MV);
    zero_cnt(c, K_M0);
    zero_cnt(c, K_CH);
    const int64_t mv = move_loop(c, r, c.prm.M_static, epU, epMv, epM0, epCh, nU);
    if (r > 0) pushdown(c, r, epCh, mv);
    if (r == L) break;
    level_alloc(c, r + 1);
    c.T = r + 1;
    const int32_t epD = c.next_epoch();
    const int32_t nD = dissolve_all(c, r, epD);
    const int64_t merges = refine_loop(c, r, c.prm.M_static, epD, nD);
    if (merges == 0) {
      reset_par(c, r, nD);
      level_free(c, r + 1);
      c.T = r;
      break;
    }
    const int32_t epC = c.next_epoch();
    aggregate(c, r, epD, epC, 0, true, nD);
  }
  if (rd_cnt(c, K_ERR)) ldl_throw(LDL_E_INVALID, "internal: a new supernode already had a parent, or records exceeded their bound");
  check_scan_wait(c);
}

// The static build's record and table buffers are sized by the whole graph
// (every node is in the first frontier); batches need a small fraction, so
// they are freed here and grow again to what batches use.
static void release_build_scratch(ldl_ctx& c) {
  CK(cudaStreamSynchronize(c.s));
  DBuf<u64>* bu[] = {&c.rk, &c.rv, &c.tk, &c.tv, &c.rk2, &c.rv2, &c.crk, &c.crv, &c.fk, &c.trk, &c.trv};
  for (auto* b : bu) b->release();
  c.rsum.release();
  c.rsum2.release();
  c.gkeys.release();
  c.gvals.release();
  c.glist.release();
  c.gtab_clean = 0;
  c.pb_hi.release();
  c.pb_lo.release();
  c.pb_c.release();
  c.CS.release();
  c.P.hist.release();
  c.P.pos.release();
  c.P.usum.release();
  c.P.flag.release();
}

// ---------------------------------------------------------------- transactions
// Every CSR of the hierarchy (adjacency of each level, children lists of each
// level below the top), visited in a fixed order.
template <class F>
static void for_each_csr(ldl_ctx& c, F&& f) {
  f(c.lv[0].out0);
  for (int r = 1; r <= c.T; ++r) f(c.lv[r].out);
  for (int r = 0; r < c.T; ++r) f(c.lv[r].children);
}

// Start of an atomic batch, after validation and before the first change:
// the node arrays of every level and the community totals are copied into a
// buffer the context keeps (the only allocation here), and every CSR starts
// its undo log.
static void txn_begin(ldl_ctx& c) {
  const size_t n = (size_t)c.n;
  c.snap_segs.clear();
  size_t tot = 0;
  auto add = [&](void* p, size_t bytes) {
    if (!p || !bytes) return;
    c.snap_segs.push_back({p, bytes, tot});
    tot += (bytes + 255) & ~(size_t)255;
  };
  for (int r = 0; r <= c.T; ++r) {
    LevelState& L = c.lv[r];
    add(L.lab.p, 4 * n);
    add(L.par.p, 4 * n);
    add(L.cnt.p, 4 * n);
    add(L.kout.p, 8 * n);
    if (c.directed) add(L.kin.p, 8 * n);
    add(L.alive.p, n);
  }
  add(c.Kout.p, 8 * n);
  if (c.directed) add(c.Kin.p, 8 * n);
  add(c.e.p, 8 * n);
  c.snap.reserve((int64_t)tot, c.s);
  for (auto& sg : c.snap_segs)
    CK(cudaMemcpyAsync(c.snap.p + sg.off, sg.p, sg.bytes, cudaMemcpyDeviceToDevice, c.s));
  for_each_csr(c, [&](auto& g) { csr_txn_begin(g); });
  c.snap_m = c.m;
  c.snap_E = c.E;
  c.snap_P = c.Psum;
  c.in_txn = true;
  t_in_txn = true;
}

// The batch succeeded: pools replaced by compaction during it are freed.
static void txn_commit(ldl_ctx& c) {
  if (!c.in_txn) return;
  t_in_txn = false;
  for_each_csr(c, [&](auto& g) { csr_txn_commit(g, c.s); });
  c.in_txn = false;
}

// The batch failed after it began changing the state: put everything back
// (copies and frees only, no allocation).
static void txn_rollback(ldl_ctx& c) {
  if (!c.in_txn) return;
  c.in_txn = false;
  t_in_txn = false;
  cudaGetLastError();
  cudaError_t e = cudaStreamSynchronize(c.s);
  for (auto& sg : c.snap_segs)
    if (e == cudaSuccess) e = cudaMemcpyAsync(sg.p, c.snap.p + sg.off, sg.bytes, cudaMemcpyDeviceToDevice, c.s);
  for_each_csr(c, [&](auto& g) {
    const cudaError_t e2 = csr_txn_rollback(g, c.s);
    if (e == cudaSuccess) e = e2;
  });
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.s);
  c.m = c.snap_m;
  c.E = c.snap_E;
  c.Psum = c.snap_P;
  c.gtab_clean = 0;  // hub hash tables may hold a half-finished sweep
  if (e != cudaSuccess) {
    c.broken = true;
    ldl_throw(LDL_E_CUDA, std::string("rollback after a failed batch: ") + cudaGetErrorString(e));
  }
}

// ---------------------------------------------------------------- batch update
static void apply_batch(ldl_ctx& c, const ldl_update* upd, int64_t count, int on_device) {
  memset(&c.res, 0, sizeof(c.res));
  c.syncs = 0;
  pending_reset(c);
  CK(cudaMemsetAsync(&c.d_sc->scanned, 0, sizeof(int64_t), c.s));
  const int T = c.T;
  int64_t dm = 0;
  stage_begin(c);
  const int64_t na = ingest(c, upd, count, on_device, &dm);
  stage_end(c, ST_INGEST);
  const int32_t epCh = c.next_epoch();
  zero_cnt(c, K_CH);
  zero_cnt(c, K_ERR);
  if (na == 0) {
    c.res.n_changed = 0;
    return;
  }
  if (!c.prm.no_rollback) txn_begin(c);
  std::vector<int32_t> epA(T + 2, 0);
  for (int r = 0; r <= T; ++r) {
    epA[r] = c.next_epoch();
    zero_cnt(c, K_A0 + r);
    c.lv[r].brk_ep = c.next_epoch();
    zero_cnt(c, K_BRK0 + r);
  }
  stage_begin(c);
  const int32_t epT = c.next_epoch();
  repair_batch(c, na, epA.data(), epT, dm);
  stage_end(c, ST_REPAIR);
  const int64_t ainv = c.prm.alpha_inv;
  for (int pass = 0; pass < c.prm.N; ++pass) {
    const i128 Qpass = qnum(c);
    const int32_t epM0 = c.next_epoch();
    zero_cnt(c, K_M0);
    int32_t nM0 = -1;  // |level-0 moves of the pass|, final once level 0 is done
    for (int r = 0; r <= T; ++r) {
      // |A^r| stays on the device: the filter strides over it with a grid of
      // two blocks per SM, and one read returns |U|, the level's pending
      // record count for its flush and, from level 1 on, |M0|
      zero_cnt(c, K_U);
      filter_alive(c, r, c.lv[r].lA.p, K_A0 + r, c.lU.p, K_U, std::min<int64_t>(c.n, (int64_t)device_sms() * 512));
      int32_t nU = 0, nP = 0, m0 = 0;
      {
        const HostRead rr[3] = {{c.dcnt + K_U, &nU, sizeof(int32_t)},
                                {c.dcnt + K_PEND0 + r, &nP, sizeof(int32_t)},
                                {c.dcnt + K_M0, &m0, sizeof(int32_t)}};
        host_read(c, rr, r > 0 ? 3 : 2);
        if (r > 0) nM0 = m0;
      }
      if (nU == 0) continue;
      if (r < 8) c.res.frontier_nodes[r] += nU;
      const int32_t epU = c.next_epoch();
      zero_cnt(c, K_USTAR);
      union_into(c, c.lU.p, K_U, c.stU.p, epU, c.lUstar.p, K_USTAR, nU);
      const int32_t epMv = c.next_epoch();
      zero_cnt(c, K_MV);
      stage_begin(c);
      flush_level(c, r, nP);  // the level's weights are read from here on
      stage_end(c, ST_AGG);
      const int64_t mv = move_loop(c, r, c.prm.M, epU, epMv, epM0, epCh, nU);
      if (r > 0) {
        stage_begin(c);
        pushdown(c, r, epCh, mv);
        stage_end(c, ST_PUSH);
      }
      if (r < T) {
        stage_begin(c);
        const int32_t epD = c.next_epoch(), epX = c.next_epoch();
        sub_begin(c);
        const int32_t nD = split(c, r, epD, epX);
        sub_end(c, SU_REF_DISSOLVE);
        sub_begin(c);
        refine_loop(c, r, c.prm.M, epD, nD);
        sub_end(c, SU_REF_LOOP);
        stage_end(c, ST_REFINE);
        stage_begin(c);
        const int32_t epC = c.next_epoch();
        aggregate(c, r, epD, epC, epA[r + 1], false, nD);
        stage_end(c, ST_AGG);
      }
    }
    // frontiers of the next pass: A^0 = Expand_0(level-0 moves), others empty
    if (nM0 < 0) nM0 = rd_cnt(c, K_M0);
    for (int r = 0; r <= T; ++r) {
      epA[r] = c.next_epoch();
      zero_cnt(c, K_A0 + r);
    }
    // the expansion holds the moved nodes themselves, so A^0 is empty
    // exactly when no level-0 node moved
    if (nM0 == 0) break;
    expand_set(c, 0, c.lM0.p, K_M0, c.lv[0].stA.p, epA[0], c.lv[0].lA.p, K_A0, nM0);
    if ((qnum(c) - Qpass) * (i128)ainv < Qpass) break;
  }
  stage_begin(c);
  {
    // the pending counts of every level above 0 in one read (K_PEND0 + r are
    // adjacent; a flush changes no other level's list)
    int32_t np[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (T >= 1) {
      const HostRead rr{c.dcnt + K_PEND0 + 1, np, (int32_t)(sizeof(int32_t) * (size_t)std::min(T, 7))};
      host_read(c, &rr, 1);
    }
    for (int r = 1; r <= T; ++r) flush_level(c, r, np[r - 1]);
  }
  stage_end(c, ST_AGG);
  changed_labels_launch(c);
  // one read: changed labels, the internal error flag, entries scanned and
  // the look-back scans' error flag
  int32_t nchg = 0, err = 0, scan_bad = 0;
  int32_t* scan_flag = scan_error_flag(c.P);
  {
    const HostRead rr[4] = {{c.dcnt + K_CHG, &nchg, sizeof(int32_t)},
                            {c.dcnt + K_ERR, &err, sizeof(int32_t)},
                            {&c.d_sc->scanned, &c.res.edges_scanned, sizeof(int64_t)},
                            {scan_flag, &scan_bad, sizeof(int32_t)}};
    host_read(c, rr, scan_flag ? 4 : 3);
  }
  c.res.n_changed = nchg;
  c.res.host_syncs = c.syncs;
  CK(cudaStreamSynchronize(c.s));
  if (err) ldl_throw(LDL_E_INVALID, "internal: a new supernode already had a parent, or records exceeded their bound");
  if (scan_bad) {
    CK(cudaMemsetAsync(scan_flag, 0, sizeof(int32_t), c.s));
    ldl_throw(LDL_E_TIMEOUT, "a device scan's bounded wait gave up");
  }
}

// Reads the look-back scans' error flag (and synchronises): a bounded wait
// that gave up leaves results that cannot be trusted.
static void check_scan_wait(ldl_ctx& c) {
  int32_t* f = scan_error_flag(c.P);
  int32_t bad = 0;
  if (f) CK(cudaMemcpyAsync(&bad, f, sizeof(int32_t), cudaMemcpyDeviceToHost, c.s));
  CK(cudaStreamSynchronize(c.s));
  if (bad) {
    CK(cudaMemsetAsync(f, 0, sizeof(int32_t), c.s));
    ldl_throw(LDL_E_TIMEOUT, "a device scan's bounded wait gave up");
  }
}

template <class WT>
static void copy_adj(ldl_ctx& c, const SlackCSR<WT>& g, std::vector<int64_t>& off, std::vector<int32_t>& len,
                     std::vector<int32_t>& col, std::vector<WT>& w) {
  const size_t n = (size_t)c.n;
  off.resize(n);
  len.resize(n);
  col.resize((size_t)g.pool_top);
  w.resize((size_t)g.pool_top);
  CK(cudaMemcpyAsync(off.data(), g.off.p, 8 * n, cudaMemcpyDeviceToHost, c.s));
  CK(cudaMemcpyAsync(len.data(), g.len.p, 4 * n, cudaMemcpyDeviceToHost, c.s));
  if (g.pool_top) {
    CK(cudaMemcpyAsync(col.data(), g.col.p, 4 * (size_t)g.pool_top, cudaMemcpyDeviceToHost, c.s));
    CK(cudaMemcpyAsync(w.data(), g.w.p, sizeof(WT) * (size_t)g.pool_top, cudaMemcpyDeviceToHost, c.s));
  }
  CK(cudaStreamSynchronize(c.s));
}

// A context with its parameters checked, its pinned read-back page, events
// and global arrays allocated, and no levels yet (the caller builds or loads
// them).  On failure nothing is left behind and g_create_err says why.
ldl_status ctx_new(const ldl_params& p, int64_t n, ldl_ctx** out) {
  if (n <= 0 || n > INT32_MAX - 1 || p.L < 0 || p.L > 7 || p.N < 0 || p.M < 0 || p.M_static < 0 ||
      p.alpha_inv <= 0 || p.beta_inv <= 0 || p.gamma_num < 1 || p.gamma_den < 1 || p.gamma_num > 1024 ||
      p.gamma_den > 1024 || p.cluster_max_deg < 0) {
    g_create_err = "invalid size or parameter";
    return LDL_E_INVALID;
  }
  int32_t bins[4];
  for (int i = 0; i < 4; ++i) {
    bins[i] = p.bin_deg[i] ? p.bin_deg[i] : BIN_DEFAULT[i];
    if (bins[i] < 0 || bins[i] > BIN_MAX[i] || (i > 0 && bins[i] < bins[i - 1])) {
      g_create_err = "invalid sweep degree bins";
      return LDL_E_INVALID;
    }
  }
  ldl_ctx* c = new (std::nothrow) ldl_ctx();
  if (!c) return LDL_E_NOMEM;
  try {
    CK(cudaGetDevice(&c->dev));
    c->prm = p;
    c->n = n;
    c->directed = p.directed ? 1 : 0;
    c->bits = std::max(1, bits_for(n));
    c->s = (cudaStream_t)p.cuda_stream;
    {
      void* hp = nullptr;
      CK(cudaHostAlloc(&hp, 4096, cudaHostAllocMapped));
      c->h_pub = (volatile int64_t*)hp;
      c->h_pub[0] = 0;
      void* dp = nullptr;
      CK(cudaHostGetDevicePointer(&dp, hp, 0));
      c->d_pub = (int64_t*)dp;
    }
    CK(cudaEventCreate(&c->ev0));
    CK(cudaEventCreate(&c->ev1));
    CK(cudaEventCreate(&c->ev2));
    CK(cudaEventCreate(&c->ev3));
    c->lv.resize(p.L + 1);
    c->kstats = p.kernel_stats ? 1 : 0;
    for (int i = 0; i < 4; ++i) c->bin_deg[i] = bins[i];
    alloc_globals(*c);
  } catch (const LdlError& e) {
    g_create_err = e.msg;
    free_all(*c);
    delete c;
    cudaGetLastError();
    return e.st;
  }
  *out = c;
  return LDL_OK;
}

void set_create_error(const std::string& msg) { g_create_err = msg; }

// ================================================================== C ABI
extern "C" {

void ldl_default_params(ldl_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->directed = 0;
  p->gamma_num = 1;
  p->gamma_den = 1;
  p->N = 2;
  p->L = 4;
  p->M = 5;
  p->M_static = 20;
  p->alpha_inv = 1000;
  p->beta_inv = 100;
  p->cuda_stream = nullptr;
}

ldl_status ldl_create(const ldl_params* params, int64_t n, int64_t nnz, const int64_t* row_ptr,
                      const int32_t* col, const int32_t* w, ldl_ctx** out) {
  if (!out || !params || !row_ptr || (nnz > 0 && (!col || !w))) {
    g_create_err = "null argument";
    return LDL_E_INVALID;
  }
  *out = nullptr;
  if (nnz < 0 || n <= 0 || n > INT32_MAX - 1 || row_ptr[0] != 0 || row_ptr[n] != nnz) {
    g_create_err = "row_ptr must start at 0 and end at nnz (n in [1, 2^31-2], nnz >= 0)";
    return LDL_E_INVALID;
  }
  ldl_ctx* c = nullptr;
  const ldl_status st = ctx_new(*params, n, &c);
  if (st != LDL_OK) return st;
  try {
    level_alloc(*c, 0);
    upload_graph(*c, nnz, row_ptr, col, w);
    static_build(*c);
    release_build_scratch(*c);
  } catch (const LdlError& e) {
    g_create_err = e.msg;
    free_all(*c);
    delete c;
    cudaGetLastError();
    return e.st;
  }
  *out = c;
  return LDL_OK;
}

ldl_status ldl_apply_batch(ldl_ctx* c, const ldl_update* updates, int64_t count, int32_t on_device,
                           ldl_result* out) {
  if (!c) return LDL_E_INVALID;
  if (count < 0 || (count > 0 && !updates)) {
    c->err = "bad batch arguments";
    return LDL_E_INVALID;
  }
  if (c->broken) {
    c->err = "the context's state was lost by an earlier failed rollback; destroy it";
    return LDL_E_CUDA;
  }
  // the device bytes a batch asks for (including a request that fails) per
  // update, kept as the context's worst case for ldl_batch_estimate_bytes
  auto learn = [&]() {
    t_count_batch = false;
    if (count > 0) c->grow_per_update = std::max(c->grow_per_update, (t_batch_bytes + count - 1) / count);
  };
  try {
    DeviceScope ds(c->dev);
    t_batch_bytes = 0;
    t_count_batch = true;
    try {
      apply_batch(*c, updates, count, on_device);
      CK(cudaStreamSynchronize(c->s));
      txn_commit(*c);
      learn();
    } catch (const LdlError& e) {
      learn();
      c->err = e.msg;
      txn_rollback(*c);
      cudaGetLastError();
      return e.st;
    }
  } catch (const LdlError& e) {
    t_count_batch = false;
    c->err += std::string("; ") + e.msg;
    cudaGetLastError();
    return LDL_E_CUDA;
  }
  if (out) {
    *out = c->res;
    out->labels = c->lv[0].lab.p;
    out->n = c->n;
    out->changed = c->lChg.p;
    out->levels = c->T + 1;
    for (int r = 0; r < 8; ++r) {
      const bool has = r <= c->T;
      c->out_par[r] = has ? c->lv[r].par.p : nullptr;
      c->out_lab[r] = has ? c->lv[r].lab.p : nullptr;
      c->out_alive[r] = has ? c->lv[r].alive.p : nullptr;
    }
    out->parent = c->out_par;
    out->comm = c->out_lab;
    out->refined = c->out_par;
    out->alive = c->out_alive;
  }
  return LDL_OK;
}

ldl_status ldl_batch_estimate_bytes(const ldl_ctx* c, int64_t count, int64_t* bytes) {
  if (!c || !bytes || count < 0) return LDL_E_INVALID;
  const int64_t n = c->n, levels = c->T + 1;
  int64_t b = 0;
  if (!c->prm.no_rollback) {  // the snapshot buffer, allocated by the first atomic batch
    const int64_t want = levels * n * (c->directed ? 29 : 21) + n * (c->directed ? 24 : 16);
    if (c->snap.cap < want) b += want;
  }
  // records of the repair and of the aggregate levels: a budget of 8 per
  // update and level beyond the record buffers' current capacity, each kept
  // in about four 16-byte buffers (keys, values, sort scratch)
  const int64_t rec = 16 * count * levels;
  b += std::max<int64_t>(0, rec - c->rk.cap) * 16 * 4;
  // pending records of the levels above 0, applied when a level is next read
  for (int r = 1; r <= c->T; ++r) b += std::max<int64_t>(0, rec - c->lv[r].pk.cap) * 16;
  // a pool whose headroom is short may be compacted into one twice its live
  // capacity, kept beside the old one until the batch commits
  auto pool = [&](const auto& g, int64_t wbytes) {
    const int64_t head = g.col.cap - g.pool_top;
    if (head < g.pool_top / 4 + 4 * count) b += 2 * (g.pool_top + 4 * count) * (4 + wbytes);
  };
  pool(c->lv[0].out0, 4);
  for (int r = 1; r <= c->T; ++r) pool(c->lv[r].out, 8);
  // a batch whose frontier spreads over hubs can need far more: the most any
  // earlier batch of this context asked for per update bounds it from below
  b = std::max(b, c->grow_per_update * count);
  *bytes = b;
  return LDL_OK;
}

ldl_status ldl_modularity(const ldl_ctx* c, double* q) {
  if (!c || !q) return LDL_E_INVALID;
  if (c->m == 0) {
    *q = 0.0;
    return LDL_OK;
  }
  const double m = (double)c->m;
  *q = (double)qnum(*c) / ((double)c->prm.gamma_den * m * m);
  return LDL_OK;
}

ldl_status ldl_modularity_num(const ldl_ctx* c, int64_t* q_hi, uint64_t* q_lo, int64_t* m) {
  if (!c) return LDL_E_INVALID;
  const i128 q = qnum(*c);
  if (q_hi) *q_hi = (int64_t)(q >> 64);
  if (q_lo) *q_lo = (uint64_t)q;
  if (m) *m = c->m;
  return LDL_OK;
}

void ldl_destroy(ldl_ctx* c) {
  if (!c) return;
  try {
    DeviceScope ds(c->dev);
    free_all(*c);
  } catch (...) {
  }
  delete c;
}

const char* ldl_last_error(const ldl_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

int32_t ldl_levels(const ldl_ctx* c) { return c ? c->T + 1 : 0; }

int64_t ldl_num_vertices(const ldl_ctx* c) { return c ? c->n : 0; }

int32_t ldl_is_directed(const ldl_ctx* c) { return c ? c->directed : 0; }

ldl_status ldl_get_level(const ldl_ctx* cc, int32_t r, int32_t* lab, int32_t* par, int64_t* kout, int64_t* kin,
                         int32_t* cnt, uint8_t* alive) {
  if (!cc || r < 0 || r > cc->T) return LDL_E_INVALID;
  ldl_ctx& c = const_cast<ldl_ctx&>(*cc);
  try {
    DeviceScope ds(c.dev);
    const LevelState& L = c.lv[r];
    const size_t n = (size_t)c.n;
    if (lab) CK(cudaMemcpyAsync(lab, L.lab.p, 4 * n, cudaMemcpyDeviceToHost, c.s));
    if (par) CK(cudaMemcpyAsync(par, L.par.p, 4 * n, cudaMemcpyDeviceToHost, c.s));
    if (kout) CK(cudaMemcpyAsync(kout, L.kout.p, 8 * n, cudaMemcpyDeviceToHost, c.s));
    if (kin) CK(cudaMemcpyAsync(kin, kin_of(c, r), 8 * n, cudaMemcpyDeviceToHost, c.s));
    if (cnt) CK(cudaMemcpyAsync(cnt, L.cnt.p, 4 * n, cudaMemcpyDeviceToHost, c.s));
    if (alive) CK(cudaMemcpyAsync(alive, L.alive.p, n, cudaMemcpyDeviceToHost, c.s));
    CK(cudaStreamSynchronize(c.s));
    if (r == c.T && par)
      for (size_t v = 0; v < n; ++v) par[v] = -1;
  } catch (const LdlError& e) {
    c.err = e.msg;
    return e.st;
  }
  return LDL_OK;
}

ldl_status ldl_level_nnz(const ldl_ctx* cc, int32_t r, int64_t* nnz) {
  if (!cc || !nnz || r < 0 || r > cc->T) return LDL_E_INVALID;
  ldl_ctx& c = const_cast<ldl_ctx&>(*cc);
  try {
    DeviceScope ds(c.dev);
    std::vector<int32_t> len((size_t)c.n);
    const DBuf<int32_t>& lp = r == 0 ? c.lv[0].out0.len : c.lv[r].out.len;
    CK(cudaMemcpyAsync(len.data(), lp.p, 4 * (size_t)c.n, cudaMemcpyDeviceToHost, c.s));
    CK(cudaStreamSynchronize(c.s));
    int64_t s = 0;
    for (int32_t x : len) s += x;
    *nnz = s;
  } catch (const LdlError& e) {
    c.err = e.msg;
    return e.st;
  }
  return LDL_OK;
}

ldl_status ldl_get_adjacency(const ldl_ctx* cc, int32_t r, int64_t* row_ptr, int32_t* col, int64_t* w) {
  if (!cc || !row_ptr || r < 0 || r > cc->T) return LDL_E_INVALID;
  ldl_ctx& c = const_cast<ldl_ctx&>(*cc);
  try {
    DeviceScope ds(c.dev);
    std::vector<int64_t> off;
    std::vector<int32_t> len, cl;
    std::vector<std::pair<int32_t, int64_t>> row;
    int64_t k = 0;
    auto emit = [&](auto& wv) {
      for (int64_t v = 0; v < c.n; ++v) {
        row_ptr[v] = k;
        row.clear();
        for (int32_t j = 0; j < len[v]; ++j) row.emplace_back(cl[off[v] + j], (int64_t)wv[off[v] + j]);
        std::sort(row.begin(), row.end());
        for (auto& p : row) {
          if (col) col[k] = p.first;
          if (w) w[k] = p.second;
          ++k;
        }
      }
      row_ptr[c.n] = k;
    };
    if (r == 0) {
      std::vector<int32_t> wv;
      copy_adj<int32_t>(c, c.lv[0].out0, off, len, cl, wv);
      emit(wv);
    } else {
      std::vector<int64_t> wv;
      copy_adj<int64_t>(c, c.lv[r].out, off, len, cl, wv);
      emit(wv);
    }
  } catch (const LdlError& e) {
    c.err = e.msg;
    return e.st;
  }
  return LDL_OK;
}

ldl_status ldl_get_communities(const ldl_ctx* cc, int64_t* kout, int64_t* kin, int64_t* e) {
  if (!cc) return LDL_E_INVALID;
  ldl_ctx& c = const_cast<ldl_ctx&>(*cc);
  try {
    DeviceScope ds(c.dev);
    const size_t n = (size_t)c.n;
    if (kout) CK(cudaMemcpyAsync(kout, c.Kout.p, 8 * n, cudaMemcpyDeviceToHost, c.s));
    if (kin) CK(cudaMemcpyAsync(kin, Kin_of(c), 8 * n, cudaMemcpyDeviceToHost, c.s));
    if (e) CK(cudaMemcpyAsync(e, c.e.p, 8 * n, cudaMemcpyDeviceToHost, c.s));
    CK(cudaStreamSynchronize(c.s));
  } catch (const LdlError& er) {
    c.err = er.msg;
    return er.st;
  }
  return LDL_OK;
}

ldl_status ldl_stage_times(const ldl_ctx* c, double* times) {
  if (!c || !times) return LDL_E_INVALID;
  for (int i = 0; i < 16; ++i) times[i] = c->stage_ms[i];
  return LDL_OK;
}

ldl_status ldl_set_timing(ldl_ctx* c, int32_t on) {
  if (!c) return LDL_E_INVALID;
  c->timing = on ? 1 : 0;
  for (double& x : c->stage_ms) x = 0;
  return LDL_OK;
}

void ldl_debug_fail_alloc_after(int64_t k) { g_fail_after.store(k > 0 ? k : 0); }

void ldl_debug_alloc_counts(int64_t* all, int64_t* in_batch) {
  if (all) *all = g_allocs.load();
  if (in_batch) *in_batch = g_txn_allocs.load();
}

ldl_status ldl_debug_scan_wait_timeout(void) {
  try {
    return scan_wait_gives_up(nullptr) ? LDL_E_TIMEOUT : LDL_OK;
  } catch (const LdlError& e) {
    return e.st;
  }
}

int64_t ldl_launch_count(void) { return g_launches.load(); }

ldl_status ldl_debug_sort_pairs(ldl_ctx* c, int64_t count, uint64_t* keys, uint64_t* vals, int32_t bits) {
  if (!c || count < 0 || bits < 1 || bits > 64 || (count > 0 && (!keys || !vals))) return LDL_E_INVALID;
  if (bits < 64) {
    for (int64_t i = 0; i < count; ++i)
      if (keys[i] >> bits) {
        c->err = "ldl_debug_sort_pairs: a key has bits above `bits`";
        return LDL_E_INVALID;
      }
  }
  ldl_ctx& x = *c;
  DBuf<u64> dk, dv, tk, tv;
  ldl_status st = LDL_OK;
  try {
    DeviceScope ds(c->dev);
    const size_t k = (size_t)count;
    dk.reserve(count + 1, x.s);
    dv.reserve(count + 1, x.s);
    if (k) {
      CK(cudaMemcpyAsync(dk.p, keys, 8 * k, cudaMemcpyHostToDevice, x.s));
      CK(cudaMemcpyAsync(dv.p, vals, 8 * k, cudaMemcpyHostToDevice, x.s));
    }
    sort_pairs(dk, dv, tk, tv, count, bits, x.P, x.s);
    if (k) {
      CK(cudaMemcpyAsync(keys, dk.p, 8 * k, cudaMemcpyDeviceToHost, x.s));
      CK(cudaMemcpyAsync(vals, dv.p, 8 * k, cudaMemcpyDeviceToHost, x.s));
    }
    CK(cudaStreamSynchronize(x.s));
  } catch (const LdlError& e) {
    c->err = e.msg;
    cudaGetLastError();
    st = e.st;
  }
  try {
    DeviceScope ds(c->dev);
    cudaStreamSynchronize(x.s);
    dk.release();
    dv.release();
    tk.release();
    tv.release();
  } catch (const LdlError& e) {
    if (st == LDL_OK) st = e.st;
  }
  return st;
}

ldl_status ldl_debug_decouple(ldl_ctx* c, int64_t count, const int32_t* v, const int32_t* src, const int32_t* dst,
                              const int64_t* g_hi, const uint64_t* g_lo, uint8_t* accepted) {
  if (!c || count < 0 || count > c->n || (count > 0 && (!v || !src || !dst || !g_hi || !g_lo || !accepted)))
    return LDL_E_INVALID;
  std::vector<uint8_t> seen((size_t)c->n, 0);
  for (int64_t k = 0; k < count; ++k) {
    if (v[k] < 0 || v[k] >= c->n || src[k] < 0 || src[k] >= c->n || dst[k] < 0 || dst[k] >= c->n ||
        src[k] == dst[k] || seen[(size_t)v[k]]) {
      c->err = "ldl_debug_decouple: ids must lie in [0, n), nodes must be distinct and src != dst";
      return LDL_E_INVALID;
    }
    seen[(size_t)v[k]] = 1;
  }
  try {
    DeviceScope ds(c->dev);
    ldl_ctx& x = *c;
    const size_t k = (size_t)count;
    if (k) {
      CK(cudaMemcpyAsync(x.cv.p, v, 4 * k, cudaMemcpyHostToDevice, x.s));
      CK(cudaMemcpyAsync(x.csrc.p, src, 4 * k, cudaMemcpyHostToDevice, x.s));
      CK(cudaMemcpyAsync(x.cdst.p, dst, 4 * k, cudaMemcpyHostToDevice, x.s));
      CK(cudaMemcpyAsync(x.cghi.p, g_hi, 8 * k, cudaMemcpyHostToDevice, x.s));
      CK(cudaMemcpyAsync(x.cglo.p, g_lo, 8 * k, cudaMemcpyHostToDevice, x.s));
    }
    set_cnt(x, K_CAND, (int32_t)count);
    const ldl_result keep = x.res;
    const int64_t keep_syncs = x.syncs;
    const DecoupleOut d = decouple(x);
    x.res = keep;
    x.syncs = keep_syncs;
    std::vector<int32_t> bv((size_t)std::max(d.nb, 1));
    if (d.nb > 0) CK(cudaMemcpyAsync(bv.data(), x.bv.p, 4 * (size_t)d.nb, cudaMemcpyDeviceToHost, x.s));
    CK(cudaStreamSynchronize(x.s));
    std::vector<uint8_t> acc((size_t)x.n, 0);
    for (int32_t i = 0; i < d.nb; ++i) acc[(size_t)bv[(size_t)i]] = 1;
    for (int64_t i = 0; i < count; ++i) accepted[i] = acc[(size_t)v[i]];
  } catch (const LdlError& e) {
    c->err = e.msg;
    cudaGetLastError();
    return e.st;
  }
  return LDL_OK;
}

ldl_status ldl_copy_changed(const ldl_ctx* cc, int32_t* ids, int32_t* labels) {
  if (!cc) return LDL_E_INVALID;
  ldl_ctx& c = const_cast<ldl_ctx&>(*cc);
  const int64_t k = c.res.n_changed;
  if (k == 0) return LDL_OK;
  if (!ids) return LDL_E_INVALID;
  try {
    DeviceScope ds(c.dev);
    CK(cudaMemcpyAsync(ids, c.lChg.p, sizeof(int32_t) * (size_t)k, cudaMemcpyDeviceToHost, c.s));
    CK(cudaStreamSynchronize(c.s));
    if (labels) {
      gather_labels(c, c.lChg.p, (int32_t)k, c.lTmp.p);
      CK(cudaMemcpyAsync(labels, c.lTmp.p, sizeof(int32_t) * (size_t)k, cudaMemcpyDeviceToHost, c.s));
      CK(cudaStreamSynchronize(c.s));
    }
  } catch (const LdlError& e) {
    c.err = e.msg;
    return e.st;
  }
  return LDL_OK;
}

ldl_status ldl_set_kernel_stats(ldl_ctx* c, int32_t on) {
  if (!c) return LDL_E_INVALID;
  try {
    DeviceScope ds(c->dev);
    c->kstats = on ? 1 : 0;
    c->kev_used = 0;
    for (int k = 0; k < KS_GROUPS; ++k) c->ks_launch[k] = 0;
    CK(cudaMemsetAsync(c->d_sc->sw_entries, 0, sizeof(int64_t) * 2 * KS_GROUPS, c->s));
    CK(cudaStreamSynchronize(c->s));
  } catch (const LdlError& e) {
    c->err = e.msg;
    return e.st;
  }
  return LDL_OK;
}

ldl_status ldl_get_kernel_stats(const ldl_ctx* c, double* out) {
  if (!c || !out) return LDL_E_INVALID;
  try {
    DeviceScope ds(c->dev);
    double ms[KS_GROUPS] = {0, 0, 0, 0, 0, 0, 0};
    if (c->kev_used) CK(cudaEventSynchronize(c->kev[c->kev_used - 1]));
    for (size_t i = 0; i + KS_EVENTS <= c->kev_used; i += KS_EVENTS)
      for (int j = 0; j + 1 < KS_EVENTS; ++j) {
        float t = 0;
        if (ks_interval_group(j) < 0) continue;
        CK(cudaEventElapsedTime(&t, c->kev[i + j], c->kev[i + j + 1]));
        ms[ks_interval_group(j)] += t;
      }
    DevScalars h;
    CK(cudaMemcpy(&h, c->d_sc, sizeof(DevScalars), cudaMemcpyDeviceToHost));
    for (int k = 0; k < KS_GROUPS; ++k) {
      out[4 * k + 0] = c->ks_launch[k];
      out[4 * k + 1] = ms[k];
      out[4 * k + 2] = (double)h.sw_bytes[k];
      out[4 * k + 3] = (double)h.sw_entries[k];
    }
  } catch (const LdlError& e) {
    return e.st;
  }
  return LDL_OK;
}

}  // extern "C"
