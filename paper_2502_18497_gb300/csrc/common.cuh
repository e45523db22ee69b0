// Shared device helpers and internal declarations of the LD-Leiden library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ldl.h"

typedef __int128 i128;
typedef int64_t i64;
typedef uint64_t u64;

#define LDL_NONE (-1)
#define WARP 32

// ---------------------------------------------------------------- errors
struct LdlError {
  ldl_status st;
  std::string msg;
};

void ldl_throw(ldl_status st, const std::string& msg);
void ldl_cuda_check(cudaError_t e, const char* what, const char* file, int line);
#define CK(x) ldl_cuda_check((x), #x, __FILE__, __LINE__)
extern std::atomic<int64_t> g_launches;  // kernels launched by this library
#define CKL(name) (g_launches.fetch_add(1, std::memory_order_relaxed), ldl_cuda_check(cudaGetLastError(), name, __FILE__, __LINE__))

// ---------------------------------------------------------------- device memory
// All device allocations of a context go through dalloc/dfree so that a test
// can make the k-th one fail.
void* dalloc(size_t bytes);
void dfree(void* p);

template <class T>
struct DBuf {
  T* p = nullptr;
  int64_t cap = 0;
  void reserve(int64_t n, cudaStream_t s, bool keep = false) {
    if (n <= cap) return;
    int64_t nc = cap ? cap : 1024;
    while (nc < n) nc = nc * 3 / 2 + 1024;
    T* q = (T*)dalloc((size_t)nc * sizeof(T));
    if (keep && p && cap) CK(cudaMemcpyAsync(q, p, (size_t)cap * sizeof(T), cudaMemcpyDeviceToDevice, s));
    if (p) {
      CK(cudaStreamSynchronize(s));
      dfree(p);
    }
    p = q;
    cap = nc;
  }
  void exact(int64_t n) {  // allocate exactly n (no growth policy)
    if (n <= cap) return;
    T* q = (T*)dalloc((size_t)(n > 0 ? n : 1) * sizeof(T));
    if (p) dfree(p);
    p = q;
    cap = n;
  }
  void release() {
    if (p) dfree(p);
    p = nullptr;
    cap = 0;
  }
};

// ---------------------------------------------------------------- int128 helpers
// One device value to copy to the host (see host_read).
struct HostRead {
  const void* src;  // device
  void* dst;        // host
  int32_t bytes;
};
using HostReadFn = void (*)(void* owner, const HostRead* r, int n);

struct I128 {  // two's complement halves; host and device
  int64_t hi;
  uint64_t lo;
};

__host__ __device__ inline i128 i128_of(int64_t hi, uint64_t lo) {
  return (i128)(((unsigned __int128)(uint64_t)hi << 64) | (unsigned __int128)lo);
}

// Atomic add of a signed 128-bit value into (hi, lo) halves.
__device__ inline void atomic_add_i128(I128* dst, i128 v) {
  if (v == 0) return;
  uint64_t vl = (uint64_t)v;
  int64_t vh = (int64_t)(v >> 64);
  unsigned long long old = atomicAdd((unsigned long long*)&dst->lo, (unsigned long long)vl);
  uint64_t carry = ((uint64_t)old + vl) < (uint64_t)old ? 1 : 0;
  int64_t add_hi = vh + (int64_t)carry;
  if (add_hi != 0) atomicAdd((unsigned long long*)&dst->hi, (unsigned long long)add_hi);
}

__device__ inline void atomic_add_i64(int64_t* p, int64_t v) {
  atomicAdd((unsigned long long*)p, (unsigned long long)v);
}

__device__ inline i128 shfl_down_i128(i128 v, int d) {
  uint64_t lo = (uint64_t)v;
  int64_t hi = (int64_t)(v >> 64);
  lo = __shfl_down_sync(0xffffffffu, lo, d);
  hi = __shfl_down_sync(0xffffffffu, hi, d);
  return i128_of(hi, lo);
}

__device__ inline i128 shfl_i128(i128 v, int src) {
  uint64_t lo = (uint64_t)v;
  int64_t hi = (int64_t)(v >> 64);
  lo = __shfl_sync(0xffffffffu, lo, src);
  hi = __shfl_sync(0xffffffffu, hi, src);
  return i128_of(hi, lo);
}

// Width-w variants: lanes are split into segments of w (a power of two);
// shuffles stay inside a lane's own segment.
__device__ inline i128 shfl_down_i128_w(i128 v, int d, int w) {
  uint64_t lo = (uint64_t)v;
  int64_t hi = (int64_t)(v >> 64);
  lo = __shfl_down_sync(0xffffffffu, lo, d, w);
  hi = __shfl_down_sync(0xffffffffu, hi, d, w);
  return i128_of(hi, lo);
}

__device__ inline i128 shfl_i128_w(i128 v, int src, int w) {
  uint64_t lo = (uint64_t)v;
  int64_t hi = (int64_t)(v >> 64);
  lo = __shfl_sync(0xffffffffu, lo, src, w);
  hi = __shfl_sync(0xffffffffu, hi, src, w);
  return i128_of(hi, lo);
}

__device__ inline i128 warp_sum_i128(i128 v) {
  for (int d = 16; d > 0; d >>= 1) v += shfl_down_i128(v, d);
  return v;  // valid in lane 0
}

__device__ inline int64_t warp_sum_i64(int64_t v) {
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  return v;
}

__device__ inline int warp_sum_i32(int v) {
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  return v;
}

// Argmax pair (g, c): larger g wins, equal g goes to the smaller c; "have"
// marks a valid entry.  Reduced over the whole warp (result in every lane).
struct Best {
  i128 g;
  int32_t c;
  int32_t have;
};

__device__ inline bool best_better(const Best& a, const Best& b) {  // a beats b
  if (!a.have) return false;
  if (!b.have) return true;
  if (a.g != b.g) return a.g > b.g;
  return a.c < b.c;
}

__device__ inline Best warp_best(Best x) {
  for (int d = 16; d > 0; d >>= 1) {
    Best o;
    o.g = shfl_down_i128(x.g, d);
    o.c = __shfl_down_sync(0xffffffffu, x.c, d);
    o.have = __shfl_down_sync(0xffffffffu, x.have, d);
    if (best_better(o, x)) x = o;
  }
  x.g = shfl_i128(x.g, 0);
  x.c = __shfl_sync(0xffffffffu, x.c, 0);
  x.have = __shfl_sync(0xffffffffu, x.have, 0);
  return x;
}

// The same argmax over each segment of G lanes (every lane of the warp takes
// part; the result lands in every lane of the segment).
template <int G>
__device__ inline Best group_best(Best x) {
  for (int d = G / 2; d > 0; d >>= 1) {
    Best o;
    o.g = shfl_down_i128_w(x.g, d, G);
    o.c = __shfl_down_sync(0xffffffffu, x.c, d, G);
    o.have = __shfl_down_sync(0xffffffffu, x.have, d, G);
    if (best_better(o, x)) x = o;
  }
  x.g = shfl_i128_w(x.g, 0, G);
  x.c = __shfl_sync(0xffffffffu, x.c, 0, G);
  x.have = __shfl_sync(0xffffffffu, x.have, 0, G);
  return x;
}

__device__ inline uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

// Append to a list with a dedup stamp: returns true if x was newly added.
__device__ inline bool stamp_add(int32_t* stamp, int32_t ep, int32_t x, int32_t* list, int32_t* count) {
  if (stamp[x] == ep) return false;
  if (atomicExch(&stamp[x], ep) == ep) return false;
  int32_t pos = atomicAdd(count, 1);
  list[pos] = x;
  return true;
}

// Warp-aggregated append: every lane of the warp calls it together; lanes with
// `want` append x.  One atomic per warp.
__device__ inline void warp_append(bool want, int32_t x, int32_t* list, int32_t* count) {
  const unsigned m = __ballot_sync(0xffffffffu, want);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  int32_t base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (want) list[base + __popc(m & ((1u << lane) - 1u))] = x;
}

// Claims x for the set with epoch ep (true only for the first claimer).
__device__ inline bool stamp_claim(int32_t* stamp, int32_t ep, int32_t x) {
  if (stamp[x] == ep) return false;
  return atomicExch(&stamp[x], ep) != ep;
}

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
// Streaming multiprocessors of the current device (queried once per device).
int device_sms();
// Blocks for n items of `block` per block, at most per_sm blocks per SM of
// the current device (grid-stride kernels cover the rest).
inline int grid_for(int64_t n, int block, int per_sm = 32) {
  int64_t g = (n + block - 1) / block;
  const int64_t cap = (int64_t)per_sm * device_sms();
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// Makes the context's device current for the duration of an entry point and
// restores the caller's device afterwards.
struct DeviceScope {
  int prev = -1, dev = -1;
  explicit DeviceScope(int d);
  ~DeviceScope();
};

// ---------------------------------------------------------------- slack CSR
// Rows in [0, n): row v occupies pool[off[v], off[v]+len[v]) with capacity
// cap[v].  A row that outgrows its capacity is moved to the end of the pool.
template <class WT>
struct SlackCSR {
  int64_t n = 0;
  DBuf<int64_t> off;
  DBuf<int32_t> len, cap;
  DBuf<int32_t> col;
  DBuf<WT> w;
  int64_t pool_top = 0;  // host mirror of the first free pool slot
  // Undo log of a batch that may be rolled back (csr_txn_*).  While logging,
  // every update records, before it changes anything, the old offset, length
  // and capacity of each row it touches, the old contents of the rows it
  // rewrites and the old weights it overwrites; a compaction first saves the
  // whole offset table, and the pool in use when the batch began is kept
  // until the batch commits.  A rollback replays the events in reverse.
  struct Event {
    bool offsets;          // a saved offset table (before a compaction) or a row chunk
    int64_t r0, nr;        // row entries
    int64_t w0, nw;        // weight entries
    int64_t o0;            // saved offsets
    int32_t* col;          // the pool the update wrote into
  };
  bool logging = false;
  int32_t* col0 = nullptr;  // the pool at the start of the batch
  WT* w0 = nullptr;
  int64_t cap0 = 0, top0 = 0;
  std::vector<std::pair<int32_t*, WT*>> retired;
  std::vector<Event> events;
  int64_t rtop = 0, wtop = 0, ctop = 0, otop = 0;
  DBuf<int64_t> lrow, loff, lsrc, lpos, lofs;
  DBuf<int32_t> llen, lcap, lcol;
  DBuf<WT> lw, lold;
  void release() {
    off.release(); len.release(); cap.release(); col.release(); w.release();
    for (auto& x : retired) {
      if (x.first != col.p) dfree(x.first);
      if (x.second != w.p) dfree(x.second);
    }
    retired.clear();
    lrow.release(); loff.release(); lsrc.release(); lpos.release(); lofs.release();
    llen.release(); lcap.release(); lcol.release(); lw.release(); lold.release();
    events.clear();
    logging = false;
    pool_top = 0;
  }
};

// ---------------------------------------------------------------- scalar block
// One small device struct read back in a single copy.
// Sweep kernel groups with their own statistics: 0 8-lane groups, 1 warps,
// 2 128-thread blocks, 3 256-thread blocks, 4 block clusters, 5 the hub
// accumulation kernel, 6 the rest of the hub path (table set-up, evaluation,
// final reduction).  A sweep records KS_EVENTS events; interval j (event j to
// j + 1) is charged to group ks_interval_group(j), or to none (-1: the host's
// wait for the bin counts).
constexpr int KS_GROUPS = 7;
constexpr int KS_EVENTS = 10;
__host__ __device__ constexpr int ks_interval_group(int j) { return j < 5 ? j : j == 5 ? -1 : j == 7 ? 5 : 6; }

struct DevScalars {
  I128 dq;          // numerator change of the current mini-batch
  I128 dp;          // change of sum_C K_out K_in
  I128 p_old, p_new;
  int64_t de;       // change of sum_C e_C
  int64_t dm;       // change of m (batch)
  int64_t need;     // pool slots needed by relocation
  int64_t need2;    // second accumulator (record counts)
  int64_t scanned;  // adjacency entries scanned
  int64_t err_key;  // packed (index << 8 | status) of the first failing update
  int64_t pool_top;
  int64_t seg_n, seg_stot, seg_wtot;  // CSR update: segments, scratch and rebuild totals
  int64_t sw_entries[KS_GROUPS];  // per sweep kernel group: adjacency entries read since statistics
                                  // were enabled
  int64_t sw_bytes[KS_GROUPS];    // algorithmic bytes of the same sweeps
  int32_t cnt[16];  // list counters
  int32_t undecided;
  int32_t pad;
};

enum {  // indices into DevScalars::cnt
  C_LIST0 = 0, C_LIST1, C_LIST2, C_LIST3, C_LIST4, C_LIST5, C_LIST6, C_LIST7,
  C_CAND, C_REC, C_SEG, C_ACC, C_TC, C_X, C_Y, C_Z
};
