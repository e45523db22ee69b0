// Frontier sweeps of Algorithm 1: candidate-set expansion (Expand, SPExpand),
// BestMove / BestRef with the exact Eq. 2 gain, the decoupling
// filter of Sec. III-E as deterministic parallel rounds, and the commit of an
// accepted mini-batch with the additive repair of the community totals and
// the exact modularity change dQ(B) with its rollback test.
#include <atomic>
#include <cooperative_groups.h>

#include "chunks.cuh"
#include "kern.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int TPB = 256;
constexpr int HG8 = 64;      // hash slots per 8-lane group (lowest bin)
constexpr int HG32 = 256;    // hash slots per warp (second bin)
constexpr int HB = 4096;     // per-block hash slots (upper mid bin)
constexpr int MID_DEG = 2048;   // rows above it: clusters (optional) or the hub path
constexpr int CL = 8;             // blocks per cluster (hub rows up to CLUSTER_DEG entries)
constexpr int CL_SLOTS = 8192;    // hash slots per block of a cluster (96 KB of shared memory)
constexpr int CLUSTER_DEG = CL * CL_SLOTS / 2;  // upper limit of cluster_max_deg
constexpr int64_t HUB_TABLE_SLOTS = (int64_t)1 << 28;  // hub hash slots held at once (3 GB)
// the bound in force (a test hook lowers it)
std::atomic<int64_t> g_hub_table_slots{HUB_TABLE_SLOTS};
// the bin bounds a context may use keep every table at most half full
static_assert(BIN_MAX[0] == HG8 / 2 && BIN_MAX[1] == HG32 / 2 && BIN_MAX[2] == 2048 / 2 &&
                  BIN_MAX[3] == HB / 2 && BIN_MAX[3] == MID_DEG,
              "bin bounds and table sizes");
constexpr int EVAL_CH = 4096;  // hub table slots evaluated per block

// ---------------------------------------------------------------- expand
// out = U plus every out- and in-neighbour of U (dedup by stamp).
template <class WT>
__global__ void k_expand(Adj<WT> out, Adj<WT> in, ChunkMap m, int32_t* stamp, int32_t ep, int32_t* olist,
                         int32_t* nout) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = m.pre[m.n_hint];
  for (int64_t c = warp; c < total; c += nw) {
    const Chunk ch = chunk_of(m, c);
    if (ch.first && lane == 0) stamp_add(stamp, ep, ch.v, olist, nout);
    if (ch.row < 0) continue;
    const Adj<WT>& A = ch.row ? in : out;
    const int64_t o = A.off[ch.v];
    for (int32_t base = ch.k0; base < ch.k1; base += 32) {
      const int32_t k = base + lane;
      bool want = false;
      int32_t u = 0;
      if (k < ch.k1) {
        u = A.col[o + k];
        want = stamp_claim(stamp, ep, u);
      }
      warp_append(want, u, olist, nout);
    }
  }
}

__global__ void k_filter_alive(const int32_t* list, const int32_t* nlist, const uint8_t* alive, int32_t* olist,
                               int32_t* nout) {
  const int32_t nl = *nlist;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nl; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = list[t];
    if (!alive || alive[v]) olist[atomicAdd(nout, 1)] = v;
  }
}

__global__ void k_union(const int32_t* list, const int32_t* nlist, int32_t* stamp, int32_t ep, int32_t* olist,
                        int32_t* nout) {
  const int32_t nl = *nlist;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nl; t += (int64_t)gridDim.x * blockDim.x)
    stamp_add(stamp, ep, list[t], olist, nout);
}

// ---------------------------------------------------------------- sweep
// MODE 0: BestMove over community labels.  MODE 1: BestRef over refined ids
// (level-r parents) restricted to neighbours of the same community.
template <class WT>
struct SweepArgs {
  Adj<WT> out, in;
  int directed;
  const int32_t* lab;
  const int32_t* par;
  const int64_t* kout;
  const int64_t* kin;
  const int64_t* Tout;  // MODE 0: community K_out; MODE 1: level r+1 k_out
  const int64_t* Tin;
  int64_t m, gn, gd;
  int32_t* cv;
  int32_t* csrc;
  int32_t* cdst;
  int64_t* cghi;
  uint64_t* cglo;
  int32_t* ncand;
  int64_t* scanned;
  DevScalars* stats;
};

__device__ inline void hash_add(int32_t* K, int64_t* V, uint32_t mask, int32_t key, int64_t w) {
  uint32_t h = hash32((uint32_t)key) & mask;
  while (true) {
    const int32_t prev = atomicCAS(&K[h], -1, key);
    if (prev == -1 || prev == key) {
      atomicAdd((unsigned long long*)&V[h], (unsigned long long)w);
      return;
    }
    h = (h + 1) & mask;
  }
}

__device__ inline int64_t hash_get(const int32_t* K, const int64_t* V, uint32_t mask, int32_t key) {
  uint32_t h = hash32((uint32_t)key) & mask;
  while (true) {
    const int32_t k = K[h];
    if (k == key) return V[h];
    if (k == -1) return 0;
    h = (h + 1) & mask;
  }
}

template <class WT, int MODE>
__device__ inline void accumulate(const SweepArgs<WT>& A, const Adj<WT>& adj, int32_t v, int32_t cv_, int32_t* K,
                                  int64_t* V, uint32_t mask, int tid, int nthreads) {
  // ACC entries per thread per step: their loads and label gathers are all in
  // flight before the first insert
  constexpr int ACC = 4;
  const int64_t o = adj.off[v];
  const int32_t l = adj.len[v];
  for (int32_t k0 = tid; k0 < l; k0 += ACC * nthreads) {
    int32_t u[ACC];
    int64_t w[ACC];
#pragma unroll
    for (int j = 0; j < ACC; ++j) {
      const int32_t k = k0 + j * nthreads;
      u[j] = k < l ? adj.col[o + k] : -1;
      w[j] = k < l ? (int64_t)adj.w[o + k] : 0;
    }
    int32_t key[ACC];
#pragma unroll
    for (int j = 0; j < ACC; ++j) {
      key[j] = -1;
      if (u[j] >= 0 && u[j] != v && (MODE == 0 || A.lab[u[j]] == cv_)) key[j] = MODE == 0 ? A.lab[u[j]] : A.par[u[j]];
    }
#pragma unroll
    for (int j = 0; j < ACC; ++j)
      if (key[j] >= 0) hash_add(K, V, mask, key[j], w[j]);
  }
}

// accumulate() for a row whose offset and length the caller already holds.
template <class WT, int MODE>
__device__ inline void accumulate_row(const SweepArgs<WT>& A, const int32_t* col, const WT* wt, int64_t o, int32_t l,
                                      int32_t v, int32_t cv_, int32_t* K, int64_t* V, uint32_t mask, int tid,
                                      int nthreads) {
  constexpr int ACC = 4;
  for (int32_t k0 = tid; k0 < l; k0 += ACC * nthreads) {
    int32_t u[ACC];
    int64_t w[ACC];
#pragma unroll
    for (int j = 0; j < ACC; ++j) {
      const int32_t k = k0 + j * nthreads;
      u[j] = k < l ? col[o + k] : -1;
      w[j] = k < l ? (int64_t)wt[o + k] : 0;
    }
    int32_t key[ACC];
#pragma unroll
    for (int j = 0; j < ACC; ++j) {
      key[j] = -1;
      if (u[j] >= 0 && u[j] != v && (MODE == 0 || A.lab[u[j]] == cv_)) key[j] = MODE == 0 ? A.lab[u[j]] : A.par[u[j]];
    }
#pragma unroll
    for (int j = 0; j < ACC; ++j)
      if (key[j] >= 0) hash_add(K, V, mask, key[j], w[j]);
  }
}

// A node's row offsets and lengths, label and strengths, loaded one node
// ahead of its sweep so that these dependent loads overlap the previous
// node's work.
struct NodeMeta {
  int32_t v, a, lo, li;
  int64_t oo, oi, ko, ki;
};

template <class WT>
__device__ inline NodeMeta node_meta(const SweepArgs<WT>& A, int32_t v) {
  NodeMeta m;
  m.v = v;
  m.lo = A.out.len[v];
  m.oo = A.out.off[v];
  m.li = A.directed ? A.in.len[v] : 0;
  m.oi = A.directed ? A.in.off[v] : 0;
  m.a = A.lab[v];
  m.ko = A.kout[v];
  m.ki = A.kin[v];
  return m;
}

// Exact gain of v into key (see Eq. 2 with a' = a \ {v}).
template <int MODE>
__device__ inline i128 gain_of(int32_t key, int64_t acc, int64_t wa, int32_t a, int64_t ko, int64_t ki,
                               const int64_t* Tout, const int64_t* Tin, int64_t m, int64_t gn, int64_t gd,
                               int64_t mult) {
  if (MODE == 0) {
    const i128 dw = (i128)mult * (acc - wa);
    const i128 dd = (i128)ko * (Tin[key] - Tin[a] + ki) + (i128)ki * (Tout[key] - Tout[a] + ko);
    return (i128)gd * m * dw - (i128)gn * dd;
  } else {
    const i128 dw = (i128)mult * acc;
    const i128 dd = (i128)ko * Tin[key] + (i128)ki * Tout[key];
    return (i128)gd * m * dw - (i128)gn * dd;
  }
}

// Algorithmic bytes of a sweep (the minimum a sweep must move): per adjacency
// entry the neighbour id, its weight and its label (refinement: also its
// parent); per swept node its offsets, lengths, label and strengths; per
// evaluated (node, target) pair the target's totals.
template <class WT, int MODE>
__device__ inline int64_t sweep_bytes(bool directed, int64_t entries, int64_t nodes, int64_t pairs) {
  const int64_t per_entry = 4 + sizeof(WT) + 4 + (MODE == 1 ? 4 : 0);
  const int64_t per_node = (8 + 4) * (directed ? 2 : 1) + 4 + 16 + 4;
  const int64_t per_pair = directed ? 16 : 8;
  return per_entry * entries + per_node * nodes + per_pair * pairs;
}

// The argmax (gain desc, target asc) in the gain's integer type GT: int64 when
// the host has checked that no gain or intermediate product of this sweep can
// reach 2^62 (sweep_gain_fits_i64), else int128.  Both give the same exact
// gains, so the choice never changes a result.
template <class GT>
struct BestG {
  GT g;
  int32_t c;
  int32_t have;
};

template <class GT>
__device__ inline bool better(const BestG<GT>& a, const BestG<GT>& b) {
  if (!a.have) return false;
  if (!b.have) return true;
  if (a.g != b.g) return a.g > b.g;
  return a.c < b.c;
}

__device__ inline int64_t shfl_down_g(int64_t v, int d, int w) { return __shfl_down_sync(0xffffffffu, v, d, w); }
__device__ inline i128 shfl_down_g(i128 v, int d, int w) { return shfl_down_i128_w(v, d, w); }
__device__ inline int64_t shfl_g(int64_t v, int src, int w) { return __shfl_sync(0xffffffffu, v, src, w); }
__device__ inline i128 shfl_g(i128 v, int src, int w) { return shfl_i128_w(v, src, w); }

// Argmax over each segment of G lanes (every lane takes part; the result
// lands in every lane of the segment).  G = 32: the whole warp.
template <class GT, int G>
__device__ inline BestG<GT> seg_best(BestG<GT> x) {
  for (int d = G / 2; d > 0; d >>= 1) {
    BestG<GT> o;
    o.g = shfl_down_g(x.g, d, G);
    o.c = __shfl_down_sync(0xffffffffu, x.c, d, G);
    o.have = __shfl_down_sync(0xffffffffu, x.have, d, G);
    if (better(o, x)) x = o;
  }
  x.g = shfl_g(x.g, 0, G);
  x.c = __shfl_sync(0xffffffffu, x.c, 0, G);
  x.have = __shfl_sync(0xffffffffu, x.have, 0, G);
  return x;
}

// Evaluates the slots start, start + step, ... < H of a node's table: the
// exact gain (as gain_of) into every target but `self`, the best kept in b.
// EV slots per step have their totals gathered before any gain is computed.
template <int MODE, class GT>
__device__ inline void eval_slots(const int32_t* K, const int64_t* V, uint32_t H, uint32_t start, uint32_t step,
                                  int32_t self, int32_t a, int64_t wa, int64_t ko, int64_t ki, const int64_t* Tout,
                                  const int64_t* Tin, int64_t m, int64_t gn, int64_t gd, int64_t mult, BestG<GT>& b,
                                  int64_t& pairs) {
  constexpr int EV = 1;
  const int64_t tia = MODE == 0 ? Tin[a] : 0, toa = MODE == 0 ? Tout[a] : 0;
  for (uint32_t k0 = start; k0 < H; k0 += EV * step) {
    int32_t key[EV];
    int64_t acc[EV], ti[EV], to[EV];
#pragma unroll
    for (int j = 0; j < EV; ++j) {
      const uint32_t k = k0 + j * step;
      key[j] = k < H ? K[k] : -1;
      if (key[j] == self) key[j] = -1;
      acc[j] = key[j] >= 0 ? V[k] : 0;
    }
#pragma unroll
    for (int j = 0; j < EV; ++j) {
      ti[j] = key[j] >= 0 ? Tin[key[j]] : 0;
      to[j] = key[j] >= 0 ? Tout[key[j]] : 0;
    }
#pragma unroll
    for (int j = 0; j < EV; ++j) {
      if (key[j] < 0) continue;
      ++pairs;
      GT g;
      if (MODE == 0) {
        const GT dw = (GT)mult * (GT)(acc[j] - wa);
        const GT dd = (GT)ko * (GT)(ti[j] - tia + ki) + (GT)ki * (GT)(to[j] - toa + ko);
        g = (GT)gd * (GT)m * dw - (GT)gn * dd;
      } else {
        const GT dw = (GT)mult * (GT)acc[j];
        const GT dd = (GT)ko * (GT)ti[j] + (GT)ki * (GT)to[j];
        g = (GT)gd * (GT)m * dw - (GT)gn * dd;
      }
      if (g > 0) {
        BestG<GT> c{g, key[j], 1};
        if (better(c, b)) b = c;
      }
    }
  }
}

template <class WT>
__device__ inline void emit_cand(const SweepArgs<WT>& A, int32_t v, int32_t src, const Best& b) {
  const int32_t p = atomicAdd(A.ncand, 1);
  A.cv[p] = v;
  A.csrc[p] = src;
  A.cdst[p] = b.c;
  A.cghi[p] = (int64_t)(b.g >> 64);
  A.cglo[p] = (uint64_t)b.g;
}

template <class WT, class GT>
__device__ inline void emit_cand(const SweepArgs<WT>& A, int32_t v, int32_t src, const BestG<GT>& b) {
  const int32_t p = atomicAdd(A.ncand, 1);
  A.cv[p] = v;
  A.csrc[p] = src;
  A.cdst[p] = b.c;
  A.cghi[p] = (int64_t)((i128)b.g >> 64);
  A.cglo[p] = (uint64_t)b.g;
}

// One group of G lanes per node with a group-private shared hash of
// HG8 slots (G = 8, the lowest degrees) or HG32 slots (G = 32, a warp per
// node).  All groups
// of a warp advance together, so the warp-wide shuffles of the argmax see
// every lane; a group without a node in an iteration only takes part in them.
template <class WT, int MODE, int G, class GT>
__global__ void __launch_bounds__(TPB, 5) k_sweep_group(SweepArgs<WT> A, const int32_t* list, const int32_t* nlist) {
  constexpr int HG = G == 8 ? HG8 : HG32;
  constexpr int GPW = 32 / G;  // groups per warp
  __shared__ int32_t hk[TPB / G][HG];
  __shared__ int64_t hv[TPB / G][HG];
  const int lane = threadIdx.x & 31, gl = threadIdx.x & (G - 1);
  int32_t* K = hk[threadIdx.x / G];
  int64_t* V = hv[threadIdx.x / G];
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const int32_t nl = *nlist;
  const int64_t mult = A.directed ? 1 : 2;
  int64_t scanned = 0, pairs = 0, nodes = 0;
  for (int64_t base = warp * GPW; base < nl; base += ngroups) {
    const int64_t t = base + lane / G;
    const bool act = t < nl;
    const int32_t v = act ? list[t] : 0;
    const int32_t deg = act ? A.out.len[v] + (A.directed ? A.in.len[v] : 0) : 0;
    int H = G;
    while (H < 2 * deg && H < HG) H <<= 1;
    for (int k = gl; k < H; k += G) {
      K[k] = -1;
      V[k] = 0;
    }
    __syncwarp();
    BestG<GT> b{0, 0, 0};
    int32_t a = 0;
    if (act) {
      a = A.lab[v];
      accumulate<WT, MODE>(A, A.out, v, a, K, V, H - 1, gl, G);
      if (A.directed) accumulate<WT, MODE>(A, A.in, v, a, K, V, H - 1, gl, G);
      if (gl == 0) {
        scanned += deg;
        ++nodes;
      }
    }
    __syncwarp();
    if (act) {
      const int64_t wa = MODE == 0 ? hash_get(K, V, H - 1, a) : 0;
      const int64_t ko = A.kout[v], ki = A.kin[v];
      eval_slots<MODE, GT>(K, V, (uint32_t)H, (uint32_t)gl, (uint32_t)G, MODE == 0 ? a : v, a, wa, ko, ki, A.Tout,
                           A.Tin, A.m, A.gn, A.gd, mult, b, pairs);
    }
    b = seg_best<GT, G>(b);
    if (act && gl == 0 && b.have) emit_cand(A, v, MODE == 0 ? a : v, b);
    __syncwarp();
  }
  const int64_t bytes = warp_sum_i64(sweep_bytes<WT, MODE>(A.directed, scanned, nodes, pairs));
  scanned = warp_sum_i64(scanned);
  if (lane == 0 && (scanned | bytes)) {
    atomic_add_i64(A.scanned, scanned);
    atomic_add_i64(&A.stats->sw_entries[G == 32 ? 1 : 0], scanned);
    atomic_add_i64(&A.stats->sw_bytes[G == 32 ? 1 : 0], bytes);
  }
}

// one block per node; the hash lives in dynamic shared memory (mid degrees)
// or in a global-memory slice (hubs, table != nullptr)
// Entries of a node's rows staged in registers: entry k of the node is its
// out-row entry k (k < lo) or its in-row entry k - lo; thread tid holds the
// entries tid + j * NT.  First the neighbour ids and weights ...
template <class WT, int NT, int ACC>
__device__ inline void stage_rows(const SweepArgs<WT>& A, const NodeMeta& m, int32_t (&u)[ACC], int64_t (&w)[ACC]) {
#pragma unroll
  for (int j = 0; j < ACC; ++j) {
    const int32_t k = (int32_t)threadIdx.x + j * NT;
    u[j] = -1;
    w[j] = 0;
    if (k < m.lo) {
      u[j] = A.out.col[m.oo + k];
      w[j] = (int64_t)A.out.w[m.oo + k];
    } else if (k < m.lo + m.li) {
      u[j] = A.in.col[m.oi + (k - m.lo)];
      w[j] = (int64_t)A.in.w[m.oi + (k - m.lo)];
    }
  }
}

// ... then each id becomes its hash key (neighbour label, or for BestRef the
// neighbour's refined community when it shares v's label; -1: skipped).
template <class WT, int MODE, int ACC>
__device__ inline void stage_keys(const SweepArgs<WT>& A, int32_t v, int32_t a, int32_t (&u)[ACC]) {
#pragma unroll
  for (int j = 0; j < ACC; ++j) {
    const int32_t x = u[j];
    int32_t key = -1;
    if (x >= 0 && x != v) {
      const int32_t lx = A.lab[x];
      if (MODE == 0) key = lx;
      else if (lx == a) key = A.par[x];
    }
    u[j] = key;
  }
}

// One block of NT threads per node (a row of up to HMAX/2 entries, hash table
// of up to HMAX slots in shared memory).  Software-pipelined over the block's
// nodes: the row entries and labels of the next node are loaded into
// registers while the current node's table is evaluated, and the node after
// that has its offsets, lengths and strengths loaded one node further ahead,
// so a node's fill only inserts into shared memory.  Entries beyond the
// staged HMAX/2 (not produced by the default bins) are inserted directly.
template <class WT, int MODE, int NT, int HMAX, class GT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_sweep_block(SweepArgs<WT> A, const int32_t* list,
                                                               const int32_t* nlist) {
  extern __shared__ unsigned char smem[];
  __shared__ BestG<GT> wb[NT / 32];
  constexpr int ACC = HMAX / (2 * NT);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int32_t nl = *nlist;
  const int64_t mult = A.directed ? 1 : 2;
  int64_t ent_all = 0, nodes = 0, pairs_all = 0;
  NodeMeta cur{}, nxt{};
  int32_t ek[ACC];
  int64_t ew[ACC];
  if (blockIdx.x < nl) {
    cur = node_meta(A, list[blockIdx.x]);
    stage_rows<WT, NT, ACC>(A, cur, ek, ew);
    stage_keys<WT, MODE, ACC>(A, cur.v, cur.a, ek);
  }
  if (blockIdx.x + gridDim.x < nl) nxt = node_meta(A, list[blockIdx.x + gridDim.x]);
  for (int64_t t = blockIdx.x; t < nl; t += gridDim.x) {
    const int32_t v = cur.v;
    int64_t* V = (int64_t*)smem;
    int32_t* K = (int32_t*)(smem + sizeof(int64_t) * HMAX);
    const int64_t d = (int64_t)cur.lo + cur.li;
    uint32_t H = 256;
    while (H < 2 * d && H < HMAX) H <<= 1;
    for (uint32_t k = threadIdx.x; k < H; k += NT) {
      K[k] = -1;
      V[k] = 0;
    }
    __syncthreads();
    const int32_t a = cur.a;
#pragma unroll
    for (int j = 0; j < ACC; ++j)
      if (ek[j] >= 0) hash_add(K, V, H - 1, ek[j], ew[j]);
    if (d > ACC * NT) {  // entries beyond the staged ones
      for (int64_t k = ACC * NT + threadIdx.x; k < d; k += NT) {
        int32_t x;
        int64_t wx;
        if (k < cur.lo) {
          x = A.out.col[cur.oo + k];
          wx = (int64_t)A.out.w[cur.oo + k];
        } else {
          x = A.in.col[cur.oi + (k - cur.lo)];
          wx = (int64_t)A.in.w[cur.oi + (k - cur.lo)];
        }
        int32_t kx[1] = {x};
        stage_keys<WT, MODE, 1>(A, v, a, kx);
        if (kx[0] >= 0) hash_add(K, V, H - 1, kx[0], wx);
      }
    }
    __syncthreads();
    const bool has_next = t + gridDim.x < nl;
    if (has_next) stage_rows<WT, NT, ACC>(A, nxt, ek, ew);  // in flight during the evaluation
    const int64_t wa = MODE == 0 ? hash_get(K, V, H - 1, a) : 0;
    const int64_t ko = cur.ko, ki = cur.ki;
    BestG<GT> b{0, 0, 0};
    int64_t pairs = 0;
    eval_slots<MODE, GT>(K, V, H, threadIdx.x, NT, MODE == 0 ? a : v, a, wa, ko, ki, A.Tout, A.Tin, A.m, A.gn, A.gd,
                         mult, b, pairs);
    if (has_next) stage_keys<WT, MODE, ACC>(A, nxt.v, nxt.a, ek);  // label gathers overlap the argmax
    b = seg_best<GT, 32>(b);
    if (lane == 0) wb[wid] = b;
    pairs_all += pairs;
    __syncthreads();
    if (threadIdx.x == 0) {
      BestG<GT> r = wb[0];
      for (int w = 1; w < NT / 32; ++w)
        if (better(wb[w], r)) r = wb[w];
      if (r.have) emit_cand(A, v, MODE == 0 ? a : v, r);
      ent_all += d;
      ++nodes;
    }
    __syncthreads();
    cur = nxt;
    if (t + 2 * (int64_t)gridDim.x < nl) nxt = node_meta(A, list[t + 2 * (int64_t)gridDim.x]);
  }
  // statistics once per block
  const int64_t bytes = warp_sum_i64(sweep_bytes<WT, MODE>(A.directed, ent_all, nodes, pairs_all));
  if (lane == 0 && bytes) atomic_add_i64(&A.stats->sw_bytes[NT == 128 ? 2 : 3], bytes);
  if (threadIdx.x == 0 && ent_all) {
    atomic_add_i64(A.scanned, ent_all);
    atomic_add_i64(&A.stats->sw_entries[NT == 128 ? 2 : 3], ent_all);
  }
}

template <class WT>
__global__ void k_bin(Adj<WT> out, Adj<WT> in, int directed, const int32_t* list, const int32_t* nlist,
                      int32_t* bt, int32_t* nt, int32_t* bs, int32_t* ns, int32_t* bm, int32_t* nm, int32_t* bm2,
                      int32_t* nm2, int32_t* bc, int32_t* nc, int32_t* bl, int32_t* nlarge, int64_t* lsz,
                      int64_t* tabtop, int32_t t0, int32_t t1, int32_t t2, int32_t t3,
                      int32_t cluster_max) {
  const int32_t nl = *nlist;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // warp-uniform trip count so that the appends can be warp-aggregated
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < nl; base += stride) {
    const int64_t t = base + (threadIdx.x & 31);
    int bin = -1;
    int32_t v = 0;
    int64_t d = 0;
    if (t < nl) {
      v = list[t];
      d = (int64_t)out.len[v] + (directed ? in.len[v] : 0);
      bin = d <= t0 ? 0 : d <= t1 ? 1 : d <= t2 ? 2 : d <= t3 ? 3 : d <= cluster_max ? 4 : 5;
    }
    warp_append(bin == 0, v, bt, nt);
    warp_append(bin == 1, v, bs, ns);
    warp_append(bin == 2, v, bm, nm);
    warp_append(bin == 3, v, bm2, nm2);
    warp_append(bin == 4, v, bc, nc);
    if (bin == 5) {
      int64_t sz = 1;
      while (sz < 2 * d) sz <<= 1;
      const int32_t p = atomicAdd(nlarge, 1);
      bl[p] = v;
      lsz[p] = sz;
      atomicAdd((unsigned long long*)tabtop, (unsigned long long)sz);
    }
  }
}

// ---------------------------------------------------------------- cluster bin
// One thread-block cluster of CL blocks per node of MID_DEG < degree <=
// CLUSTER_DEG.  The node's hash table of H slots (a power of two >= 2 *
// degree) is spread over the blocks' shared memories: slot h lives in block
// h / (H / CL) at h % (H / CL), and every thread of the cluster inserts into
// it with distributed-shared-memory atomics.  Each block then evaluates its
// own slots, and the blocks' bests meet in block 0.  Every thread of the
// cluster runs every iteration, so the cluster barriers always complete.
template <class WT, int MODE>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(TPB)
    k_sweep_cluster(SweepArgs<WT> A, const int32_t* list, const int32_t* nlist) {
  extern __shared__ unsigned char smem[];
  int64_t* V = (int64_t*)smem;
  int32_t* K = (int32_t*)(smem + sizeof(int64_t) * CL_SLOTS);
  __shared__ Best wb[TPB / 32];
  __shared__ Best cbest[CL];
  __shared__ int64_t s_wa;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t cid = blockIdx.x / CL, ncl = gridDim.x / CL;
  const int32_t nl = *nlist;
  const int64_t mult = A.directed ? 1 : 2;
  int64_t ent_all = 0, nodes = 0, pairs_all = 0;
  for (int64_t t = cid; t < nl; t += ncl) {
    const int32_t v = list[t];
    const int64_t d = (int64_t)A.out.len[v] + (A.directed ? A.in.len[v] : 0);
    uint32_t H = CL * 64;
    while (H < 2 * d && H < (uint32_t)(CL * CL_SLOTS)) H <<= 1;
    const uint32_t HL = H / CL;
    for (uint32_t k = threadIdx.x; k < HL; k += TPB) {
      K[k] = -1;
      V[k] = 0;
    }
    cl.sync();
    const int32_t a = A.lab[v];
    for (int side = 0; side < (A.directed ? 2 : 1); ++side) {
      const Adj<WT>& adj = side ? A.in : A.out;
      const int64_t o = adj.off[v];
      const int32_t l = adj.len[v];
      // warp-uniform trip count: lanes with equal keys find their slot once
      // (one remote compare-and-swap probe by the lowest such lane), then
      // every lane adds its weight with a remote reduction
      for (int32_t base = rank * TPB + wid * 32; base < l; base += CL * TPB) {
        const int32_t k = base + lane;
        int32_t key = -1;
        int64_t w = 0;
        if (k < l) {
          const int32_t u = adj.col[o + k];
          if (u != v && (MODE == 0 || A.lab[u] == a)) {
            key = MODE == 0 ? A.lab[u] : A.par[u];
            w = (int64_t)adj.w[o + k];
          }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(peers) - 1;
        uint32_t h = 0;
        if (key >= 0 && lane == leader) {
          h = hash32((uint32_t)key) & (H - 1);
          while (true) {
            const int32_t prev = atomicCAS(&cl.map_shared_rank(K, (int)(h / HL))[h % HL], -1, key);
            if (prev == -1 || prev == key) break;
            h = (h + 1) & (H - 1);
          }
        }
        h = __shfl_sync(0xffffffffu, h, leader);
        if (key >= 0)
          atomicAdd((unsigned long long*)&cl.map_shared_rank(V, (int)(h / HL))[h % HL], (unsigned long long)w);
      }
    }
    cl.sync();
    if (threadIdx.x == 0) {
      int64_t wa = 0;
      if (MODE == 0) {
        uint32_t h = hash32((uint32_t)a) & (H - 1);
        while (true) {
          const int32_t k = cl.map_shared_rank(K, (int)(h / HL))[h % HL];
          if (k == a) {
            wa = cl.map_shared_rank(V, (int)(h / HL))[h % HL];
            break;
          }
          if (k == -1) break;
          h = (h + 1) & (H - 1);
        }
      }
      s_wa = wa;
    }
    __syncthreads();
    const int64_t wa = s_wa;
    const int64_t ko = A.kout[v], ki = A.kin[v];
    Best b{0, 0, 0};
    for (uint32_t k = threadIdx.x; k < HL; k += TPB) {
      const int32_t key = K[k];
      if (key < 0) continue;
      if (MODE == 0 ? key == a : key == v) continue;
      ++pairs_all;
      const i128 g = gain_of<MODE>(key, V[k], wa, a, ko, ki, A.Tout, A.Tin, A.m, A.gn, A.gd, mult);
      if (g > 0) {
        Best c{g, key, 1};
        if (best_better(c, b)) b = c;
      }
    }
    b = warp_best(b);
    if (lane == 0) wb[wid] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
      Best r = wb[0];
      for (int w = 1; w < TPB / 32; ++w)
        if (best_better(wb[w], r)) r = wb[w];
      cl.map_shared_rank(cbest, 0)[rank] = r;
    }
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) {
      Best r = cbest[0];
      for (int q = 1; q < CL; ++q)
        if (best_better(cbest[q], r)) r = cbest[q];
      if (r.have) emit_cand(A, v, MODE == 0 ? a : v, r);
      ent_all += d;
      ++nodes;
    }
  }
  cl.sync();  // no block leaves while another may still touch its shared memory
  const int64_t bytes = warp_sum_i64(sweep_bytes<WT, MODE>(A.directed, ent_all, nodes, pairs_all));
  if (lane == 0 && bytes) atomic_add_i64(&A.stats->sw_bytes[4], bytes);
  if (threadIdx.x == 0 && ent_all) {
    atomic_add_i64(A.scanned, ent_all);
    atomic_add_i64(&A.stats->sw_entries[4], ent_all);
  }
}

// ---------------------------------------------------------------- hubs
// Hub rows are spread over the whole GPU: one global hash table per hub
// (a power of two >= 2 * degree), filled by chunks of its rows.  A probe that
// claims an empty slot appends it to the hub's slot list (at most degree
// entries, so hub i's list fits at loff[i] / 2), and only the listed slots are
// evaluated, in chunks whose partial bests are reduced per hub, and then
// cleared, so the tables stay clean between sweeps without a full re-fill.
__global__ void k_hub_init(int32_t* K, int64_t* V, int64_t total) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    K[t] = -1;
    V[t] = 0;
  }
}

__global__ void k_eval_counts(const int32_t* hcnt, int32_t nh, int64_t* ecnt) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= nh; i += gridDim.x * blockDim.x)
    ecnt[i] = i < nh ? (hcnt[i] + EVAL_CH - 1) / EVAL_CH : 0;
}

// listed slots back to empty (after the evaluation)
__global__ void k_hub_clear(int32_t nh, const int64_t* loff, const int64_t* epre, const int32_t* hcnt,
                            const int32_t* glist, int32_t* gK, int64_t* gV) {
  const int64_t total = epre[nh];
  for (int64_t e = blockIdx.x; e < total; e += gridDim.x) {
    int64_t lo = 0, hi = nh;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (epre[mid] <= e) lo = mid; else hi = mid;
    }
    const int64_t s0 = (e - epre[lo]) * EVAL_CH, s1 = min((int64_t)hcnt[lo], s0 + EVAL_CH);
    const int32_t* L = glist + loff[lo] / 2;
    for (int64_t j = s0 + threadIdx.x; j < s1; j += blockDim.x) {
      const int64_t slot = loff[lo] + L[j];
      gK[slot] = -1;
      gV[slot] = 0;
    }
  }
}

template <class WT, int MODE>
__global__ void k_hub_acc(SweepArgs<WT> A, ChunkMap m, const int64_t* loff, const int64_t* lsz, int32_t* gK,
                          int64_t* gV, int32_t* glist, int32_t* hcnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = m.pre[m.n_hint];
  int64_t scanned = 0;
  for (int64_t c = warp; c < total; c += nw) {
    const Chunk ch = chunk_of(m, c);
    if (ch.row < 0) continue;
    const int32_t v = ch.v;
    const int32_t cv_ = A.lab[v];
    int32_t* K = gK + loff[ch.idx];
    int64_t* V = gV + loff[ch.idx];
    const uint32_t mask = (uint32_t)lsz[ch.idx] - 1;
    const Adj<WT>& adj = ch.row ? A.in : A.out;
    const int64_t o = adj.off[v];
    for (int32_t base = ch.k0; base < ch.k1; base += 32) {  // warp-uniform
      const int32_t k = base + lane;
      int32_t key = -1;
      int64_t w = 0;
      if (k < ch.k1) {
        const int32_t u = adj.col[o + k];
        if (u != v && (MODE == 0 || A.lab[u] == cv_)) {
          key = MODE == 0 ? A.lab[u] : A.par[u];
          w = (int64_t)adj.w[o + k];
        }
      }
      // lanes with equal keys: one probe by the lowest, then one reduction each
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      const int leader = __ffs(peers) - 1;
      uint32_t h = 0;
      bool fresh = false;
      if (key >= 0 && lane == leader) {
        h = hash32((uint32_t)key) & mask;
        while (true) {
          const int32_t prev = atomicCAS(&K[h], -1, key);
          if (prev == -1 || prev == key) {
            fresh = prev == -1;
            break;
          }
          h = (h + 1) & mask;
        }
      }
      // new keys of the warp (all of one hub) are listed with one counter atomic
      const unsigned fm = __ballot_sync(0xffffffffu, fresh);
      if (fm) {
        int32_t base = 0;
        if (lane == __ffs(fm) - 1) base = atomicAdd(&hcnt[ch.idx], __popc(fm));
        base = __shfl_sync(0xffffffffu, base, __ffs(fm) - 1);
        if (fresh) glist[loff[ch.idx] / 2 + base + __popc(fm & ((1u << lane) - 1u))] = (int32_t)h;
      }
      h = __shfl_sync(0xffffffffu, h, leader);
      if (key >= 0) atomicAdd((unsigned long long*)&V[h], (unsigned long long)w);
    }
    if (lane == 0) scanned += ch.k1 - ch.k0;
  }
  if (lane == 0 && scanned) {
    atomic_add_i64(A.scanned, scanned);
    atomic_add_i64(&A.stats->sw_entries[5], scanned);
    atomic_add_i64(&A.stats->sw_bytes[5], sweep_bytes<WT, MODE>(A.directed, scanned, 0, 0));
  }
}

template <class WT, int MODE>
__global__ void __launch_bounds__(TPB) k_hub_eval(SweepArgs<WT> A, const int32_t* hubs, int32_t nh,
                                                  const int64_t* loff, const int64_t* lsz, const int64_t* epre,
                                                  const int32_t* gK, const int64_t* gV, const int32_t* glist,
                                                  const int32_t* hcnt, int64_t* pb_hi, uint64_t* pb_lo,
                                                  int32_t* pb_c) {
  __shared__ Best wb[TPB / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t mult = A.directed ? 1 : 2;
  const int64_t total = epre[nh];
  for (int64_t e = blockIdx.x; e < total; e += gridDim.x) {
    int64_t lo = 0, hi = nh;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (epre[mid] <= e) lo = mid; else hi = mid;
    }
    const int64_t i = lo;
    const int32_t v = hubs[i];
    const int32_t* K = gK + loff[i];
    const int64_t* V = gV + loff[i];
    const uint32_t H = (uint32_t)lsz[i];
    const int64_t s0 = (e - epre[i]) * EVAL_CH;
    const int64_t s1 = min((int64_t)hcnt[i], s0 + EVAL_CH);
    const int32_t* Lst = glist + loff[i] / 2;
    const int32_t a = A.lab[v];
    const int64_t wa = MODE == 0 ? hash_get(K, V, H - 1, a) : 0;
    const int64_t ko = A.kout[v], ki = A.kin[v];
    Best b{0, 0, 0};
    int64_t pairs = 0;
    for (int64_t j = s0 + threadIdx.x; j < s1; j += TPB) {
      const int32_t slot = Lst[j];
      const int32_t key = K[slot];
      if (MODE == 0 ? key == a : key == v) continue;
      ++pairs;
      const i128 g = gain_of<MODE>(key, V[slot], wa, a, ko, ki, A.Tout, A.Tin, A.m, A.gn, A.gd, mult);
      if (g > 0) {
        Best c{g, key, 1};
        if (best_better(c, b)) b = c;
      }
    }
    b = warp_best(b);
    pairs = warp_sum_i64(pairs);
    if (lane == 0) {
      wb[wid] = b;
      if (pairs) atomic_add_i64(&A.stats->sw_bytes[6], sweep_bytes<WT, MODE>(A.directed, 0, 0, pairs));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      Best r = wb[0];
      for (int w = 1; w < TPB / 32; ++w)
        if (best_better(wb[w], r)) r = wb[w];
      pb_hi[e] = r.have ? (int64_t)(r.g >> 64) : 0;
      pb_lo[e] = r.have ? (uint64_t)r.g : 0;
      pb_c[e] = r.have ? r.c : -1;
    }
    __syncthreads();
  }
}

template <class WT, int MODE>
__global__ void k_hub_final(SweepArgs<WT> A, const int32_t* hubs, int32_t nh, const int64_t* epre,
                            const int64_t* pb_hi, const uint64_t* pb_lo, const int32_t* pb_c) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < nh; i += nw) {
    Best b{0, 0, 0};
    for (int64_t e = epre[i] + lane; e < epre[i + 1]; e += 32) {
      if (pb_c[e] < 0) continue;
      Best c{i128_of(pb_hi[e], pb_lo[e]), pb_c[e], 1};
      if (best_better(c, b)) b = c;
    }
    b = warp_best(b);
    if (lane == 0) {
      const int32_t v = hubs[i];
      atomic_add_i64(&A.stats->sw_bytes[6], sweep_bytes<WT, MODE>(A.directed, 0, 1, 0));
      if (b.have) emit_cand(A, v, MODE == 0 ? A.lab[v] : v, b);
    }
  }
}

// ---------------------------------------------------------------- decouple
// Candidate i precedes j when its gain is larger, or equal with a smaller node.
__device__ inline bool precedes(const int64_t* ghi, const uint64_t* glo, const int32_t* cv, int32_t i, int32_t j) {
  const i128 gi = i128_of(ghi[i], glo[i]), gj = i128_of(ghi[j], glo[j]);
  if (gi != gj) return gi > gj;
  return cv[i] < cv[j];
}

__device__ inline void claim(int32_t* best, int32_t c, int32_t i, const int64_t* ghi, const uint64_t* glo,
                             const int32_t* cv) {
  int32_t cur = best[c];
  while (cur == -1 || precedes(ghi, glo, cv, i, cur)) {
    const int32_t old = atomicCAS(&best[c], cur, i);
    if (old == cur) return;
    cur = old;
  }
}

// A candidate is decided once every earlier candidate touching its source and
// its target is decided: either the community already has a role (set by its
// first accepted candidate, which precedes every undecided one) or this
// candidate is the earliest undecided one touching it.  A round: every
// undecided candidate claims its still role-free communities (CAS keeping the
// earliest), then the decidable ones are decided, then accepted candidates
// give their communities roles (emitter / acceptor) and the claims are reset.

// Whole decoupling filter in one cooperative launch when the candidates are
// many: the three phases of a round, one grid barrier after each, and the
// round counters alternate between two slots (the
// next round's slot is cleared while the current one is still being read).
// Every block reads the same count after the barrier, so all leave together;
// at most nc + 1 rounds (each decides the earliest undecided candidate).
__global__ void __launch_bounds__(TPB) k_dec_grid(int32_t nc, int32_t* cst, const int32_t* cv, const int32_t* src,
                                                  const int32_t* dst, const int64_t* ghi, const uint64_t* glo,
                                                  int32_t* role, int32_t* best, int32_t* bv, int32_t* bsrc,
                                                  int32_t* bdst, int32_t* nb, int32_t* undecided, int32_t* stat) {
  cg::grid_group grid = cg::this_grid();
  const int32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  for (int32_t i = tid; i < nc; i += nth) cst[i] = 0;
  if (tid == 0) undecided[0] = undecided[1] = 0;
  grid.sync();
  int32_t rounds = 0;
  bool ok = true;
  for (;;) {
    const int par = rounds & 1;
    for (int32_t i = tid; i < nc; i += nth) {
      if (cst[i] != 0) continue;
      if (role[src[i]] == 0) claim(best, src[i], i, ghi, glo, cv);
      if (role[dst[i]] == 0) claim(best, dst[i], i, ghi, glo, cv);
    }
    grid.sync();
    int32_t left = 0;
    for (int32_t i = tid; i < nc; i += nth) {
      if (cst[i] != 0) continue;
      const int32_t ra = role[src[i]], rb = role[dst[i]];
      const bool da = ra != 0 || best[src[i]] == i;
      const bool db = rb != 0 || best[dst[i]] == i;
      if (da && db) cst[i] = (ra != 2 && rb != 1) ? 3 : 2;
      else ++left;
    }
    left = warp_sum_i32(left);
    if ((threadIdx.x & 31) == 0 && left) atomicAdd(&undecided[par], left);
    grid.sync();
    for (int32_t i = tid; i < nc; i += nth) {
      best[src[i]] = -1;
      best[dst[i]] = -1;
      if (cst[i] == 3) {
        role[src[i]] = 1;
        role[dst[i]] = 2;
        cst[i] = 1;
      }
    }
    if (tid == 0) undecided[par ^ 1] = 0;
    grid.sync();
    const int32_t l = *(volatile int32_t*)&undecided[par];
    ++rounds;
    if (l == 0) break;
    if (rounds > nc + 1) {
      ok = false;
      break;
    }
  }
  for (int32_t i = tid; i < nc; i += nth) {
    role[src[i]] = 0;
    role[dst[i]] = 0;
    if (cst[i] == 1) {
      const int32_t p = atomicAdd(nb, 1);
      bv[p] = cv[i];
      bsrc[p] = src[i];
      bdst[p] = dst[i];
    }
  }
  if (tid == 0) *stat = ok ? rounds : -1;
}

// Whole decoupling filter in one block when the candidates are few: the
// claim / decide / role phases of every round are separated by block
// barriers, and the loop ends when no candidate is undecided (at most one
// round per candidate, since every round decides the earliest undecided
// one).  *stat receives the number of rounds, or -1 if that bound was hit.
constexpr int DEC_SMALL = 8192;
constexpr int DEC_THREADS = 1024;

constexpr int DEC_PER = DEC_SMALL / DEC_THREADS;  // candidates per thread
static_assert(DEC_PER * DEC_THREADS == DEC_SMALL, "whole candidates per thread");
// the candidates' gains and nodes, staged in shared memory for the claims
constexpr size_t DEC_SMEM = (size_t)DEC_SMALL * (sizeof(int64_t) + sizeof(uint64_t) + sizeof(int32_t));

// The same rounds in one block for up to DEC_SMALL candidates: thread tid
// owns candidates tid + j * DEC_THREADS, whose communities and state stay in
// registers; the gains and nodes that claims compare sit in shared memory.
__global__ void __launch_bounds__(DEC_THREADS) k_dec_block(const int32_t* ncp, const int32_t* cv, const int32_t* src,
                                                           const int32_t* dst, const int64_t* ghi,
                                                           const uint64_t* glo, int32_t* role, int32_t* best,
                                                           int32_t* bv, int32_t* bsrc, int32_t* bdst, int32_t* nb,
                                                           int32_t* stat) {
  extern __shared__ unsigned char dsm[];
  int64_t* sghi = (int64_t*)dsm;
  uint64_t* sglo = (uint64_t*)(dsm + sizeof(int64_t) * DEC_SMALL);
  int32_t* scv = (int32_t*)(dsm + (sizeof(int64_t) + sizeof(uint64_t)) * DEC_SMALL);
  __shared__ int32_t left;
  const int tid = threadIdx.x;
  const int32_t nc = *ncp;
  if (nc > DEC_SMALL) {  // left to the multi-block rounds
    if (tid == 0) *stat = -2;
    return;
  }
  // state per owned candidate: 0 undecided, 1 accepted, 2 rejected, 3 accepted
  // this round (roles pending), 4 no candidate
  int32_t sa[DEC_PER], sb[DEC_PER], st[DEC_PER];
#pragma unroll
  for (int j = 0; j < DEC_PER; ++j) {
    const int32_t i = tid + j * DEC_THREADS;
    const bool have = i < nc;
    st[j] = have ? 0 : 4;
    sa[j] = have ? src[i] : 0;
    sb[j] = have ? dst[i] : 0;
    if (have) {
      sghi[i] = ghi[i];
      sglo[i] = glo[i];
      scv[i] = cv[i];
    }
  }
  __syncthreads();
  int32_t rounds = 0;
  bool ok = true;
  for (;;) {
#pragma unroll
    for (int j = 0; j < DEC_PER; ++j) {
      if (st[j] != 0) continue;
      const int32_t i = tid + j * DEC_THREADS;
      if (role[sa[j]] == 0) claim(best, sa[j], i, sghi, sglo, scv);
      if (role[sb[j]] == 0) claim(best, sb[j], i, sghi, sglo, scv);
    }
    if (tid == 0) left = 0;
    __syncthreads();
    int32_t mine = 0;
#pragma unroll
    for (int j = 0; j < DEC_PER; ++j) {
      if (st[j] != 0) continue;
      const int32_t i = tid + j * DEC_THREADS;
      const int32_t ra = role[sa[j]], rb = role[sb[j]];
      const bool da = ra != 0 || best[sa[j]] == i;
      const bool db = rb != 0 || best[sb[j]] == i;
      if (da && db) st[j] = (ra != 2 && rb != 1) ? 3 : 2;
      else ++mine;
    }
    if (mine) atomicAdd(&left, mine);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < DEC_PER; ++j) {
      if (st[j] == 4) continue;
      best[sa[j]] = -1;
      best[sb[j]] = -1;
      if (st[j] == 3) {
        role[sa[j]] = 1;
        role[sb[j]] = 2;
        st[j] = 1;
      }
    }
    ++rounds;
    __syncthreads();
    const int32_t l = left;
    __syncthreads();  // every thread has read `left` before it is reset
    if (l == 0) break;
    if (rounds > nc + 1) {
      ok = false;
      break;
    }
  }
#pragma unroll
  for (int j = 0; j < DEC_PER; ++j) {
    if (st[j] == 4) continue;
    role[sa[j]] = 0;
    role[sb[j]] = 0;
    if (st[j] == 1) {
      const int32_t p = atomicAdd(nb, 1);
      bv[p] = scv[tid + j * DEC_THREADS];
      bsrc[p] = sa[j];
      bdst[p] = sb[j];
    }
  }
  if (tid == 0) *stat = ok ? rounds : -1;
}

// ---------------------------------------------------------------- commit (move)
__global__ void k_commit_mark(int32_t nb, const int32_t* bv, const int32_t* bsrc, const int32_t* bdst,
                              int32_t* lab, int32_t* oldlab, int32_t* stB, int32_t epB, int32_t* stT, int32_t epT,
                              int32_t* lT, int32_t* nT, int32_t* stCh, int32_t epCh, int32_t* lCh, int32_t* nCh,
                              int32_t* lab_before, int level0) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    const int32_t v = bv[i];
    oldlab[v] = bsrc[i];
    stB[v] = epB;
    if (level0 && stamp_add(stCh, epCh, v, lCh, nCh)) lab_before[v] = bsrc[i];
    lab[v] = bdst[i];
    stamp_add(stT, epT, bsrc[i], lT, nT);
    stamp_add(stT, epT, bdst[i], lT, nT);
  }
}

__global__ void k_snap(const int32_t* lT, const int32_t* nT, const int64_t* Kout, const int64_t* Kin,
                       const int64_t* e, int64_t* sko, int64_t* ski, int64_t* se) {
  const int32_t n = *nT;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int32_t c = lT[k];
    sko[k] = Kout[c];
    ski[k] = Kin[c];
    se[k] = e[c];
  }
}

__global__ void k_commit_K(int32_t nb, const int32_t* bv, const int32_t* bsrc, const int32_t* bdst,
                           const int64_t* kout, const int64_t* kin, int64_t* Kout, int64_t* Kin, int directed) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    const int32_t v = bv[i];
    atomic_add_i64(&Kout[bsrc[i]], -kout[v]);
    atomic_add_i64(&Kout[bdst[i]], kout[v]);
    if (directed) {
      atomic_add_i64(&Kin[bsrc[i]], -kin[v]);
      atomic_add_i64(&Kin[bdst[i]], kin[v]);
    }
  }
}

// Internal-weight repair: every arc with a moved endpoint is counted once
// (from the moved tail's out-row, or from the moved head's in-row when the
// tail did not move).
template <class WT>
__global__ void k_commit_e(Adj<WT> out, Adj<WT> in, ChunkMap m, const int32_t* bsrc, const int32_t* bdst,
                           const int32_t* lab, const int32_t* oldlab, const int32_t* stB, int32_t epB, int64_t* e) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = m.pre[m.n_hint];
  for (int64_t c = warp; c < total; c += nw) {
    const Chunk ch = chunk_of(m, c);
    if (ch.row < 0) continue;
    const int32_t a = bsrc[ch.idx], b = bdst[ch.idx];
    int64_t da = 0, db = 0;
    if (ch.row == 0) {
      const int64_t o = out.off[ch.v];
      for (int32_t k = ch.k0 + lane; k < ch.k1; k += 32) {
        const int32_t u = out.col[o + k];
        const int64_t w = (int64_t)out.w[o + k];
        const bool mu = stB[u] == epB;
        const int32_t cold = mu ? oldlab[u] : lab[u];
        const int32_t cnew = lab[u];
        if (cold == a) da -= w;
        if (cnew == b) db += w;
      }
    } else {
      const int64_t o = in.off[ch.v];
      for (int32_t k = ch.k0 + lane; k < ch.k1; k += 32) {
        const int32_t u = in.col[o + k];
        if (stB[u] == epB) continue;
        const int64_t w = (int64_t)in.w[o + k];
        const int32_t cu = lab[u];
        if (cu == a) da -= w;
        if (cu == b) db += w;
      }
    }
    da = warp_sum_i64(da);
    db = warp_sum_i64(db);
    if (lane == 0) {
      if (da) atomic_add_i64(&e[a], da);
      if (db) atomic_add_i64(&e[b], db);
    }
  }
}

// dQ(B) = sum over touched communities of gd*m*de_C - gn*d(K_out K_in).
__global__ void k_commit_dq(const int32_t* lT, const int32_t* nT, const int64_t* Kout, const int64_t* Kin,
                            const int64_t* e, const int64_t* sko, const int64_t* ski, const int64_t* se, int64_t m,
                            int64_t gn, int64_t gd, DevScalars* sc) {
  const int32_t n = *nT;
  i128 dq = 0, dp = 0;
  int64_t de = 0;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int32_t c = lT[k];
    const int64_t dec = e[c] - se[k];
    const i128 dpc = (i128)Kout[c] * Kin[c] - (i128)sko[k] * ski[k];
    de += dec;
    dp += dpc;
    dq += (i128)gd * m * dec - (i128)gn * dpc;
  }
  dq = warp_sum_i128(dq);
  dp = warp_sum_i128(dp);
  de = warp_sum_i64(de);
  if ((threadIdx.x & 31) == 0) {
    atomic_add_i128(&sc->dq, dq);
    atomic_add_i128(&sc->dp, dp);
    if (de) atomic_add_i64(&sc->de, de);
  }
}

__global__ void k_rollback(int32_t nb, const int32_t* bv, const int32_t* bsrc, int32_t* lab, const int32_t* lT,
                           const int32_t* nT, int64_t* Kout, int64_t* Kin, int64_t* e, const int64_t* sko,
                           const int64_t* ski, const int64_t* se, int directed) {
  const int32_t n = *nT;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) lab[bv[i]] = bsrc[i];
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int32_t c = lT[k];
    Kout[c] = sko[k];
    if (directed) Kin[c] = ski[k];
    e[c] = se[k];
  }
}

__global__ void k_mark_moved(int32_t nb, const int32_t* bv, int32_t* stMv, int32_t epMv, int32_t* lMv, int32_t* nMv,
                             int32_t* stM0, int32_t epM0, int32_t* lM0, int32_t* nM0) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    stamp_add(stMv, epMv, bv[i], lMv, nMv);
    if (stM0) stamp_add(stM0, epM0, bv[i], lM0, nM0);
  }
}

// ---------------------------------------------------------------- refine commit
__global__ void k_commit_ref(int32_t nb, const int32_t* bv, const int32_t* bdst, int32_t* par, const int64_t* kout,
                             const int64_t* kin, int64_t* kout1, int64_t* kin1, int32_t* cnt1, int directed) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    const int32_t v = bv[i], X = bdst[i];
    par[v] = X;
    atomic_add_i64(&kout1[X], kout[v]);
    atomic_add_i64(&kout1[v], -kout[v]);
    if (directed) {
      atomic_add_i64(&kin1[X], kin[v]);
      atomic_add_i64(&kin1[v], -kin[v]);
    }
    atomicAdd(&cnt1[X], 1);
    atomicAdd(&cnt1[v], -1);
  }
}

// SPExpand: dissolved, still-singleton neighbours of moved nodes inside the
// moved node's community.
template <class WT>
__global__ void k_spexpand(Adj<WT> out, Adj<WT> in, ChunkMap m, const int32_t* lab, const int32_t* par,
                           const int32_t* cnt1, const int32_t* stD, int32_t epD, int32_t* stR, int32_t epR,
                           int32_t* lR, int32_t* nR) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = m.pre[m.n_hint];
  for (int64_t c = warp; c < total; c += nw) {
    const Chunk ch = chunk_of(m, c);
    if (ch.row < 0) continue;
    const Adj<WT>& A = ch.row ? in : out;
    const int64_t o = A.off[ch.v];
    const int32_t cv_ = lab[ch.v];
    for (int32_t base = ch.k0; base < ch.k1; base += 32) {
      const int32_t k = base + lane;
      bool want = false;
      int32_t u = 0;
      if (k < ch.k1) {
        u = A.col[o + k];
        want = stD[u] == epD && lab[u] == cv_ && par[u] == u && cnt1[u] == 1 && stamp_claim(stR, epR, u);
      }
      warp_append(want, u, lR, nR);
    }
  }
}

}  // namespace

// ================================================================== host side
static int chunk_grid(int64_t n_hint) { return grid_for(n_hint * 64, TPB, 16); }

void expand_set(ldl_ctx& c, int r, const int32_t* list, int idx_n, int32_t* stamp, int32_t ep, int32_t* olist,
                int idx_out, int64_t n_hint) {
  if (n_hint <= 0) return;
  const int g = chunk_grid(n_hint);
  if (r == 0) {
    Adj<int32_t> o = adj_out0(c), i = adj_in0(c);
    ChunkMap m = chunk_map(c, list, c.dcnt + idx_n, n_hint, o.len, c.directed ? i.len : nullptr);
    k_expand<int32_t><<<g, TPB, 0, c.s>>>(o, i, m, stamp, ep, olist, c.dcnt + idx_out);
  } else {
    Adj<int64_t> o = adj_out(c, r), i = adj_in(c, r);
    ChunkMap m = chunk_map(c, list, c.dcnt + idx_n, n_hint, o.len, c.directed ? i.len : nullptr);
    k_expand<int64_t><<<g, TPB, 0, c.s>>>(o, i, m, stamp, ep, olist, c.dcnt + idx_out);
  }
  CKL("k_expand");
}

void filter_alive(ldl_ctx& c, int r, const int32_t* list, int idx_n, int32_t* olist, int idx_out, int64_t n_hint) {
  k_filter_alive<<<grid_for(n_hint, TPB), TPB, 0, c.s>>>(list, c.dcnt + idx_n, r ? c.lv[r].alive.p : nullptr, olist,
                                                         c.dcnt + idx_out);
  CKL("k_filter_alive");
}

void union_into(ldl_ctx& c, const int32_t* list, int idx_n, int32_t* stamp, int32_t ep, int32_t* olist, int idx_out,
                int64_t n_hint) {
  k_union<<<grid_for(n_hint, TPB), TPB, 0, c.s>>>(list, c.dcnt + idx_n, stamp, ep, olist, c.dcnt + idx_out);
  CKL("k_union");
}

// the next KS_EVENTS statistics events of the context, created on first use
// No exact gain of a sweep, nor any intermediate product of it, reaches 2^62
// when (2 gamma_den + 4 gamma_num) m^2 < 2^62: |w(v,.)| <= m, strengths and
// totals are at most m, so gd*m*|dw| <= 2 gd m^2 and gn*|dd| <= 4 gn m^2.
static bool sweep_gain_fits_i64(const ldl_ctx& c) {
  const i128 m = (i128)c.m;
  const i128 bound = (i128)(2 * (int64_t)c.prm.gamma_den + 4 * (int64_t)c.prm.gamma_num) * m * m;
  return bound < ((i128)1 << 62);
}

// The bins of nodes with at most 2048 entries, in the gain type GT.
template <class WT, int MODE, class GT>
static void sweep_bins(ldl_ctx& c, const SweepArgs<WT>& A, int64_t n_hint, cudaEvent_t* kev) {
  k_sweep_group<WT, MODE, 8, GT><<<grid_for(n_hint * 8, TPB, 5), TPB, 0, c.s>>>(A, c.binT.p, c.dcnt + K_TINY);
  CKL("k_sweep_group<8>");
  if (kev) CK(cudaEventRecord(kev[1], c.s));
  k_sweep_group<WT, MODE, 32, GT><<<grid_for(n_hint * 32, TPB, 5), TPB, 0, c.s>>>(A, c.binS.p, c.dcnt + K_SMALL);
  CKL("k_sweep_group<32>");
  if (kev) CK(cudaEventRecord(kev[2], c.s));
  {
    const size_t sm = (sizeof(int64_t) + sizeof(int32_t)) * 2048;
    k_sweep_block<WT, MODE, 128, 2048, GT><<<grid_for(n_hint, 1, 16), 128, sm, c.s>>>(A, c.binM.p, c.dcnt + K_MID);
    CKL("k_sweep_block(mid1)");
  }
  if (kev) CK(cudaEventRecord(kev[3], c.s));
  {
    const size_t sm = (sizeof(int64_t) + sizeof(int32_t)) * HB;
    CK(cudaFuncSetAttribute(k_sweep_block<WT, MODE, 256, HB, GT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)sm));
    k_sweep_block<WT, MODE, 256, HB, GT><<<grid_for(n_hint, 1, 4), 256, sm, c.s>>>(A, c.binM2.p, c.dcnt + K_MID2);
    CKL("k_sweep_block(mid2)");
  }
}

static cudaEvent_t* kstats_events(ldl_ctx& c) {
  while (c.kev.size() < c.kev_used + KS_EVENTS) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    c.kev.push_back(e);
  }
  cudaEvent_t* e = c.kev.data() + c.kev_used;
  c.kev_used += KS_EVENTS;
  return e;
}

template <class WT, int MODE>
static int32_t sweep_t(ldl_ctx& c, int r, Adj<WT> out, Adj<WT> in, const int32_t* list, int idx_n,
                       int64_t n_hint) {
  LevelState& L = c.lv[r];
  SweepArgs<WT> A;
  A.out = out;
  A.in = in;
  A.directed = c.directed;
  A.lab = L.lab.p;
  A.par = L.par.p;
  A.kout = L.kout.p;
  A.kin = kin_of(c, r);
  if (MODE == 0) {
    A.Tout = c.Kout.p;
    A.Tin = Kin_of(c);
  } else {
    A.Tout = c.lv[r + 1].kout.p;
    A.Tin = kin_of(c, r + 1);
  }
  A.m = c.m;
  A.gn = c.prm.gamma_num;
  A.gd = c.prm.gamma_den;
  A.cv = c.cv.p;
  A.csrc = c.csrc.p;
  A.cdst = c.cdst.p;
  A.cghi = c.cghi.p;
  A.cglo = c.cglo.p;
  A.ncand = c.dcnt + K_CAND;
  A.scanned = &c.d_sc->scanned;
  A.stats = c.d_sc;
  {
    ZeroSpans z;
    z.mask = cnt_bit(K_CAND) | cnt_bit(K_TINY) | cnt_bit(K_SMALL) | cnt_bit(K_MID) | cnt_bit(K_MID2) |
             cnt_bit(K_CLU) | cnt_bit(K_LARGE);
    z.p[0] = &c.d_sc->need;
    z.nw[0] = 1;
    zero_many(c, z);
  }
  k_bin<WT><<<grid_for(n_hint, TPB), TPB, 0, c.s>>>(out, in, c.directed, list, c.dcnt + idx_n, c.binT.p,
                                                     c.dcnt + K_TINY, c.binS.p, c.dcnt + K_SMALL, c.binM.p,
                                                     c.dcnt + K_MID, c.binM2.p, c.dcnt + K_MID2, c.binC.p,
                                                     c.dcnt + K_CLU, c.binL.p, c.dcnt + K_LARGE, c.binLsz.p,
                                                     &c.d_sc->need, c.bin_deg[0], c.bin_deg[1], c.bin_deg[2],
                                                     c.bin_deg[3], std::min(c.prm.cluster_max_deg, CLUSTER_DEG));
  CKL("k_bin");
  // Every bin but the hubs is swept by a grid-stride kernel that reads its
  // bin's count on the device, so these launch before the counts come back
  // and the host's wait below overlaps them.  n_hint bounds every bin.
  cudaEvent_t* kev = c.kstats ? kstats_events(c) : nullptr;
  if (kev) CK(cudaEventRecord(kev[0], c.s));
  if (sweep_gain_fits_i64(c)) sweep_bins<WT, MODE, int64_t>(c, A, n_hint, kev);
  else sweep_bins<WT, MODE, i128>(c, A, n_hint, kev);
  if (kev) CK(cudaEventRecord(kev[4], c.s));
  if (c.prm.cluster_max_deg > c.bin_deg[3]) {
    const size_t sm = (sizeof(int64_t) + sizeof(int32_t)) * CL_SLOTS;
    CK(cudaFuncSetAttribute(k_sweep_cluster<WT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int ncl = (int)std::min<int64_t>(n_hint, std::max(1, device_sms() * 2 / CL));
    k_sweep_cluster<WT, MODE><<<ncl * CL, TPB, sm, c.s>>>(A, c.binC.p, c.dcnt + K_CLU);
    CKL("k_sweep_cluster");
  }
  if (kev) CK(cudaEventRecord(kev[5], c.s));
  // counters K_SMALL .. K_CLU, the hub tables' size and the list's length in one read
  int32_t cn[K_CLU - K_SMALL + 1];
  int64_t tab = 0;
  int32_t nlist = 0;
  {
    const HostRead rr[3] = {{c.dcnt + K_SMALL, cn, (int32_t)sizeof(cn)}, {&c.d_sc->need, &tab, sizeof(int64_t)},
                            {c.dcnt + idx_n, &nlist, sizeof(int32_t)}};
    host_read(c, rr, 3);
  }
  const int32_t ct = cn[K_TINY - K_SMALL], cs = cn[0], cm = cn[K_MID - K_SMALL], cm2 = cn[K_MID2 - K_SMALL];
  const int32_t cc = cn[K_CLU - K_SMALL], ch = cn[K_LARGE - K_SMALL];
  if (kev) CK(cudaEventRecord(kev[6], c.s));  // the wait above is charged to no kernel
  if (ch > 0) {
    // Hub tables hold 2..4 slots per entry.  When all hubs' tables together
    // exceed the slot budget (static builds of the largest graphs), the hubs
    // are swept in consecutive groups whose tables fit, reusing the space.
    std::vector<int32_t> gb{0, ch};
    int64_t tab_use = tab;
    const int64_t budget = g_hub_table_slots.load();
    if (tab > budget) {
      std::vector<int64_t> sz((size_t)ch);
      CK(cudaMemcpyAsync(sz.data(), c.binLsz.p, sizeof(int64_t) * (size_t)ch, cudaMemcpyDeviceToHost, c.s));
      CK(cudaStreamSynchronize(c.s));
      ++c.syncs;
      gb.assign(1, 0);
      int64_t acc = 0;
      tab_use = 0;
      for (int32_t h = 0; h < ch; ++h) {
        if (acc + sz[(size_t)h] > budget && h > gb.back()) {
          gb.push_back(h);
          tab_use = std::max(tab_use, acc);
          acc = 0;
        }
        acc += sz[(size_t)h];
      }
      gb.push_back(ch);
      tab_use = std::max(tab_use, acc);
    }
    c.gkeys.reserve(tab_use, c.s);
    c.gvals.reserve(tab_use, c.s);
    if (c.gtab_clean != c.gkeys.cap || c.gvals.cap != c.gkeys.cap) {  // fresh tables: fill once
      k_hub_init<<<grid_for(c.gkeys.cap, TPB), TPB, 0, c.s>>>(c.gkeys.p, c.gvals.p, c.gkeys.cap);
      CKL("k_hub_init");
      c.gtab_clean = c.gkeys.cap;
    }
    c.glist.reserve(tab_use / 2 + 1, c.s);
    c.hcnt.reserve(ch + 1, c.s);
    // table sizes end with a zero so that each group's offset scan has a total
    CK(cudaMemsetAsync(c.binLsz.p + ch, 0, sizeof(int64_t), c.s));
    c.hub_ecnt.reserve(ch + 2, c.s);
    c.hub_epre.reserve(ch + 2, c.s);
    const int64_t ech = tab_use / 2 / EVAL_CH + ch + 1;  // bounds the evaluation chunks of any group
    c.pb_hi.reserve(ech, c.s);
    c.pb_lo.reserve(ech, c.s);
    c.pb_c.reserve(ech, c.s);
    if (kev) CK(cudaEventRecord(kev[7], c.s));
    for (size_t gi = 0; gi + 1 < gb.size(); ++gi) {
      const int32_t g0 = gb[gi], nh = gb[gi + 1] - g0;
      const int32_t* L = c.binL.p + g0;
      int64_t* Lsz = c.binLsz.p + g0;
      int64_t* Loff = c.binLoff.p + g0;
      const int32_t* cntp = c.dcnt + K_LARGE;
      if (gb.size() > 2) {
        set_cnt(c, K_HUBG, nh);
        cntp = c.dcnt + K_HUBG;
      }
      CK(cudaMemsetAsync(c.hcnt.p, 0, sizeof(int32_t) * (size_t)(nh + 1), c.s));
      // table offsets per hub of the group, in list order
      scan_exclusive(Lsz, Loff, nh + 1, c.P, c.s, false);
      ChunkMap m = chunk_map(c, L, cntp, nh, out.len, c.directed ? in.len : nullptr);
      k_hub_acc<WT, MODE><<<grid_for((int64_t)nh * 2048, TPB, 16), TPB, 0, c.s>>>(
          A, m, Loff, Lsz, c.gkeys.p, c.gvals.p, c.glist.p, c.hcnt.p);
      CKL("k_hub_acc");
      if (kev && gi + 2 == gb.size()) CK(cudaEventRecord(kev[8], c.s));
      // evaluation chunks per hub from its occupied-slot count (device only)
      k_eval_counts<<<grid_for(nh + 1, TPB), TPB, 0, c.s>>>(c.hcnt.p, nh, c.hub_ecnt.p);
      CKL("k_eval_counts");
      scan_exclusive(c.hub_ecnt.p, c.hub_epre.p, nh + 1, c.P, c.s, false);
      const int ge = grid_for(ech, 1, 8);
      k_hub_eval<WT, MODE><<<ge, TPB, 0, c.s>>>(A, L, nh, Loff, Lsz, c.hub_epre.p, c.gkeys.p, c.gvals.p, c.glist.p,
                                                c.hcnt.p, c.pb_hi.p, c.pb_lo.p, c.pb_c.p);
      CKL("k_hub_eval");
      k_hub_final<WT, MODE><<<grid_for((int64_t)nh * 32, TPB), TPB, 0, c.s>>>(A, L, nh, c.hub_epre.p, c.pb_hi.p,
                                                                             c.pb_lo.p, c.pb_c.p);
      CKL("k_hub_final");
      k_hub_clear<<<ge, TPB, 0, c.s>>>(nh, Loff, c.hub_epre.p, c.hcnt.p, c.glist.p, c.gkeys.p, c.gvals.p);
      CKL("k_hub_clear");
    }
  } else if (kev) {
    CK(cudaEventRecord(kev[7], c.s));
    CK(cudaEventRecord(kev[8], c.s));
  }
  if (kev) {
    // times and bytes are resolved when the statistics are read, so that
    // collecting them adds no host synchronisation to the sweep
    CK(cudaEventRecord(kev[9], c.s));
    c.ks_launch[0] += ct > 0;
    c.ks_launch[1] += cs > 0;
    c.ks_launch[2] += cm > 0;
    c.ks_launch[3] += cm2 > 0;
    c.ks_launch[4] += cc > 0;
    c.ks_launch[5] += ch > 0;
    c.ks_launch[6] += ch > 0 ? 3 : 0;  // evaluation, final reduction, clearing
  }
  return nlist;
}

extern "C" void ldl_debug_hub_table_slots(int64_t slots) {
  g_hub_table_slots.store(slots > 0 ? slots : HUB_TABLE_SLOTS);
}

int32_t sweep(ldl_ctx& c, int r, int mode, const int32_t* list, int idx_n, int64_t n_hint) {
  if (r == 0) {
    if (mode == 0) return sweep_t<int32_t, 0>(c, r, adj_out0(c), adj_in0(c), list, idx_n, n_hint);
    return sweep_t<int32_t, 1>(c, r, adj_out0(c), adj_in0(c), list, idx_n, n_hint);
  }
  if (mode == 0) return sweep_t<int64_t, 0>(c, r, adj_out(c, r), adj_in(c, r), list, idx_n, n_hint);
  return sweep_t<int64_t, 1>(c, r, adj_out(c, r), adj_in(c, r), list, idx_n, n_hint);
}

DecoupleOut decouple(ldl_ctx& c, int extra) {
  // The single-block filter runs first and reads the candidate count on the
  // device; one read then returns the count, the accepted number and the
  // filter's status (-2: too many candidates for one block).
  static_assert(K_B == K_CAND + 1 && K_UNDEC == K_CAND + 2, "adjacent counters");
  zero_cnt(c, K_B);
  CK(cudaFuncSetAttribute(k_dec_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DEC_SMEM));
  k_dec_block<<<1, DEC_THREADS, DEC_SMEM, c.s>>>(c.dcnt + K_CAND, c.cv.p, c.csrc.p, c.cdst.p, c.cghi.p, c.cglo.p,
                                                 c.role.p, c.best.p, c.bv.p, c.bsrc.p, c.bdst.p, c.dcnt + K_B,
                                                 c.dcnt + K_UNDEC);
  CKL("k_dec_block");
  int32_t out[3], ex = 0;
  {
    const HostRead rr[2] = {{c.dcnt + K_CAND, out, (int32_t)sizeof(out)},
                            {c.dcnt + (extra >= 0 ? extra : K_CAND), &ex, sizeof(int32_t)}};
    host_read(c, rr, extra >= 0 ? 2 : 1);
  }
  const int32_t nc = out[0];
  if (nc <= 0) return {0, 0, ex};
  if (out[2] != -2) {
    if (out[2] < 0) ldl_throw(LDL_E_INVALID, "internal: decoupling did not converge");
    c.res.decouple_rounds += out[2];
    return {nc, out[1], ex};
  }
  // many candidates: one cooperative launch of co-resident blocks runs all rounds
  int per_sm = 0;
  const int sms = device_sms();
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dec_grid, TPB, 0));
  const int g = std::max(1, std::min(grid_for(nc, TPB), sms * per_sm));
  zero_cnt(c, K_B);
  static_assert(K_TMP2 == K_TMP + 1, "adjacent counters");
  int32_t ncv = nc;
  int32_t* cst = c.cst.p;
  const int32_t *cvp = c.cv.p, *srcp = c.csrc.p, *dstp = c.cdst.p;
  const int64_t* ghi = c.cghi.p;
  const uint64_t* glo = c.cglo.p;
  int32_t *role = c.role.p, *best = c.best.p, *bv = c.bv.p, *bsrc = c.bsrc.p, *bdst = c.bdst.p;
  int32_t* nbp = c.dcnt + K_B;
  int32_t* undec = c.dcnt + K_TMP;  // K_TMP, K_TMP2: the two round counters
  int32_t* stat = c.dcnt + K_UNDEC;
  void* args[] = {&ncv, &cst, &cvp, &srcp, &dstp, &ghi, &glo, &role, &best, &bv, &bsrc, &bdst, &nbp, &undec, &stat};
  CK(cudaLaunchCooperativeKernel((const void*)k_dec_grid, dim3(g), dim3(TPB), args, 0, c.s));
  CKL("k_dec_grid");
  int32_t fin[2];  // K_B, K_UNDEC
  const HostRead rr{c.dcnt + K_B, fin, sizeof(fin)};
  host_read(c, &rr, 1);
  if (fin[1] < 0) ldl_throw(LDL_E_INVALID, "internal: decoupling did not converge");
  c.res.decouple_rounds += fin[1];
  return {nc, fin[0], ex};
}


void commit_move(ldl_ctx& c, int r, int32_t nb, int32_t epB, int32_t epT, int32_t epCh) {
  LevelState& L = c.lv[r];
  const int g = grid_for(nb, TPB);
  {
    // K_T, and the mini-batch's ΔQ numerator, Δ sum K_out K_in and Δ sum e_C
    static_assert(offsetof(DevScalars, dp) == offsetof(DevScalars, dq) + sizeof(I128), "adjacent scalars");
    ZeroSpans z;
    z.mask = cnt_bit(K_T);
    z.p[0] = (int64_t*)&c.d_sc->dq;
    z.nw[0] = (int32_t)(2 * sizeof(I128) / sizeof(int64_t));
    z.p[1] = &c.d_sc->de;
    z.nw[1] = 1;
    zero_many(c, z);
  }
  k_commit_mark<<<g, TPB, 0, c.s>>>(nb, c.bv.p, c.bsrc.p, c.bdst.p, L.lab.p, c.oldlab.p, c.stB.p, epB, c.stT.p, epT,
                                    c.lT.p, c.dcnt + K_T, c.stCh.p, epCh, c.lCh.p, c.dcnt + K_CH, c.lab_before.p,
                                    r == 0);
  CKL("k_commit_mark");
  k_snap<<<grid_for(2 * (int64_t)nb, TPB), TPB, 0, c.s>>>(c.lT.p, c.dcnt + K_T, c.Kout.p, Kin_of(c), c.e.p,
                                                          c.snapKo.p, c.snapKi.p, c.snapE.p);
  CKL("k_snap");
  k_commit_K<<<g, TPB, 0, c.s>>>(nb, c.bv.p, c.bsrc.p, c.bdst.p, L.kout.p, kin_of(c, r), c.Kout.p, Kin_of(c),
                                 c.directed);
  CKL("k_commit_K");
  const int gw = chunk_grid(nb);
  if (r == 0) {
    Adj<int32_t> o = adj_out0(c), i = adj_in0(c);
    ChunkMap m = chunk_map(c, c.bv.p, c.dcnt + K_B, nb, o.len, i.len);
    k_commit_e<int32_t><<<gw, TPB, 0, c.s>>>(o, i, m, c.bsrc.p, c.bdst.p, L.lab.p, c.oldlab.p, c.stB.p, epB, c.e.p);
  } else {
    Adj<int64_t> o = adj_out(c, r), i = adj_in(c, r);
    ChunkMap m = chunk_map(c, c.bv.p, c.dcnt + K_B, nb, o.len, i.len);
    k_commit_e<int64_t><<<gw, TPB, 0, c.s>>>(o, i, m, c.bsrc.p, c.bdst.p, L.lab.p, c.oldlab.p, c.stB.p, epB, c.e.p);
  }
  CKL("k_commit_e");
  k_commit_dq<<<grid_for(2 * (int64_t)nb, TPB), TPB, 0, c.s>>>(c.lT.p, c.dcnt + K_T, c.Kout.p, Kin_of(c), c.e.p,
                                                               c.snapKo.p, c.snapKi.p, c.snapE.p, c.m,
                                                               c.prm.gamma_num, c.prm.gamma_den, c.d_sc);
  CKL("k_commit_dq");
}

CommitOut commit_read(ldl_ctx& c, int extra_idx, int32_t* extra) {
  CommitOut o;
  I128 dq, dp;
  const HostRead rr[5] = {{&c.d_sc->dq, &dq, sizeof(I128)}, {&c.d_sc->dp, &dp, sizeof(I128)},
                          {&c.d_sc->de, &o.de, sizeof(int64_t)}, {c.dcnt + K_T, &o.ntc, sizeof(int32_t)},
                          {c.dcnt + (extra ? extra_idx : K_T), extra, sizeof(int32_t)}};
  host_read(c, rr, extra ? 5 : 4);
  o.dq = i128_of(dq.hi, dq.lo);
  o.dp = i128_of(dp.hi, dp.lo);
  return o;
}

void rollback_move(ldl_ctx& c, int r, int32_t nb, int32_t ntc) {
  LevelState& L = c.lv[r];
  const int64_t m = nb > ntc ? nb : ntc;
  k_rollback<<<grid_for(m, TPB), TPB, 0, c.s>>>(nb, c.bv.p, c.bsrc.p, L.lab.p, c.lT.p, c.dcnt + K_T, c.Kout.p,
                                                Kin_of(c), c.e.p, c.snapKo.p, c.snapKi.p, c.snapE.p, c.directed);
  CKL("k_rollback");
}

void mark_moved(ldl_ctx& c, int r, int32_t nb, int32_t epMv, int32_t epM0) {
  k_mark_moved<<<grid_for(nb, TPB), TPB, 0, c.s>>>(nb, c.bv.p, c.stMv.p, epMv, c.lMv.p, c.dcnt + K_MV,
                                                   r == 0 ? c.stM0.p : nullptr, epM0, c.lM0.p, c.dcnt + K_M0);
  CKL("k_mark_moved");
}

void commit_ref(ldl_ctx& c, int r, int32_t nb) {
  LevelState& L = c.lv[r];
  LevelState& N = c.lv[r + 1];
  k_commit_ref<<<grid_for(nb, TPB), TPB, 0, c.s>>>(nb, c.bv.p, c.bdst.p, L.par.p, L.kout.p, kin_of(c, r), N.kout.p,
                                                   kin_of(c, r + 1), N.cnt.p, c.directed);
  CKL("k_commit_ref");
}

void spexpand(ldl_ctx& c, int r, int32_t nb, int32_t epD, int32_t epR, int32_t* lR, int idx_R) {
  LevelState& L = c.lv[r];
  const int g = chunk_grid(nb);
  if (r == 0) {
    Adj<int32_t> o = adj_out0(c), i = adj_in0(c);
    ChunkMap m = chunk_map(c, c.bv.p, c.dcnt + K_B, nb, o.len, c.directed ? i.len : nullptr);
    k_spexpand<int32_t><<<g, TPB, 0, c.s>>>(o, i, m, L.lab.p, L.par.p, c.lv[r + 1].cnt.p, c.stD.p, epD, c.stR.p,
                                            epR, lR, c.dcnt + idx_R);
  } else {
    Adj<int64_t> o = adj_out(c, r), i = adj_in(c, r);
    ChunkMap m = chunk_map(c, c.bv.p, c.dcnt + K_B, nb, o.len, c.directed ? i.len : nullptr);
    k_spexpand<int64_t><<<g, TPB, 0, c.s>>>(o, i, m, L.lab.p, L.par.p, c.lv[r + 1].cnt.p, c.stD.p, epD, c.stR.p,
                                            epR, lR, c.dcnt + idx_R);
  }
  CKL("k_spexpand");
}
