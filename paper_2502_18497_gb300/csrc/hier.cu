// Hierarchy maintenance of Algorithm 1: batch ingest and validation (the
// batch's application to level 0), statistic repair along the parent chain
// and InitFrontier, label push-down after supernode moves, the refined-community
// split of TouchedRefined, and the Eq. 3 subtract-add aggregate repair with
// NextFrontier.
#include "chunks.cuh"
#include "kern.cuh"

namespace {

constexpr int TPB = 256;

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// ---------------------------------------------------------------- ingest
__device__ inline void set_err(unsigned long long* err, int64_t idx, int code) {
  atomicMin(err, ((unsigned long long)idx << 8) | (unsigned long long)code);
}

__global__ void k_validate(const ldl_update* u, int64_t cnt, int64_t n, unsigned long long* err) {
  GRID_STRIDE(i, cnt) {
    const ldl_update x = u[i];
    int code = 0;
    if (x.src < 0 || x.src >= n || x.dst < 0 || x.dst >= n) code = LDL_E_RANGE;
    else if (x.op != LDL_INSERT && x.op != LDL_DELETE && x.op != LDL_REWEIGHT) code = LDL_E_INVALID;
    else if (x.op == LDL_INSERT && x.w < 1) code = LDL_E_INVALID;
    else if (x.op == LDL_REWEIGHT && x.w < 0) code = LDL_E_NEG_WEIGHT;
    if (code) set_err(err, i, code);
  }
}

__global__ void k_upd_keys(const ldl_update* u, int64_t cnt, int bits, int directed, u64* keys, u64* vals) {
  GRID_STRIDE(i, cnt) {
    int64_t a = u[i].src, b = u[i].dst;
    if (!directed && a > b) {
      int64_t t = a; a = b; b = t;
    }
    keys[i] = ((u64)a << bits) | (u64)b;
    vals[i] = (u64)i;
  }
}

__global__ void k_unique_starts(const u64* keys, int64_t n, const int32_t* flag, const int64_t* pos, u64* ukeys,
                                int64_t* ustart) {
  GRID_STRIDE(i, n) {
    if (flag[i]) {
      ukeys[pos[i]] = keys[i];
      ustart[pos[i]] = i;
    }
  }
}

// Per edge key: apply its updates in array order to the current weight.
__global__ void k_seq(const ldl_update* u, int64_t cnt, const u64* vals, const int64_t* ustart, int64_t nu,
                      const u64* ukeys, const int64_t* oldw, int bits, int directed, int64_t* delta,
                      unsigned long long* err, int64_t* dm) {
  GRID_STRIDE(k, nu) {
    const int64_t s = ustart[k], e = (k + 1 < nu) ? ustart[k + 1] : cnt;
    const int64_t w0 = oldw[k];
    int64_t cur = w0;
    for (int64_t t = s; t < e; ++t) {
      const int64_t idx = (int64_t)vals[t];
      const ldl_update x = u[idx];
      int bad = 0;
      if (x.op == LDL_INSERT) {
        cur += x.w;
        if (cur > INT32_MAX) bad = LDL_E_OVERFLOW;
      } else if (x.op == LDL_DELETE) {
        if (cur == 0) bad = LDL_E_NO_EDGE;
        cur = 0;
      } else {
        if (cur == 0) bad = LDL_E_NO_EDGE;
        cur = x.w;
      }
      if (bad) {
        set_err(err, idx, bad);
        cur = w0;
        break;
      }
    }
    const int64_t d = cur - w0;
    delta[k] = d;
    if (d) {
      const u64 key = ukeys[k];
      const int64_t a = (int64_t)(key >> bits), b = (int64_t)(key & ((((u64)1) << bits) - 1));
      atomic_add_i64(dm, (directed || a == b) ? d : 2 * d);
    }
  }
}

__global__ void k_emit_arcs(const u64* ukeys, const int64_t* delta, int64_t nu, int bits, int directed, u64* ok,
                            u64* ov, int32_t* cnt) {
  GRID_STRIDE(k, nu) {
    const int64_t d = delta[k];
    if (!d) continue;
    const u64 key = ukeys[k];
    const u64 a = key >> bits, b = key & ((((u64)1) << bits) - 1);
    int32_t p = atomicAdd(cnt, 1);
    ok[p] = key;
    ov[p] = (u64)d;
    if (!directed && a != b) {
      p = atomicAdd(cnt, 1);
      ok[p] = (b << bits) | a;
      ov[p] = (u64)d;
    }
  }
}

// (row, col) -> (col + row_off, row): the in-direction records of a level
// whose in-rows live at row_off (directed graphs keep both in one CSR).
__global__ void k_transpose(const u64* k, const u64* v, int64_t n, int bits, u64* ok, u64* ov, int64_t row_off) {
  const u64 mask = (((u64)1) << bits) - 1;
  GRID_STRIDE(i, n) {
    ok[i] = (((k[i] & mask) + (u64)row_off) << bits) | (k[i] >> bits);
    ov[i] = v[i];
  }
}

// ---------------------------------------------------------------- repair
__global__ void k_dirty(const u64* keys, int64_t na, int bits, const int32_t* lab, int32_t* stT, int32_t epT,
                        int32_t* lT, int32_t* nT) {
  const u64 mask = (((u64)1) << bits) - 1;
  GRID_STRIDE(i, na) {
    stamp_add(stT, epT, lab[keys[i] >> bits], lT, nT);
    stamp_add(stT, epT, lab[keys[i] & mask], lT, nT);
  }
}

// sum over listed communities of K_out * K_in into an int128 accumulator
__global__ void k_psum(const int32_t* list, const int32_t* nlist, const int64_t* Kout, const int64_t* Kin,
                       I128* acc) {
  const int32_t n = *nlist;
  i128 s = 0;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int32_t c = list[k];
    s += (i128)Kout[c] * Kin[c];
  }
  s = warp_sum_i128(s);
  if ((threadIdx.x & 31) == 0) atomic_add_i128(acc, s);
}

__global__ void k_stat_arcs(const u64* keys, const int64_t* delta, int64_t na, int bits, int directed,
                            const int32_t* lab, int64_t* kout, int64_t* kin, int64_t* Kout, int64_t* Kin, int64_t* e,
                            int64_t* de, int32_t* stA, int32_t epA, int32_t* lA, int32_t* nA) {
  const u64 mask = (((u64)1) << bits) - 1;
  int64_t sde = 0;
  GRID_STRIDE(t, na) {
    const int32_t i = (int32_t)(keys[t] >> bits), j = (int32_t)(keys[t] & mask);
    const int64_t d = delta[t];
    atomic_add_i64(&kout[i], d);
    if (directed) atomic_add_i64(&kin[j], d);
    const int32_t ci = lab[i], cj = lab[j];
    atomic_add_i64(&Kout[ci], d);
    if (directed) atomic_add_i64(&Kin[cj], d);
    if (ci == cj) {
      atomic_add_i64(&e[ci], d);
      sde += d;
    }
    stamp_add(stA, epA, i, lA, nA);
    stamp_add(stA, epA, j, lA, nA);
  }
  if (sde) atomic_add_i64(de, sde);
}

// Per-level pointers for walks up the parent chain (levels 0..7).
struct Chain {
  const int32_t* par[8];  // pi_q
  int64_t* kout[8];
  int64_t* kin[8];
  u64* pk[8];             // pending weight records of level q
  u64* pv[8];
  int32_t* stA[8];        // frontier A^q: stamp, epoch, list
  int32_t epA[8];
  int32_t* lA[8];
};

// Weight records (keys, vals) of level q0 carried up the hierarchy: with
// `self` a record joins level q0's pending list; mapped through pi_q0,
// pi_q0+1, ... it joins the pending list of every level above up to `top`,
// until an endpoint has no parent (W_{q+1}(pi(i), pi(j)) takes the weight of
// every level-q arc (i, j)).  With `add_k` the strengths of those levels take
// the weight as well.  Records are not reduced here: the pending list of a
// level is sorted, summed and applied when the level is next read.
// Warp-aggregated append of one record per lane that wants one (every lane
// of the warp calls it together): one atomic per warp.
__device__ inline void warp_append_rec(bool want, u64 key, int64_t v, u64* pk, u64* pv, int32_t* count) {
  const unsigned m = __ballot_sync(0xffffffffu, want);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  int32_t base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (want) {
    const int32_t p = base + __popc(m & ((1u << lane) - 1u));
    pk[p] = key;
    pv[p] = (u64)v;
  }
}

__global__ void k_chain_records(const u64* keys, const int64_t* vals, int64_t n, int bits, int q0, int top, int self,
                                int add_k, int directed, Chain ch, int32_t* pcnt) {
  const u64 mask = (((u64)1) << bits) - 1;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // warp-uniform trip counts, so that appends aggregate over the warp
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; base < n; base += stride) {
    const int64_t t = base + lane;
    bool on = t < n;
    u64 key = 0;
    int64_t d = 0;
    if (on) {
      key = keys[t];
      d = vals[t];
    }
    int32_t x = (int32_t)(key >> bits), y = (int32_t)(key & mask);
    if (self) warp_append_rec(on, key, d, ch.pk[q0], ch.pv[q0], &pcnt[q0]);
    for (int q = q0; q < top; ++q) {
      if (on) {
        x = ch.par[q][x];
        y = ch.par[q][y];
        on = x >= 0 && y >= 0;
      }
      if (!__any_sync(0xffffffffu, on)) break;
      if (on && add_k) {
        atomic_add_i64(&ch.kout[q + 1][x], d);
        if (directed) atomic_add_i64(&ch.kin[q + 1][y], d);
      }
      warp_append_rec(on, ((u64)x << bits) | (u64)(uint32_t)y, d, ch.pk[q + 1], ch.pv[q + 1], &pcnt[q + 1]);
    }
  }
}

// InitFrontier above level 0: A^{q+1} = pi_q(A^q) for every q < top, by
// walking each node of A^0 up its parent chain.  A walk stops at a node that
// is already marked: the walk that marked it goes on above it.
__global__ void k_chain_frontier(const int32_t* l0, const int32_t* n0, int top, Chain ch, int32_t* nA) {
  const int32_t m = *n0;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    int32_t x = l0[k];
    for (int q = 0; q < top; ++q) {
      x = ch.par[q][x];
      if (x < 0 || !stamp_add(ch.stA[q + 1], ch.epA[q + 1], x, ch.lA[q + 1], &nA[q + 1])) break;
    }
  }
}

// ---------------------------------------------------------------- push-down
// Children of each listed level-(q+1) node take its label at level q.
__global__ void k_push(ChunkMap m, const int32_t* lab_up, Adj<int32_t> ch_adj, const int32_t* par, int32_t* lab,
                       int32_t* olist, int32_t* nout, int32_t* stCh, int32_t epCh, int32_t* lCh, int32_t* nCh,
                       int32_t* lab_before) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = m.pre[m.n_hint];
  for (int64_t c = warp; c < total; c += nw) {
    const Chunk ch = chunk_of(m, c);
    if (ch.row < 0) continue;
    const int32_t L = lab_up[ch.v];
    const int64_t o = ch_adj.off[ch.v];
    for (int32_t base = ch.k0; base < ch.k1; base += 32) {
      const int32_t k = base + lane;
      int32_t u = k < ch.k1 ? ch_adj.col[o + k] : 0;
      const bool valid = k < ch.k1 && par[u] == ch.v;  // a listed node that left (emptied) is skipped
      bool first = false;
      if (valid) {
        if (stCh) {
          first = stamp_claim(stCh, epCh, u);
          if (first) lab_before[u] = lab[u];
        }
        lab[u] = L;
      }
      if (stCh) warp_append(first, u, lCh, nCh);
      if (olist) warp_append(valid, u, olist, nout);
    }
  }
}

// ---------------------------------------------------------------- dissolve
__global__ void k_stamp_list(const int32_t* l, const int32_t* n, int32_t* st, int32_t ep) {
  const int32_t m = *n;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) st[l[k]] = ep;
}

__global__ void k_dissolve(const int32_t* lD, const int32_t* nD, int32_t* par, int32_t* par_old,
                           const int64_t* kout, const int64_t* kin, int64_t* kout1, int64_t* kin1, int32_t* cnt1,
                           int directed) {
  const int32_t n = *nD;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int32_t u = lD[k];
    const int32_t p = par[u];
    par_old[u] = p;
    if (p >= 0) {
      atomic_add_i64(&kout1[p], -kout[u]);
      if (directed) atomic_add_i64(&kin1[p], -kin[u]);
      atomicAdd(&cnt1[p], -1);
    }
    par[u] = u;
    atomic_add_i64(&kout1[u], kout[u]);
    if (directed) atomic_add_i64(&kin1[u], kin[u]);
    atomicAdd(&cnt1[u], 1);
  }
}

__global__ void k_reset_par(const int32_t* lD, int32_t nD, int32_t* par, int64_t* kout1, int64_t* kin1,
                            int32_t* cnt1, int directed) {
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nD; k += gridDim.x * blockDim.x) {
    const int32_t u = lD[k];
    par[u] = -1;
    kout1[u] = 0;
    if (directed) kin1[u] = 0;
    cnt1[u] = 0;
  }
}

// ---------------------------------------------------------------- split
// TouchedRefined of a batch update (see split()).  The refined communities
// holding an endpoint of a deleted level-r arc are re-checked (before any
// node leaves, so with their current parents).
__global__ void k_brk_check(const int32_t* lK, const int32_t* nK, const uint8_t* alive, const int32_t* par,
                            int32_t* stX, int32_t epX, int32_t* lX, int32_t* nX, int32_t* ckf, int32_t epF) {
  const int32_t n = *nK;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int32_t z = lK[k];
    if (alive[z] && par[z] >= 0) {
      stamp_add(stX, epX, par[z], lX, nX);
      ckf[par[z]] = epF;  // an arc inside it may be gone: its components are computed
    }
  }
}

// A node of U* whose label differs from its refined community's label (or
// that has no refined community) leaves it as a singleton named by its own
// id; its old refined community is re-checked.
__global__ void k_leave(const int32_t* lU, const int32_t* nU, const uint8_t* alive, const int32_t* lab,
                        const int32_t* labN, int32_t* par, int32_t* par_old, const int64_t* kout, const int64_t* kin,
                        int64_t* kout1, int64_t* kin1, int32_t* cnt1, int directed, int32_t* stL, int32_t epL,
                        int32_t* stD, int32_t epD, int32_t* lD, int32_t* nD, int32_t* stX, int32_t epX, int32_t* lX,
                        int32_t* nX, int32_t* nbr) {
  const int32_t n = *nU;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int32_t u = lU[k];
    if (!alive[u]) continue;
    const int32_t X = par[u];
    if (X >= 0 && labN[X] == lab[u]) continue;
    stL[u] = epL;
    par_old[u] = X;
    nbr[u] = 0;
    if (X >= 0) {
      stamp_add(stX, epX, X, lX, nX);
      atomic_add_i64(&kout1[X], -kout[u]);
      if (directed) atomic_add_i64(&kin1[X], -kin[u]);
      atomicAdd(&cnt1[X], -1);
    }
    par[u] = u;
    atomic_add_i64(&kout1[u], kout[u]);
    if (directed) atomic_add_i64(&kin1[u], kin[u]);
    atomicAdd(&cnt1[u], 1);
    stamp_add(stD, epD, u, lD, nD);
  }
}

// A refined community that lost nodes stays connected when every node that
// left had at most one neighbour in it and no arc inside it was deleted
// (removing leaves keeps a connected graph connected).  Counts each leaving
// node's neighbours in its old refined community (an arc seen from both
// rows of a directed pair counts twice: the test only errs towards a check)
// and flags the community for a connectivity check at the second one.
template <class WT>
__global__ void k_leave_degree(Adj<WT> out, Adj<WT> in, ChunkMap m, const int32_t* par, const int32_t* par_old,
                               const int32_t* stL, int32_t epL, int32_t* nbr, int32_t* ckf, int32_t epF) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = m.pre[m.n_hint];
  for (int64_t c = warp; c < total; c += nw) {
    const Chunk ch = chunk_of(m, c);
    if (ch.row < 0) continue;
    const int32_t v = ch.v;
    const int32_t X = par_old[v];
    if (X < 0 || stL[v] != epL) continue;
    const Adj<WT>& A = ch.row ? in : out;
    const int64_t o = A.off[v];
    for (int32_t k = ch.k0 + lane; k < ch.k1; k += 32) {
      const int32_t y = A.col[o + k];
      if (y == v) continue;
      const bool inX = stL[y] == epL ? par_old[y] == X : par[y] == X;
      if (inX && atomicAdd(&nbr[v], 1) == 1) ckf[X] = epF;
    }
  }
}

// Remaining members of the re-checked refined communities whose connectivity
// is in doubt (flagged, or their seed node left); each starts as its own
// component.
__global__ void k_members(Adj<int32_t> ch_adj, ChunkMap m, const int32_t* par, const int32_t* stL, int32_t epL,
                          const int32_t* ckf, int32_t epF, int32_t* comp, int32_t* lG, int32_t* nG) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = m.pre[m.n_hint];
  for (int64_t c = warp; c < total; c += nw) {
    const Chunk ch = chunk_of(m, c);
    if (ch.row < 0) continue;
    const int32_t X = ch.v;
    if (ckf[X] != epF && stL[X] != epL) continue;
    const int64_t o = ch_adj.off[X];
    for (int32_t base = ch.k0; base < ch.k1; base += 32) {
      const int32_t k = base + lane;
      bool want = false;
      int32_t u = 0;
      if (k < ch.k1) {
        u = ch_adj.col[o + k];
        want = stL[u] != epL && par[u] == X;  // listed nodes that emptied or left are skipped
        if (want) comp[u] = u;
      }
      warp_append(want, u, lG, nG);
    }
  }
}

// Root of x's tree.  Parent links only point to smaller ids of the same
// component and a root never becomes a root again, so reads that lag behind
// other threads still lead to a node of x's component; they bypass L1 so that
// a thread sees links other SMs made.  With `halve`, x's link is shortened to
// its grandparent on the way (only a non-root's link is ever written, and
// compare-and-swap hooks only roots, so the two never collide).
__device__ inline int32_t uf_find(int32_t* comp, int32_t x, bool halve) {
  int32_t p = __ldcg(&comp[x]);
  while (p != x) {
    const int32_t q = __ldcg(&comp[p]);
    if (halve && q != p) comp[x] = q;
    x = p;
    p = q;
  }
  return x;
}

// Joins the trees of u and y: always hooks the larger root under the smaller
// one (a compare-and-swap that fails because another thread hooked first is
// retried), so every component ends rooted at its lowest member.
__device__ inline void uf_union(int32_t* comp, int32_t u, int32_t y) {
  for (;;) {
    const int32_t a = uf_find(comp, u, true), b = uf_find(comp, y, true);
    if (a == b) return;
    const int32_t hi = a > b ? a : b, lo = a > b ? b : a;
    if (atomicCAS(&comp[hi], hi, lo) == hi) return;
  }
}

// Connected components of the collected members over the arcs between two
// remaining members of the same refined community, by a lock-free union-find
// with neighbour sampling (the Afforest scheme of Sutton, Ben-Nun and Barak,
// IPDPS 2018).  First every member is joined along at most UF_SAMPLE of the
// qualifying arcs among the first 32 entries of its rows (k_uf_sample); in a
// community that is still connected this already puts most members into the
// seed node's tree.  Then k_uf walks all arcs of the members that are not (yet)
// in their community seed's tree.  The components are exact: every arc with an
// endpoint outside the seed's tree is joined from that endpoint's side (both
// rows of a member are walked, so the arc is seen from either end), and an arc
// whose two endpoints were both in the seed's tree when they were checked
// joins nothing new, because trees only ever merge.
constexpr int UF_SAMPLE = 2;

template <class WT>
__global__ void k_uf_sample(Adj<WT> out, Adj<WT> in, int directed, const int32_t* lG, const int32_t* nG,
                            const int32_t* par, const int32_t* stL, int32_t epL, int32_t* comp) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int32_t n = *nG;
  for (int64_t t = warp; t < n; t += nw) {
    const int32_t u = lG[t];
    const int32_t X = par[u];
    int taken = 0;  // warp-uniform
    for (int side = 0; side < (directed ? 2 : 1) && taken < UF_SAMPLE; ++side) {
      const Adj<WT>& A = side ? in : out;
      const int32_t l = A.len[u];
      bool q = false;
      int32_t y = 0;
      if (lane < l) {
        y = A.col[A.off[u] + lane];
        q = y != u && par[y] == X && stL[y] != epL;
      }
      const unsigned mask = __ballot_sync(0xffffffffu, q);
      const int before = __popc(mask & ((1u << lane) - 1u));
      if (q && before < UF_SAMPLE - taken) uf_union(comp, u, y);
      taken += min(__popc(mask), UF_SAMPLE - taken);
    }
  }
}

template <class WT>
__global__ void k_uf(Adj<WT> out, Adj<WT> in, ChunkMap m, const int32_t* par, const uint8_t* alive,
                     const int32_t* stL, int32_t epL, int32_t* comp) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = m.pre[m.n_hint];
  for (int64_t c = warp; c < total; c += nw) {
    const Chunk ch = chunk_of(m, c);
    if (ch.row < 0) continue;
    const int32_t u = ch.v;
    const int32_t X = par[u];
    // the community's seed node X is a member when it is alive, stays and is
    // its own parent (then the members gathering set its tree)
    const bool seed = alive[X] && stL[X] != epL && par[X] == X;
    if (seed && uf_find(comp, u, true) == uf_find(comp, X, true)) continue;
    const Adj<WT>& A = ch.row ? in : out;
    const int64_t o = A.off[u];
    for (int32_t k = ch.k0 + lane; k < ch.k1; k += 32) {
      const int32_t y = A.col[o + k];
      if (y == u || par[y] != X || stL[y] == epL) continue;
      uf_union(comp, u, y);
    }
  }
}

// Every member's label becomes its component's root (its lowest member).
// The find here writes nothing but the member's own label: a shortening
// write could otherwise replace another member's final root by an ancestor
// read before that root was written.  Every own write is a node of the same
// component (the root, or before it an ancestor), so other threads' finds
// still end at the root.
__global__ void k_uf_final(const int32_t* lG, const int32_t* nG, int32_t* comp) {
  const int32_t n = *nG;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int32_t u = lG[k];
    comp[u] = uf_find(comp, u, false);
  }
}

// A component keeps its refined community's id when it holds the community's
// seed node (the node with that id, still a member); any other component is
// renamed after its lowest member.
__global__ void k_rename(const int32_t* lG, const int32_t* nG, const int32_t* comp, const uint8_t* alive,
                         const int32_t* stL, int32_t epL, int32_t* par, int32_t* par_old, const int64_t* kout,
                         const int64_t* kin, int64_t* kout1, int64_t* kin1, int32_t* cnt1, int directed,
                         int32_t* stD, int32_t epD, int32_t* lD, int32_t* nD) {
  const int32_t n = *nG;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int32_t u = lG[k];
    const int32_t X = par[u];
    const int32_t root = comp[u];
    const bool keep = alive[X] && stL[X] != epL && par[X] == X && comp[X] == root;
    if (keep) continue;
    par_old[u] = X;
    par[u] = root;
    atomic_add_i64(&kout1[X], -kout[u]);
    if (directed) atomic_add_i64(&kin1[X], -kin[u]);
    atomicAdd(&cnt1[X], -1);
    atomic_add_i64(&kout1[root], kout[u]);
    if (directed) atomic_add_i64(&kin1[root], kin[u]);
    atomicAdd(&cnt1[root], 1);
    stamp_add(stD, epD, u, lD, nD);
  }
}

// the listed nodes that are singleton refined communities
__global__ void k_singletons(const int32_t* l, const int32_t* n, const int32_t* par, const int32_t* cnt1, int32_t* out,
                             int32_t* nout) {
  const int32_t m = *n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < m; base += stride) {
    const int64_t k = base + (threadIdx.x & 31);
    int32_t u = 0;
    bool want = false;
    if (k < m) {
      u = l[k];
      want = par[u] == u && cnt1[u] == 1;
    }
    warp_append(want, u, out, nout);
  }
}

// ---------------------------------------------------------------- aggregate
__global__ void k_changed(const int32_t* lD, const int32_t* nD, const int32_t* par, const int32_t* par_old,
                          int32_t* stC, int32_t epC, int32_t* lC, int32_t* nC) {
  const int32_t n = *nD;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int32_t u = lD[k];
    if (par[u] != par_old[u]) stamp_add(stC, epC, u, lC, nC);
  }
}

template <class WT>
__global__ void k_deg_sum(Adj<WT> out, Adj<WT> in, const int32_t* l, const int32_t* n, int64_t* acc_out,
                          int64_t* acc_in) {
  const int32_t m = *n;
  int64_t so = 0, si = 0;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    so += (int64_t)out.len[l[k]];
    si += (int64_t)in.len[l[k]];
  }
  so = warp_sum_i64(so);
  si = warp_sum_i64(si);
  if ((threadIdx.x & 31) == 0 && so) atomic_add_i64(acc_out, so);
  if ((threadIdx.x & 31) == 0 && si) atomic_add_i64(acc_in, si);
}

// Subtract-add records of Eq. 3 for every arc incident to a changed node,
// each arc counted once (from its changed tail's out-row, or from its changed
// head's in-row when the tail is unchanged).
template <class WT>
__global__ void k_emit(Adj<WT> out, Adj<WT> in, ChunkMap m, const int32_t* par, const int32_t* par_old,
                       const int32_t* stC, int32_t epC, int bits, u64* rk, u64* rv, int32_t* cnt, int64_t cap,
                       int32_t* err) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = m.pre[m.n_hint];
  for (int64_t c = warp; c < total; c += nw) {
    const Chunk ch = chunk_of(m, c);
    if (ch.row < 0) continue;
    const int32_t u = ch.v;
    const int32_t po = par_old[u], pn = par[u];
    const Adj<WT>& A = ch.row ? in : out;
    const int64_t o = A.off[u];
    // 64 entries per step, up to four records per lane, one counter atomic
    // per warp and step
    for (int32_t base = ch.k0; base < ch.k1; base += 64) {
      u64 rkey[4] = {0, 0, 0, 0}, rval[4] = {0, 0, 0, 0};
      bool ok[4] = {false, false, false, false};  // fixed slots: (first entry -, +), (second entry -, +)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int32_t k = base + h * 32 + lane;
        if (k >= ch.k1) continue;
        const int32_t v = A.col[o + k];
        const int64_t w = (int64_t)A.w[o + k];
        const bool vc = stC[v] == epC;
        if (ch.row == 0) {  // arc (u, v) from u's out-row
          const int32_t pvo = vc ? par_old[v] : par[v];
          const int32_t pvn = par[v];
          ok[2 * h] = po >= 0 && pvo >= 0;
          rkey[2 * h] = ((u64)po << bits) | (u64)pvo;
          rval[2 * h] = (u64)(-w);
          ok[2 * h + 1] = true;
          rkey[2 * h + 1] = ((u64)pn << bits) | (u64)pvn;
          rval[2 * h + 1] = (u64)w;
        } else if (!vc) {  // arc (v, u) from u's in-row, v unchanged
          const int32_t pv = par[v];
          ok[2 * h] = po >= 0;
          rkey[2 * h] = ((u64)pv << bits) | (u64)po;
          rval[2 * h] = (u64)(-w);
          ok[2 * h + 1] = true;
          rkey[2 * h + 1] = ((u64)pv << bits) | (u64)pn;
          rval[2 * h + 1] = (u64)w;
        }
      }
      const int nrec = (int)ok[0] + (int)ok[1] + (int)ok[2] + (int)ok[3];
      int incl = nrec;  // warp inclusive scan of the per-lane counts
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
      }
      const int wtot = __shfl_sync(0xffffffffu, incl, 31);
      int32_t wbase = 0;
      if (lane == 31 && wtot) wbase = atomicAdd(cnt, wtot);
      wbase = __shfl_sync(0xffffffffu, wbase, 31);
      int64_t p = (int64_t)wbase + incl - nrec;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (ok[j]) {
          if (p < cap) {
            rk[p] = rkey[j];
            rv[p] = rval[j];
          } else {
            atomicExch(err, 3);  // the record bound was wrong: reported, nothing written past it
          }
          ++p;
        }
    }
  }
}

// Node records (strength moves between parents) and children-list records.
__global__ void k_emit_nodes(const int32_t* lC, const int32_t* nC, const int32_t* par, const int32_t* par_old,
                             const int64_t* kout, const int64_t* kin, int bits, int32_t* ndx, int64_t* ndko,
                             int64_t* ndki, int32_t* nnd, u64* ck, u64* cv, int32_t* ncr) {
  const int32_t n = *nC;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int32_t u = lC[k];
    const int32_t po = par_old[u], pn = par[u];
    if (ndx) {
      if (po >= 0) {
        const int32_t p = atomicAdd(nnd, 1);
        ndx[p] = po;
        ndko[p] = -kout[u];
        ndki[p] = -kin[u];
      }
      const int32_t p = atomicAdd(nnd, 1);
      ndx[p] = pn;
      ndko[p] = kout[u];
      ndki[p] = kin[u];
    }
    if (po >= 0) {
      const int32_t p = atomicAdd(ncr, 1);
      ck[p] = ((u64)po << bits) | (u64)u;
      cv[p] = (u64)(int64_t)-1;
    }
    const int32_t p = atomicAdd(ncr, 1);
    ck[p] = ((u64)pn << bits) | (u64)u;
    cv[p] = (u64)(int64_t)1;
  }
}

// Strength moves (node, out delta, in delta) of level-q0 nodes carried to
// every ancestor level up to `top` (the strengths of a supernode are the sums
// of its members').
__global__ void k_chain_nodes(const int32_t* ndx, const int64_t* ndko, const int64_t* ndki, const int32_t* n,
                              int q0, int top, int directed, Chain ch) {
  const int32_t m = *n;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    int32_t x = ndx[k];
    const int64_t ko = ndko[k], ki = ndki[k];
    for (int q = q0; q < top; ++q) {
      x = ch.par[q][x];
      if (x < 0) break;
      atomic_add_i64(&ch.kout[q + 1][x], ko);
      if (directed) atomic_add_i64(&ch.kin[q + 1][x], ki);
    }
  }
}

__global__ void k_exist_cands(const int32_t* lC, const int32_t* nC, const int32_t* par, const int32_t* par_old,
                              int32_t* stE, int32_t epE, int32_t* lE, int32_t* nE) {
  const int32_t n = *nC;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int32_t u = lC[k];
    if (par_old[u] >= 0) stamp_add(stE, epE, par_old[u], lE, nE);
    stamp_add(stE, epE, par[u], lE, nE);
  }
}

// Existence after a level-q0 aggregate step, for the candidate level-q0 nodes
// (old and new parents of the changed nodes): a node with members appears
// (it has no parent yet); a node left without members dies and leaves its
// parent, and a parent that thereby loses its last member dies in turn, up
// the chain to level top.  The walk that takes a parent's member count to
// zero carries on with that parent, so each death is handled once, and the
// counts above q0 only fall meanwhile.  (An emptied node stays listed among
// its parent's children; readers of the lists check the parent.)
struct ExistChain {
  int32_t* cnt[8];
  uint8_t* alive[8];
  int32_t* par[8];
};

__global__ void k_exist_chain(const int32_t* lE, const int32_t* nE, int q0, int top, ExistChain ch, int32_t* err) {
  const int32_t n = *nE;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    int32_t x = lE[k];
    int q = q0;
    const int32_t c = ch.cnt[q][x];
    if (!ch.alive[q][x]) {
      if (c > 0) {
        ch.alive[q][x] = 1;
        if (q < top && ch.par[q][x] >= 0) atomicExch(err, 2);
      }
      continue;
    }
    if (c != 0) continue;
    for (;;) {  // x at level q has no members left
      ch.alive[q][x] = 0;
      if (q >= top) break;
      const int32_t p = ch.par[q][x];
      if (p < 0) break;
      ch.par[q][x] = -1;
      if (atomicAdd(&ch.cnt[q + 1][p], -1) != 1) break;
      x = p;
      ++q;
    }
  }
}

__global__ void k_relabel(const int32_t* l, const int32_t* n, const int32_t* par, const int32_t* lab,
                          int32_t* lab_up) {
  const int32_t m = *n;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const int32_t u = l[k];
    lab_up[par[u]] = lab[u];
  }
}

__global__ void k_nf_records(const u64* keys, int64_t n, int bits, const uint8_t* alive, int32_t* stA, int32_t epA,
                             int32_t* lA, int32_t* nA) {
  const u64 mask = (((u64)1) << bits) - 1;
  GRID_STRIDE(t, n) {
    const int32_t x = (int32_t)(keys[t] >> bits), y = (int32_t)(keys[t] & mask);
    if (alive[x]) stamp_add(stA, epA, x, lA, nA);
    if (alive[y]) stamp_add(stA, epA, y, lA, nA);
  }
}

__global__ void k_nf_nodes(const int32_t* l, const int32_t* n, const int32_t* par, const int32_t* par_old,
                           const uint8_t* alive, int32_t* stA, int32_t epA, int32_t* lA, int32_t* nA) {
  const int32_t m = *n;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const int32_t u = l[k];
    const int32_t p = par[u];
    if (p >= 0 && alive[p]) stamp_add(stA, epA, p, lA, nA);
    if (par_old) {
      const int32_t q = par_old[u];
      if (q >= 0 && alive[q]) stamp_add(stA, epA, q, lA, nA);
    }
  }
}

// ---------------------------------------------------------------- static set-up
__global__ void k_csr_records(const int64_t* rp, const int32_t* col, const int32_t* w, int64_t n, int bits,
                              u64* rk, u64* rv, unsigned long long* err) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < n; v += nw) {
    const int64_t s = rp[v], e = rp[v + 1];
    if (e < s) {
      if (lane == 0) set_err(err, 0, LDL_E_INVALID);
      continue;
    }
    for (int64_t k = s + lane; k < e; k += 32) {
      const int32_t c = col[k];
      if (c < 0 || c >= n) {
        set_err(err, 0, LDL_E_RANGE);
        rk[k] = 0;
        rv[k] = 0;
        continue;
      }
      if (w[k] < 1) set_err(err, 0, LDL_E_INVALID);
      rk[k] = ((u64)v << bits) | (u64)c;
      rv[k] = (u64)(int64_t)w[k];
    }
  }
}

__global__ void k_check_max(const int64_t* s, int64_t n, unsigned long long* err) {
  GRID_STRIDE(i, n) {
    if (s[i] > INT32_MAX) set_err(err, 0, LDL_E_OVERFLOW);
  }
}

__global__ void k_compare(const u64* a, const int64_t* av, const u64* b, const u64* bv, int64_t n,
                          unsigned long long* err) {
  GRID_STRIDE(i, n) {
    if (a[i] != b[i] || (u64)av[i] != bv[i]) set_err(err, 0, LDL_E_INVALID);
  }
}

template <class WT>
__global__ void k_row_sums(Adj<WT> a, int64_t n, int64_t* out, int64_t* self, int64_t* total) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int64_t tot = 0;
  for (int64_t v = warp; v < n; v += nw) {
    const int64_t o = a.off[v];
    const int32_t l = a.len[v];
    int64_t s = 0, sl = 0;
    for (int32_t k = lane; k < l; k += 32) {
      const int64_t w = (int64_t)a.w[o + k];
      s += w;
      if (a.col[o + k] == v) sl += w;
    }
    s = warp_sum_i64(s);
    sl = warp_sum_i64(sl);
    if (lane == 0) {
      out[v] = s;
      if (self) self[v] = sl;
      tot += s;
    }
  }
  if (lane == 0 && total && tot) atomic_add_i64(total, tot);
}

__global__ void k_iota(int32_t* a, int64_t n) {
  GRID_STRIDE(i, n) a[i] = (int32_t)i;
}

__global__ void k_fill_i32(int32_t* a, int64_t n, int32_t v) {
  GRID_STRIDE(i, n) a[i] = v;
}

__global__ void k_alive_list(const uint8_t* alive, int64_t n, int32_t* l, int32_t* cnt) {
  GRID_STRIDE(i, n) {
    if (!alive || alive[i]) l[atomicAdd(cnt, 1)] = (int32_t)i;
  }
}


__global__ void k_esum(const int64_t* e, const int64_t* Kout, const int64_t* Kin, int64_t n, int64_t* E, I128* P) {
  int64_t se = 0;
  i128 sp = 0;
  GRID_STRIDE(i, n) {
    se += e[i];
    sp += (i128)Kout[i] * Kin[i];
  }
  se = warp_sum_i64(se);
  sp = warp_sum_i128(sp);
  if ((threadIdx.x & 31) == 0) {
    if (se) atomic_add_i64(E, se);
    atomic_add_i128(P, sp);
  }
}

__global__ void k_changed_final(const int32_t* lCh, const int32_t* nCh, const int32_t* lab,
                                const int32_t* lab_before, int32_t* out, int32_t* nout) {
  const int32_t n = *nCh;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int32_t u = lCh[k];
    if (lab[u] != lab_before[u]) out[atomicAdd(nout, 1)] = u;
  }
}

__global__ void k_gather(const int32_t* ids, int32_t k, const int32_t* lab, int32_t* out) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) out[i] = lab[ids[i]];
}

}  // namespace

// ================================================================== host side
void gather_labels(ldl_ctx& c, const int32_t* ids, int32_t k, int32_t* out) {
  if (k <= 0) return;
  k_gather<<<grid_for(k, TPB), TPB, 0, c.s>>>(ids, k, c.lv[0].lab.p, out);
  CKL("k_gather");
}
static void throw_err(ldl_ctx& c, unsigned long long* d_err, const char* what) {
  unsigned long long e = 0;
  const HostRead r{d_err, &e, sizeof(e)};
  host_read(c, &r, 1);
  if (e != ~0ull) {
    const int code = (int)(e & 255);
    const long long idx = (long long)(e >> 8);
    char buf[160];
    snprintf(buf, sizeof buf, "%s: status %d at update %lld", what, code, idx);
    ldl_throw((ldl_status)code, buf);
  }
}

static void reset_err(ldl_ctx& c) {
  CK(cudaMemsetAsync(&c.d_sc->err_key, 0xff, sizeof(int64_t), c.s));
}

static unsigned long long* err_ptr(ldl_ctx& c) { return (unsigned long long*)&c.d_sc->err_key; }

int64_t ingest(ldl_ctx& c, const ldl_update* upd, int64_t count, int on_device, int64_t* dm) {
  *dm = 0;
  if (count <= 0) return 0;
  const ldl_update* du = upd;
  if (!on_device) {
    c.upd.reserve(count, c.s);
    CK(cudaMemcpyAsync(c.upd.p, upd, sizeof(ldl_update) * (size_t)count, cudaMemcpyHostToDevice, c.s));
    du = c.upd.p;
  }
  reset_err(c);
  const int g = grid_for(count, TPB);
  k_validate<<<g, TPB, 0, c.s>>>(du, count, c.n, err_ptr(c));
  CKL("k_validate");
  throw_err(c, err_ptr(c), "invalid update");
  c.rk.reserve(2 * count + 2, c.s);
  c.rv.reserve(2 * count + 2, c.s);
  k_upd_keys<<<g, TPB, 0, c.s>>>(du, count, c.bits, c.directed, c.rk.p, c.rv.p);
  CKL("k_upd_keys");
  sort_pairs(c.rk, c.rv, c.tk, c.tv, count, 2 * c.bits, c.P, c.s);
  // unique keys and their first positions
  c.P.flag.reserve(count + 1, c.s);
  c.P.pos.reserve(count + 1, c.s);
  c.rk2.reserve(count + 1, c.s);
  c.rsum.reserve(count + 1, c.s);
  c.rsum2.reserve(count + 1, c.s);
  heads_launch(c.rk.p, count, c.P.flag.p, c.s);
  const int64_t nu = scan_exclusive_i32(c.P.flag.p, c.P.pos.p, count, c.P, c.s, true);
  k_unique_starts<<<g, TPB, 0, c.s>>>(c.rk.p, count, c.P.flag.p, c.P.pos.p, c.rk2.p, c.rsum.p);
  CKL("k_unique_starts");
  c.CS.pos.reserve(nu + 1, c.s);
  c.CS.oldw.reserve(nu + 1, c.s);
  csr_lookup<int32_t>(c.lv[0].out0, c.rk2.p, nu, c.bits, c.CS.pos.p, c.CS.oldw.p, c.CS, c.P, c.s,
                      &c.d_sc->cnt[C_SEG]);
  CK(cudaMemsetAsync(&c.d_sc->dm, 0, sizeof(int64_t), c.s));
  k_seq<<<grid_for(nu, TPB), TPB, 0, c.s>>>(du, count, c.rv.p, c.rsum.p, nu, c.rk2.p, c.CS.oldw.p, c.bits,
                                            c.directed, c.rsum2.p, err_ptr(c), &c.d_sc->dm);
  CKL("k_seq");
  throw_err(c, err_ptr(c), "invalid update sequence");
  {
    const HostRead r{&c.d_sc->dm, dm, sizeof(int64_t)};
    host_read(c, &r, 1);
  }
  if (c.m + *dm >= ((int64_t)1 << 50) || c.m + *dm < 0) ldl_throw(LDL_E_OVERFLOW, "total weight m would reach 2^50");
  zero_cnt(c, K_REC);
  // up to two arcs per distinct key (an undirected edge and its mirror); the
  // sort above may have swapped rk / rv with its scratch, so their capacity
  // is only known to cover `count`
  c.rk.reserve(2 * nu + 2, c.s);
  c.rv.reserve(2 * nu + 2, c.s);
  k_emit_arcs<<<grid_for(nu, TPB), TPB, 0, c.s>>>(c.rk2.p, c.rsum2.p, nu, c.bits, c.directed, c.rk.p, c.rv.p,
                                                  c.dcnt + K_REC);
  CKL("k_emit_arcs");
  const int64_t na = rd_cnt(c, K_REC);
  sort_pairs(c.rk, c.rv, c.tk, c.tv, na, 2 * c.bits, c.P, c.s);
  return na;
}

// Sorted unique out-records of a directed level -> the same records followed
// by their in-direction copies (rows n..2n-1), still sorted: (rk2, rv2), 2*nr.
static void combine_in_out(ldl_ctx& c, const u64* keys, const u64* vals, int64_t nr) {
  c.rk2.reserve(2 * nr + 1, c.s);
  c.rv2.reserve(2 * nr + 1, c.s);
  c.trk.reserve(nr + 1, c.s);
  c.trv.reserve(nr + 1, c.s);
  k_transpose<<<grid_for(nr, TPB), TPB, 0, c.s>>>(keys, vals, nr, c.bits, c.trk.p, c.trv.p, c.n);
  CKL("k_transpose");
  // the out-records are ordered by row, so a stable sort on the new row alone
  // gives (in-row, col) order
  sort_pairs(c.trk, c.trv, c.tk, c.tv, nr, 2 * c.bits + 1, c.P, c.s, c.bits);
  CK(cudaMemcpyAsync(c.rk2.p, keys, sizeof(u64) * (size_t)nr, cudaMemcpyDeviceToDevice, c.s));
  CK(cudaMemcpyAsync(c.rv2.p, vals, sizeof(u64) * (size_t)nr, cudaMemcpyDeviceToDevice, c.s));
  CK(cudaMemcpyAsync(c.rk2.p + nr, c.trk.p, sizeof(u64) * (size_t)nr, cudaMemcpyDeviceToDevice, c.s));
  CK(cudaMemcpyAsync(c.rv2.p + nr, c.trv.p, sizeof(u64) * (size_t)nr, cudaMemcpyDeviceToDevice, c.s));
}

// apply sorted unique records to a level's adjacency (both directions); the
// endpoints of arcs that disappear are recorded for the level's next
// refinement
static void apply_level(ldl_ctx& c, int r, const u64* keys, const int64_t* vals, int64_t nr) {
  if (nr <= 0) return;
  LevelState& Lr = c.lv[r];
  // a deleted arc can only disconnect the refined community holding both of
  // its endpoints (refined communities are connected); until the level's next
  // split its parents change only where a node empties and leaves its parent
  const DelTrack trk{Lr.stK.p, Lr.brk_ep, Lr.lK.p, c.dcnt + K_BRK0 + r, c.n, r < c.T ? Lr.par.p : nullptr};
  const u64* k = keys;
  const u64* v = (const u64*)vals;
  int64_t m = nr;
  if (c.directed) {
    combine_in_out(c, keys, (const u64*)vals, nr);
    k = c.rk2.p;
    v = c.rv2.p;
    m = 2 * nr;
  }
  if (r == 0)
    csr_apply<int32_t>(c.lv[0].out0, k, (const int64_t*)v, m, c.bits, c.CS, c.P, c.s, c.d_sc, &trk);
  else
    csr_apply<int64_t>(c.lv[r].out, k, (const int64_t*)v, m, c.bits, c.CS, c.P, c.s, c.d_sc, &trk);
}

static Chain chain_of(ldl_ctx& c, const int32_t* epA) {
  Chain ch{};
  for (int q = 0; q <= c.T && q < 8; ++q) {
    LevelState& L = c.lv[q];
    ch.par[q] = L.par.p;
    ch.kout[q] = L.kout.p;
    ch.kin[q] = kin_of(c, q);
    ch.pk[q] = L.pk.p;
    ch.pv[q] = L.pv.p;
    ch.stA[q] = L.stA.p;
    ch.lA[q] = L.lA.p;
    ch.epA[q] = epA ? epA[q] : 0;
  }
  return ch;
}

// Records of level q0 onto the pending lists of level q0 (with `self`) and
// of every level above: each list is grown (keeping its contents) to hold n
// more.
static void chain_records(ldl_ctx& c, const u64* keys, const int64_t* vals, int64_t n, int q0, bool self,
                          bool add_k) {
  if (n <= 0 || (!self && q0 >= c.T)) return;
  if (n > INT32_MAX / 2) ldl_throw(LDL_E_OVERFLOW, "too many weight records in one step for the 32-bit counters");
  for (int q = self ? q0 : q0 + 1; q <= c.T; ++q) {
    LevelState& L = c.lv[q];
    // the device counters are 32-bit: a list that would pass them is applied first
    if (L.pend_ub + n > INT32_MAX - 1) flush_level(c, q);
    L.pk.reserve(L.pend_ub + n + 1, c.s, true);
    L.pv.reserve(L.pend_ub + n + 1, c.s, true);
    L.pend_ub += n;
  }
  k_chain_records<<<grid_for(n, TPB), TPB, 0, c.s>>>(keys, vals, n, c.bits, q0, c.T, self ? 1 : 0, add_k ? 1 : 0,
                                                     c.directed, chain_of(c, nullptr), c.dcnt + K_PEND0);
  CKL("k_chain_records");
}

void pending_reset(ldl_ctx& c) {
  for (auto& L : c.lv) L.pend_ub = 0;
  CK(cudaMemsetAsync(c.dcnt + K_PEND0, 0, sizeof(int32_t) * 8, c.s));
}

// Level q's pending records, sorted by (row, col) and summed per arc (zero
// sums dropped), applied to its adjacency: the level's weights become
// current before anything reads them.
void flush_level(ldl_ctx& c, int q, int64_t known) {
  LevelState& L = c.lv[q];
  if (L.pend_ub == 0) return;
  const int64_t n = known >= 0 ? known : rd_cnt(c, K_PEND0 + q);
  L.pend_ub = 0;
  zero_cnt(c, K_PEND0 + q);
  if (n <= 0) return;
  sort_pairs(L.pk, L.pv, c.tk, c.tv, n, 2 * c.bits, c.P, c.s);
  // own output buffers: a flush may run while the caller's records sit in rk / rv
  c.flk.reserve(n + 1, c.s);
  c.flv.reserve(n + 1, c.s);
  const int64_t nr = reduce_by_key(L.pk.p, L.pv.p, n, c.flk.p, c.flv.p, c.P, c.s);
  c.res.pending_records += n;
  c.res.pending_applied += nr;
  apply_level(c, q, c.flk.p, c.flv.p, nr);
}

void repair_batch(ldl_ctx& c, int64_t na, const int32_t* epA, int32_t epT, int64_t dm) {
  if (na <= 0) return;
  // Algorithm 1, applying the batch: it changes level 0
  apply_level(c, 0, c.rk.p, (const int64_t*)c.rv.p, na);
  // statistic repair: m, degrees, community totals (exactly, with sum_C K_out K_in)
  LevelState& L0 = c.lv[0];
  {
    static_assert(offsetof(DevScalars, p_new) == offsetof(DevScalars, p_old) + sizeof(I128), "adjacent scalars");
    ZeroSpans z;
    z.mask = cnt_bit(K_T);
    z.p[0] = (int64_t*)&c.d_sc->p_old;
    z.nw[0] = (int32_t)(2 * sizeof(I128) / sizeof(int64_t));
    z.p[1] = &c.d_sc->de;
    z.nw[1] = 1;
    zero_many(c, z);
  }
  k_dirty<<<grid_for(na, TPB), TPB, 0, c.s>>>(c.rk.p, na, c.bits, L0.lab.p, c.stT.p, epT, c.lT.p, c.dcnt + K_T);
  CKL("k_dirty");
  k_psum<<<grid_for(2 * na, TPB), TPB, 0, c.s>>>(c.lT.p, c.dcnt + K_T, c.Kout.p, Kin_of(c), &c.d_sc->p_old);
  CKL("k_psum");
  k_stat_arcs<<<grid_for(na, TPB), TPB, 0, c.s>>>(c.rk.p, (const int64_t*)c.rv.p, na, c.bits, c.directed, L0.lab.p,
                                                  L0.kout.p, kin_of(c, 0), c.Kout.p, Kin_of(c), c.e.p, &c.d_sc->de,
                                                  L0.stA.p, epA[0], L0.lA.p, c.dcnt + K_A0);
  CKL("k_stat_arcs");
  k_psum<<<grid_for(2 * na, TPB), TPB, 0, c.s>>>(c.lT.p, c.dcnt + K_T, c.Kout.p, Kin_of(c), &c.d_sc->p_new);
  CKL("k_psum");
  I128 p_old, p_new;
  int64_t de = 0;
  const HostRead rr[3] = {{&c.d_sc->p_old, &p_old, sizeof(I128)}, {&c.d_sc->p_new, &p_new, sizeof(I128)},
                          {&c.d_sc->de, &de, sizeof(int64_t)}};
  host_read(c, rr, 3);
  c.m += dm;
  c.E += de;
  c.Psum += i128_of(p_new.hi, p_new.lo) - i128_of(p_old.hi, p_old.lo);
  if (c.T == 0) return;
  // InitFrontier: A^{q+1} = pi_q(A^q) along the chain
  k_chain_frontier<<<grid_for(2 * na, TPB), TPB, 0, c.s>>>(L0.lA.p, c.dcnt + K_A0, c.T, chain_of(c, epA),
                                                           c.dcnt + K_A0);
  CKL("k_chain_frontier");
  // the aggregate chain: W_q(anc(i), anc(j)) += delta and the strengths of
  // every level above 0; the weights are applied when each level is next read
  chain_records(c, c.rk.p, (const int64_t*)c.rv.p, na, 0, false, true);
}

void pushdown(ldl_ctx& c, int r, int32_t epCh, int64_t moved_ub) {
  // lMv holds the level-r nodes moved in this level's move loop; its count
  // stays on the device and moved_ub bounds it (0 exactly when it is empty)
  int32_t* src = c.lMv.p;
  int idx = K_MV;
  int64_t n = std::min<int64_t>(moved_ub, c.n);
  int32_t* bufs[2] = {c.lTmp.p, c.lE2.p};
  int idxs[2] = {K_TMP, K_TMP2};
  int flip = 0;
  for (int q = r - 1; q >= 0 && n > 0; --q) {
    LevelState& L = c.lv[q];
    Adj<int32_t> ch{L.children.off.p, L.children.len.p, L.children.col.p, L.children.w.p};
    int32_t* dst = q > 0 ? bufs[flip] : nullptr;
    zero_cnt(c, idxs[flip]);
    ChunkMap m = chunk_map(c, src, c.dcnt + idx, n, L.children.len.p, nullptr);
    k_push<<<grid_for((int64_t)n * 64, TPB, 16), TPB, 0, c.s>>>(
        m, c.lv[q + 1].lab.p, ch, L.par.p, L.lab.p, dst, c.dcnt + idxs[flip], q == 0 ? c.stCh.p : nullptr, epCh,
        c.lCh.p, c.dcnt + K_CH, c.lab_before.p);
    CKL("k_push");
    if (q > 0) {
      src = bufs[flip];
      idx = idxs[flip];
      n = rd_cnt(c, idx);
      flip ^= 1;
    }
  }
}

// Static build: every alive level-r node becomes a singleton refined
// community (refinement starts from singletons).  Returns |D| (list lD).
int32_t dissolve_all(ldl_ctx& c, int r, int32_t epD) {
  LevelState& L = c.lv[r];
  LevelState& N = c.lv[r + 1];
  zero_cnt(c, K_D);
  k_alive_list<<<grid_for(c.n, TPB), TPB, 0, c.s>>>(r ? L.alive.p : nullptr, c.n, c.lD.p, c.dcnt + K_D);
  CKL("k_alive_list");
  k_stamp_list<<<grid_for(c.n, TPB), TPB, 0, c.s>>>(c.lD.p, c.dcnt + K_D, c.stD.p, epD);
  CKL("k_stamp_list");
  const int32_t nd = rd_cnt(c, K_D);
  if (nd > 0) {
    k_dissolve<<<grid_for(nd, TPB), TPB, 0, c.s>>>(c.lD.p, c.dcnt + K_D, L.par.p, c.par_old.p, L.kout.p,
                                                   kin_of(c, r), N.kout.p, kin_of(c, r + 1), N.cnt.p, c.directed);
    CKL("k_dissolve");
  }
  return nd;
}

void singletons_of(ldl_ctx& c, int r, const int32_t* list, int idx_n, int64_t n_hint, int32_t* out, int idx_out) {
  zero_cnt(c, idx_out);
  if (n_hint > 0) {
    k_singletons<<<grid_for(n_hint, TPB), TPB, 0, c.s>>>(list, c.dcnt + idx_n, c.lv[r].par.p, c.lv[r + 1].cnt.p, out,
                                                         c.dcnt + idx_out);
    CKL("k_singletons");
  }
}

void reset_par(ldl_ctx& c, int r, int32_t nD) {
  if (nD <= 0) return;
  k_reset_par<<<grid_for(nD, TPB), TPB, 0, c.s>>>(c.lD.p, nD, c.lv[r].par.p, c.lv[r + 1].kout.p,
                                                  kin_of(c, r + 1), c.lv[r + 1].cnt.p, c.directed);
  CKL("k_reset_par");
}

template <class WT>
static void leave_degree(ldl_ctx& c, int r, Adj<WT> out, Adj<WT> in, int32_t nD, int32_t epL, int32_t epF) {
  ChunkMap m = chunk_map(c, c.lD.p, c.dcnt + K_D, nD, out.len, c.directed ? in.len : nullptr);
  k_leave_degree<WT><<<grid_for((int64_t)nD * 64, TPB, 16), TPB, 0, c.s>>>(out, in, m, c.lv[r].par.p, c.par_old.p,
                                                                           c.stL.p, epL, c.nbr.p, c.ckf.p, epF);
  CKL("k_leave_degree");
}

template <class WT>
static void union_find(ldl_ctx& c, int r, Adj<WT> out, Adj<WT> in, int32_t nG, int32_t epL) {
  LevelState& L = c.lv[r];
  k_uf_sample<WT><<<grid_for((int64_t)nG * 32, TPB, 16), TPB, 0, c.s>>>(out, in, c.directed, c.lG.p, c.dcnt + K_G,
                                                                       L.par.p, c.stL.p, epL, c.comp.p);
  CKL("k_uf_sample");
  ChunkMap m = chunk_map(c, c.lG.p, c.dcnt + K_G, nG, out.len, c.directed ? in.len : nullptr);
  k_uf<WT><<<grid_for((int64_t)nG * 64, TPB, 16), TPB, 0, c.s>>>(out, in, m, L.par.p, L.alive.p, c.stL.p, epL,
                                                                  c.comp.p);
  CKL("k_uf");
}

// TouchedRefined of a batch update at level r < T (Sec. III-C: refinement
// revisits the communities touched by accepted moves).  A refined community
// lies inside one community, so every node of U* whose label differs from its
// refined community's label (moved at level r, or relabelled from its members'
// moves at level r-1), and every parentless new node, leaves it as a
// singleton named by its own id.  The refined communities that lost a node or
// hold an endpoint of a level-r arc deleted since the level was last refined
// are re-checked for connectivity over the arcs among their remaining members
// (connected components by hooking and pointer jumping): the component with
// the community's seed node keeps the id, any other is renamed after its
// lowest member.  Returns |D|, the nodes whose refined community changed
// (list lD, stamp epD, old parents in par_old); the level's deletion list is
// consumed.
int32_t split(ldl_ctx& c, int r, int32_t epD, int32_t epX) {
  LevelState& L = c.lv[r];
  LevelState& N = c.lv[r + 1];
  {
    ZeroSpans z;
    z.mask = cnt_bit(K_D) | cnt_bit(K_X);
    zero_many(c, z);
  }
  const int32_t epF = c.next_epoch();  // communities whose connectivity is in doubt
  // The level's deleted-arc endpoints and U* stay on the device: both kernels
  // stride over their lists' counts with a grid bounded by the node count.
  const int gs = grid_for(c.n, TPB, 4);
  k_brk_check<<<gs, TPB, 0, c.s>>>(L.lK.p, c.dcnt + K_BRK0 + r, L.alive.p, L.par.p, c.stX.p, epX, c.lX.p,
                                   c.dcnt + K_X, c.ckf.p, epF);
  CKL("k_brk_check");
  const int32_t epL = c.next_epoch();
  k_leave<<<gs, TPB, 0, c.s>>>(c.lUstar.p, c.dcnt + K_USTAR, L.alive.p, L.lab.p, N.lab.p, L.par.p, c.par_old.p,
                               L.kout.p, kin_of(c, r), N.kout.p, kin_of(c, r + 1), N.cnt.p, c.directed, c.stL.p, epL,
                               c.stD.p, epD, c.lD.p, c.dcnt + K_D, c.stX.p, epX, c.lX.p, c.dcnt + K_X, c.nbr.p);
  CKL("k_leave");
  int32_t cnt2[2] = {0, 0};  // K_D, then K_X (adjacent counters)
  {
    const HostRead rr[2] = {{c.dcnt + K_D, &cnt2[0], sizeof(int32_t)}, {c.dcnt + K_X, &cnt2[1], sizeof(int32_t)}};
    host_read(c, rr, 2);
  }
  const int32_t nleft = cnt2[0], nx = cnt2[1];
  bool renamed = false;  // k_rename appends to lD; otherwise |D| = nleft
  if (nx > 0) {
    if (nleft > 0) {
      if (r == 0) leave_degree<int32_t>(c, r, adj_out0(c), adj_in0(c), nleft, epL, epF);
      else leave_degree<int64_t>(c, r, adj_out(c, r), adj_in(c, r), nleft, epL, epF);
    }
    zero_cnt(c, K_G);
    Adj<int32_t> ch{L.children.off.p, L.children.len.p, L.children.col.p, L.children.w.p};
    ChunkMap m = chunk_map(c, c.lX.p, c.dcnt + K_X, nx, L.children.len.p, nullptr);
    k_members<<<grid_for((int64_t)nx * 64, TPB, 16), TPB, 0, c.s>>>(ch, m, L.par.p, c.stL.p, epL, c.ckf.p, epF,
                                                                   c.comp.p, c.lG.p, c.dcnt + K_G);
    CKL("k_members");
    const int32_t nG = rd_cnt(c, K_G);
    c.res.split_members += nG;
    renamed = nG > 0;
    if (nG > 0) {
      if (r == 0) union_find<int32_t>(c, r, adj_out0(c), adj_in0(c), nG, epL);
      else union_find<int64_t>(c, r, adj_out(c, r), adj_in(c, r), nG, epL);
      k_uf_final<<<grid_for(nG, TPB), TPB, 0, c.s>>>(c.lG.p, c.dcnt + K_G, c.comp.p);
      CKL("k_uf_final");
      k_rename<<<grid_for(nG, TPB), TPB, 0, c.s>>>(c.lG.p, c.dcnt + K_G, c.comp.p, L.alive.p, c.stL.p, epL, L.par.p,
                                                   c.par_old.p, L.kout.p, kin_of(c, r), N.kout.p, kin_of(c, r + 1),
                                                   N.cnt.p, c.directed, c.stD.p, epD, c.lD.p, c.dcnt + K_D);
      CKL("k_rename");
    }
  }
  // the deletions of this level are consumed
  L.brk_ep = c.next_epoch();
  zero_cnt(c, K_BRK0 + r);
  return renamed ? rd_cnt(c, K_D) : nleft;
}

// Row entries of the changed nodes (list lC, count on the device, at most
// n_hint) into need (out-rows) and need2 (in-rows).
template <class WT>
static void deg_sum(ldl_ctx& c, Adj<WT> out, Adj<WT> in, int64_t n_hint) {
  static_assert(offsetof(DevScalars, need2) == offsetof(DevScalars, need) + 8, "adjacent accumulators");
  CK(cudaMemsetAsync(&c.d_sc->need, 0, 2 * sizeof(int64_t), c.s));
  k_deg_sum<WT><<<grid_for(n_hint, TPB), TPB, 0, c.s>>>(out, in, c.lC.p, c.dcnt + K_C, &c.d_sc->need,
                                                        &c.d_sc->need2);
  CKL("k_deg_sum");
}

// deg: out-row and in-row entries of the changed nodes (deg_sum)
template <class WT>
static void emit_records(ldl_ctx& c, int r, Adj<WT> out, Adj<WT> in, int32_t nC, int32_t epC, bool build,
                         const int64_t (&deg)[2]) {
  // at most a subtract and an add record per visited entry; in the static
  // build no node had a parent (no subtract records) and every node is
  // changed (no in-row records), so one record per out-row entry
  const int64_t cap = (build ? deg[0] : 2 * (deg[0] + deg[1])) + 16;
  if (cap > INT32_MAX) ldl_throw(LDL_E_OVERFLOW, "aggregate records beyond the 32-bit record counter");
  c.rk2.reserve(cap, c.s);
  c.rv2.reserve(cap, c.s);
  zero_cnt(c, K_REC);
  ChunkMap m = chunk_map(c, c.lC.p, c.dcnt + K_C, nC, out.len, in.len);
  k_emit<WT><<<grid_for((int64_t)nC * 64, TPB, 16), TPB, 0, c.s>>>(out, in, m, c.lv[r].par.p, c.par_old.p,
                                                                          c.stC.p, epC, c.bits, c.rk2.p, c.rv2.p,
                                                                          c.dcnt + K_REC, cap, c.dcnt + K_ERR);
  CKL("k_emit");
}

void aggregate(ldl_ctx& c, int r, int32_t epD, int32_t epC, int32_t epA_next, bool build, int32_t nD) {
  (void)epD;
  LevelState& L = c.lv[r];
  LevelState& N = c.lv[r + 1];
  // changed nodes
  sub_begin(c);
  zero_cnt(c, K_C);
  k_changed<<<grid_for(nD, TPB), TPB, 0, c.s>>>(c.lD.p, c.dcnt + K_D, L.par.p, c.par_old.p, c.stC.p, epC, c.lC.p,
                                                c.dcnt + K_C);
  CKL("k_changed");
  // the changed nodes' row entries (lC is a subset of lD, so nD bounds the
  // launch); one read returns them with |C| and |U*| (for the relabelling)
  if (r == 0) deg_sum<int32_t>(c, adj_out0(c), adj_in0(c), nD);
  else deg_sum<int64_t>(c, adj_out(c, r), adj_in(c, r), nD);
  int32_t nC = 0, nUs = 0;
  int64_t deg[2] = {0, 0};
  {
    const HostRead rr[3] = {{c.dcnt + K_C, &nC, sizeof(int32_t)}, {c.dcnt + K_USTAR, &nUs, sizeof(int32_t)},
                            {&c.d_sc->need, deg, 2 * sizeof(int64_t)}};
    host_read(c, rr, 3);
  }
  int64_t nr = 0;
  if (nC > 0) {
    if (r == 0) emit_records<int32_t>(c, r, adj_out0(c), adj_in0(c), nC, epC, build, deg);
    else emit_records<int64_t>(c, r, adj_out(c, r), adj_in(c, r), nC, epC, build, deg);
    // node and children records (they need only the parents), so that one
    // read returns both record counts
    c.ndx.reserve(2 * (int64_t)nC + 2, c.s);
    c.ndko.reserve(2 * (int64_t)nC + 2, c.s);
    c.ndki.reserve(2 * (int64_t)nC + 2, c.s);
    c.crk.reserve(2 * (int64_t)nC + 2, c.s);
    c.crv.reserve(2 * (int64_t)nC + 2, c.s);
    {
      ZeroSpans z;
      z.mask = cnt_bit(K_NREC) | cnt_bit(K_CREC);
      zero_many(c, z);
    }
    k_emit_nodes<<<grid_for(nC, TPB), TPB, 0, c.s>>>(c.lC.p, c.dcnt + K_C, L.par.p, c.par_old.p, L.kout.p,
                                                     kin_of(c, r), c.bits, c.ndx.p, c.ndko.p, c.ndki.p,
                                                     c.dcnt + K_NREC, c.crk.p, c.crv.p, c.dcnt + K_CREC);
    CKL("k_emit_nodes");
    int32_t nrec32 = 0, ncr32 = 0;
    {
      const HostRead rr[2] = {{c.dcnt + K_REC, &nrec32, sizeof(int32_t)}, {c.dcnt + K_CREC, &ncr32, sizeof(int32_t)}};
      host_read(c, rr, 2);
    }
    const int64_t nrec = nrec32, ncr = ncr32;
    if (nrec > c.rk2.cap) ldl_throw(LDL_E_INVALID, "internal: aggregate records exceed their bound");
    sub_end(c, SU_AGG_EMIT);
    sub_begin(c);
    sort_pairs(c.rk2, c.rv2, c.tk, c.tv, nrec, 2 * c.bits, c.P, c.s);
    c.rk.reserve(nrec + 1, c.s);
    c.rv.reserve(nrec + 1, c.s);
    c.rsum.reserve(nrec + 1, c.s);
    nr = reduce_by_key(c.rk2.p, c.rv2.p, nrec, c.rk.p, c.rsum.p, c.P, c.s);
    CK(cudaMemcpyAsync(c.rv.p, c.rsum.p, sizeof(int64_t) * (size_t)nr, cudaMemcpyDeviceToDevice, c.s));
    c.res.agg_records += nr;
    sub_end(c, SU_AGG_SORT);
    sub_begin(c);
    sort_pairs(c.crk, c.crv, c.tk, c.tv, ncr, 2 * c.bits, c.P, c.s);
    // keep the level r+1 record keys for NextFrontier
    c.fk.reserve(nr + 1, c.s);
    if (nr) CK(cudaMemcpyAsync(c.fk.p, c.rk.p, sizeof(u64) * (size_t)nr, cudaMemcpyDeviceToDevice, c.s));
    if (build) {
      // level r+1 starts empty: build its adjacency and the children lists
      if (c.directed) {
        combine_in_out(c, c.rk.p, c.rv.p, nr);
        csr_build<int64_t>(N.out, 2 * c.n, c.rk2.p, (const int64_t*)c.rv2.p, 2 * nr, c.bits, 25, c.CS, c.P, c.s);
      } else {
        csr_build<int64_t>(N.out, c.n, c.rk.p, c.rsum.p, nr, c.bits, 25, c.CS, c.P, c.s);
      }
      csr_build<int32_t>(L.children, c.n, c.crk.p, (const int64_t*)c.crv.p, ncr, c.bits, 25, c.CS, c.P, c.s);
    } else {
      // the level r+1 records join its pending list and, mapped through the
      // current parents, the lists of the levels above; the strength moves
      // reach every ancestor level at once
      chain_records(c, c.rk.p, (const int64_t*)c.rv.p, nr, r + 1, true, false);
      csr_apply<int32_t>(L.children, c.crk.p, (const int64_t*)c.crv.p, ncr, c.bits, c.CS, c.P, c.s, c.d_sc);
    }
    sub_end(c, SU_AGG_APPLY);
    sub_begin(c);
    if (!build && r + 1 < c.T) {
      k_chain_nodes<<<grid_for(2 * (int64_t)nC, TPB), TPB, 0, c.s>>>(c.ndx.p, c.ndko.p, c.ndki.p, c.dcnt + K_NREC,
                                                                      r + 1, c.T, c.directed, chain_of(c, nullptr));
      CKL("k_chain_nodes");
    }
    sub_end(c, SU_AGG_UP);
    sub_begin(c);
    // existence: appear at r+1, emptied nodes cascade upwards
    int32_t epE = c.next_epoch();
    zero_cnt(c, K_E);
    k_exist_cands<<<grid_for(nC, TPB), TPB, 0, c.s>>>(c.lC.p, c.dcnt + K_C, L.par.p, c.par_old.p, c.stE.p, epE,
                                                      c.lE.p, c.dcnt + K_E);
    CKL("k_exist_cands");
    ExistChain ech{};
    for (int q = 0; q <= c.T && q < 8; ++q) {
      ech.cnt[q] = c.lv[q].cnt.p;
      ech.alive[q] = c.lv[q].alive.p;
      ech.par[q] = c.lv[q].par.p;
    }
    k_exist_chain<<<grid_for(2 * (int64_t)nC, TPB), TPB, 0, c.s>>>(c.lE.p, c.dcnt + K_E, r + 1, c.T, ech,
                                                                    c.dcnt + K_ERR);
    CKL("k_exist_chain");
    // the error flag K_ERR is read once at the end of the batch (or of the static build)
  } else {
    sub_end(c, SU_AGG_EMIT);
    sub_begin(c);
  }
  // relabel the level-(r+1) images of frontier and dissolved nodes
  if (nUs > 0) {
    k_relabel<<<grid_for(nUs, TPB), TPB, 0, c.s>>>(c.lUstar.p, c.dcnt + K_USTAR, L.par.p, L.lab.p, N.lab.p);
    CKL("k_relabel");
  }
  if (nD > 0) {
    k_relabel<<<grid_for(nD, TPB), TPB, 0, c.s>>>(c.lD.p, c.dcnt + K_D, L.par.p, L.lab.p, N.lab.p);
    CKL("k_relabel");
  }
  // NextFrontier for level r+1
  if (epA_next) {
    if (nr > 0) {
      k_nf_records<<<grid_for(nr, TPB), TPB, 0, c.s>>>(c.fk.p, nr, c.bits, N.alive.p, N.stA.p,
                                                       epA_next, N.lA.p, c.dcnt + K_A0 + r + 1);
      CKL("k_nf_records");
    }
    if (nD > 0) {
      k_nf_nodes<<<grid_for(nD, TPB), TPB, 0, c.s>>>(c.lD.p, c.dcnt + K_D, L.par.p, c.par_old.p, N.alive.p, N.stA.p,
                                                     epA_next, N.lA.p, c.dcnt + K_A0 + r + 1);
      CKL("k_nf_nodes");
    }
    if (nUs > 0) {
      k_nf_nodes<<<grid_for(nUs, TPB), TPB, 0, c.s>>>(c.lUstar.p, c.dcnt + K_USTAR, L.par.p, nullptr, N.alive.p,
                                                      N.stA.p, epA_next, N.lA.p, c.dcnt + K_A0 + r + 1);
      CKL("k_nf_nodes");
    }
  }
  sub_end(c, SU_AGG_EXIST);
}

void level_alloc(ldl_ctx& c, int r) {
  LevelState& L = c.lv[r];
  if (L.allocated) return;
  const int64_t n = c.n;
  L.lab.exact(n);
  L.par.exact(n);
  L.cnt.exact(n);
  L.kout.exact(n);
  if (c.directed) L.kin.exact(n);
  L.alive.exact(n);
  L.stA.exact(n);
  L.lA.exact(n);
  L.stK.exact(n);
  L.lK.exact(n);
  CK(cudaMemsetAsync(L.stK.p, 0, sizeof(int32_t) * (size_t)n, c.s));
  CK(cudaMemsetAsync(L.lab.p, 0, sizeof(int32_t) * (size_t)n, c.s));
  CK(cudaMemsetAsync(L.par.p, 0xff, sizeof(int32_t) * (size_t)n, c.s));
  CK(cudaMemsetAsync(L.cnt.p, 0, sizeof(int32_t) * (size_t)n, c.s));
  CK(cudaMemsetAsync(L.kout.p, 0, sizeof(int64_t) * (size_t)n, c.s));
  if (c.directed) CK(cudaMemsetAsync(L.kin.p, 0, sizeof(int64_t) * (size_t)n, c.s));
  CK(cudaMemsetAsync(L.alive.p, 0, (size_t)n, c.s));
  CK(cudaMemsetAsync(L.stA.p, 0, sizeof(int32_t) * (size_t)n, c.s));
  L.allocated = true;
}

void level_free(ldl_ctx& c, int r) { c.lv[r].release(); }

int32_t alive_list(ldl_ctx& c, int r, int32_t* list, int idx) {
  zero_cnt(c, idx);
  k_alive_list<<<grid_for(c.n, TPB), TPB, 0, c.s>>>(r ? c.lv[r].alive.p : nullptr, c.n, list, c.dcnt + idx);
  CKL("k_alive_list");
  return rd_cnt(c, idx);
}

void changed_labels_launch(ldl_ctx& c) {
  // strides over the candidates' device count with a grid bounded by the node count
  zero_cnt(c, K_CHG);
  k_changed_final<<<grid_for(c.n, TPB, 4), TPB, 0, c.s>>>(c.lCh.p, c.dcnt + K_CH, c.lv[0].lab.p, c.lab_before.p,
                                                          c.lChg.p, c.dcnt + K_CHG);
  CKL("k_changed_final");
}

void upload_graph(ldl_ctx& c, int64_t nnz, const int64_t* row_ptr, const int32_t* col, const int32_t* w) {
  const int64_t n = c.n;
  DBuf<int64_t> drp;
  DBuf<int32_t> dcol, dw;
  drp.exact(n + 1);
  dcol.exact(nnz + 1);
  dw.exact(nnz + 1);
  CK(cudaMemcpyAsync(drp.p, row_ptr, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, c.s));
  if (nnz) {
    CK(cudaMemcpyAsync(dcol.p, col, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, c.s));
    CK(cudaMemcpyAsync(dw.p, w, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, c.s));
  }
  c.rk.reserve(nnz + 1, c.s);
  c.rv.reserve(nnz + 1, c.s);
  reset_err(c);
  k_csr_records<<<grid_for(n * 32, TPB), TPB, 0, c.s>>>(drp.p, dcol.p, dw.p, n, c.bits, c.rk.p, c.rv.p, err_ptr(c));
  CKL("k_csr_records");
  CK(cudaStreamSynchronize(c.s));
  drp.release();
  dcol.release();
  dw.release();
  throw_err(c, err_ptr(c), "invalid CSR");
  sort_pairs(c.rk, c.rv, c.tk, c.tv, nnz, 2 * c.bits, c.P, c.s);
  c.rk2.reserve(nnz + 1, c.s);
  c.rsum.reserve(nnz + 1, c.s);
  const int64_t na = reduce_by_key(c.rk.p, c.rv.p, nnz, c.rk2.p, c.rsum.p, c.P, c.s);
  reset_err(c);
  k_check_max<<<grid_for(na, TPB), TPB, 0, c.s>>>(c.rsum.p, na, err_ptr(c));
  CKL("k_check_max");
  throw_err(c, err_ptr(c), "summed weight above INT32_MAX");
  // (rk2, rsum) = unique arcs
  CK(cudaMemcpyAsync(c.rk.p, c.rk2.p, sizeof(u64) * (size_t)na, cudaMemcpyDeviceToDevice, c.s));
  CK(cudaMemcpyAsync(c.rv.p, c.rsum.p, sizeof(int64_t) * (size_t)na, cudaMemcpyDeviceToDevice, c.s));
  if (na) {
    c.rk2.reserve(na + 1, c.s);
    c.rv2.reserve(na + 1, c.s);
    if (!c.directed) {
      k_transpose<<<grid_for(na, TPB), TPB, 0, c.s>>>(c.rk.p, c.rv.p, na, c.bits, c.rk2.p, c.rv2.p, 0);
      CKL("k_transpose");
      sort_pairs(c.rk2, c.rv2, c.tk, c.tv, na, 2 * c.bits, c.P, c.s, c.bits);  // rows already ordered
      reset_err(c);
      k_compare<<<grid_for(na, TPB), TPB, 0, c.s>>>(c.rk.p, (const int64_t*)c.rv.p, c.rk2.p, c.rv2.p, na,
                                                    err_ptr(c));
      CKL("k_compare");
      throw_err(c, err_ptr(c), "undirected CSR is not symmetric");
    }
  }
  LevelState& L0 = c.lv[0];
  if (c.directed) {
    combine_in_out(c, c.rk.p, c.rv.p, na);
    csr_build<int32_t>(L0.out0, 2 * n, c.rk2.p, (const int64_t*)c.rv2.p, 2 * na, c.bits, 25, c.CS, c.P, c.s);
  } else {
    csr_build<int32_t>(L0.out0, n, c.rk.p, (const int64_t*)c.rv.p, na, c.bits, 25, c.CS, c.P, c.s);
  }
  // strengths, m, labels, community totals
  CK(cudaMemsetAsync(&c.d_sc->dm, 0, sizeof(int64_t), c.s));
  const int gw = grid_for(n * 32, TPB);
  k_row_sums<int32_t><<<gw, TPB, 0, c.s>>>(adj_out0(c), n, L0.kout.p, c.e.p, &c.d_sc->dm);
  CKL("k_row_sums");
  if (c.directed) {
    k_row_sums<int32_t><<<gw, TPB, 0, c.s>>>(adj_in0(c), n, L0.kin.p, nullptr, nullptr);
    CKL("k_row_sums(in)");
  }
  k_iota<<<grid_for(n, TPB), TPB, 0, c.s>>>(L0.lab.p, n);
  CKL("k_iota");
  k_fill_i32<<<grid_for(n, TPB), TPB, 0, c.s>>>(L0.cnt.p, n, 1);
  CKL("k_fill_i32");
  CK(cudaMemsetAsync(L0.alive.p, 1, (size_t)n, c.s));
  CK(cudaMemcpyAsync(c.Kout.p, L0.kout.p, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToDevice, c.s));
  if (c.directed) CK(cudaMemcpyAsync(c.Kin.p, L0.kin.p, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToDevice, c.s));
  CK(cudaMemsetAsync(&c.d_sc->de, 0, sizeof(int64_t), c.s));
  CK(cudaMemsetAsync(&c.d_sc->p_new, 0, sizeof(I128), c.s));
  k_esum<<<grid_for(n, TPB), TPB, 0, c.s>>>(c.e.p, c.Kout.p, Kin_of(c), n, &c.d_sc->de, &c.d_sc->p_new);
  CKL("k_esum");
  DevScalars h;
  CK(cudaMemcpyAsync(&h, c.d_sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c.s));
  CK(cudaStreamSynchronize(c.s));
  c.m = h.dm;
  if (c.m >= ((int64_t)1 << 50)) ldl_throw(LDL_E_OVERFLOW, "total weight m reaches 2^50");
  c.E = h.de;
  c.Psum = i128_of(h.p_new.hi, h.p_new.lo);
}
