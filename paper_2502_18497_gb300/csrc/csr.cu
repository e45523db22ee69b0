// Device-resident CSR with per-row slack (Sec. III-A keeps adjacency at
// every level; edge inserts go into the row's slack, deletes compact the row,
// a row out of slack moves to the end of the pool).
//
// Records are (key, delta) pairs with key = row << bshift | col, sorted by
// key and unique.  One warp owns one row segment, so updates need no atomics
// on the row itself; physical entry order inside a row never affects results
// because every consumer reduces integers.
#include "csr.cuh"
#include "prims.cuh"

namespace {

__device__ inline int64_t seg_end(const u64* keys, int64_t s, int64_t nrec, int bshift) {
  // first index > s whose row differs from row(s)
  const u64 row = keys[s] >> bshift;
  const u64 bound = (row + 1) << bshift;
  int64_t lo = s + 1, hi = nrec;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (keys[mid] < bound) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void k_seg_heads(const u64* keys, int64_t nrec, int bshift, int64_t* seg, int32_t* nseg) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrec; i += (int64_t)gridDim.x * blockDim.x) {
    if (i == 0 || (keys[i] >> bshift) != (keys[i - 1] >> bshift)) seg[atomicAdd(nseg, 1)] = i;
  }
}

template <class WT>
__global__ void k_match(const int64_t* off, const int32_t* len, const int32_t* col, const WT* w, const u64* keys,
                        int64_t nrec, int bshift, const int64_t* seg, const int32_t* nseg, int32_t* pos,
                        int64_t* oldw) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const u64 cmask = (((u64)1) << bshift) - 1;
  const int64_t ns = *nseg;
  for (int64_t si = warp; si < ns; si += nw) {
    const int64_t s = seg[si];
    const int64_t e = seg_end(keys, s, nrec, bshift);
    const int64_t row = (int64_t)(keys[s] >> bshift);
    const int64_t ro = off[row];
    const int32_t rl = len[row];
    for (int32_t k = lane; k < rl; k += 32) {
      const int32_t c = col[ro + k];
      if (c < 0) continue;
      int64_t lo = s, hi = e;
      while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)(keys[mid] & cmask) < (int64_t)c) lo = mid + 1; else hi = mid;
      }
      if (lo < e && (int64_t)(keys[lo] & cmask) == (int64_t)c) {
        pos[lo] = k;
        if (oldw) oldw[lo] = (int64_t)w[ro + k];
      }
    }
  }
}

// Per segment: count inserts and deletes, decide relocation.
__global__ void k_plan(const int32_t* len, const int32_t* cap, const u64* keys, const int64_t* delta, int64_t nrec,
                       int bshift, const int64_t* seg, const int32_t* nseg, const int32_t* pos, const int64_t* oldw,
                       int32_t* newcap, int64_t* need, int32_t* err) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t ns = *nseg;
  for (int64_t si = warp; si < ns; si += nw) {
    const int64_t s = seg[si];
    const int64_t e = seg_end(keys, s, nrec, bshift);
    const int64_t row = (int64_t)(keys[s] >> bshift);
    int ins = 0, del = 0, bad = 0;
    for (int64_t i = s + lane; i < e; i += 32) {
      const bool found = pos[i] >= 0;
      const int64_t nw_ = (found ? oldw[i] : 0) + delta[i];
      if (nw_ < 0) bad = 1;
      if (!found && nw_ > 0) ++ins;
      if (!found && nw_ == 0) bad = 1;  // a zero delta on an absent entry never reaches here
      if (found && nw_ == 0) ++del;
    }
    ins = warp_sum_i32(ins);
    del = warp_sum_i32(del);
    bad = warp_sum_i32(bad);
    if (lane == 0) {
      if (bad) atomicExch(err, 1);
      const int64_t nl = (int64_t)len[row] - del + ins;
      int32_t nc = 0;
      if (nl > cap[row]) {
        int64_t want = nl + (nl >> 1) + 4;
        want = (want + 3) & ~(int64_t)3;
        nc = (int32_t)want;
        atomic_add_i64(need, want);
      }
      newcap[si] = nc;
    }
  }
}

template <class WT>
__global__ void k_relocate(int64_t* off, int32_t* len, int32_t* cap, int32_t* col, WT* w, const u64* keys,
                           int bshift, const int64_t* seg, const int32_t* nseg, const int32_t* newcap,
                           int64_t* pool_top) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t ns = *nseg;
  for (int64_t si = warp; si < ns; si += nw) {
    const int32_t nc = newcap[si];
    if (nc == 0) continue;
    const int64_t row = (int64_t)(keys[seg[si]] >> bshift);
    int64_t no = 0;
    if (lane == 0) no = (int64_t)atomicAdd((unsigned long long*)pool_top, (unsigned long long)nc);
    no = __shfl_sync(0xffffffffu, no, 0);
    const int64_t oo = off[row];
    const int32_t rl = len[row];
    for (int32_t k = lane; k < rl; k += 32) {
      col[no + k] = col[oo + k];
      w[no + k] = w[oo + k];
    }
    __syncwarp();
    if (lane == 0) {
      off[row] = no;
      cap[row] = nc;
    }
  }
}

template <class WT>
__global__ void k_write(const int64_t* off, int32_t* len, int32_t* col, WT* w, const u64* keys, const int64_t* delta,
                        int64_t nrec, int bshift, const int64_t* seg, const int32_t* nseg, const int32_t* pos,
                        const int64_t* oldw) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const u64 cmask = (((u64)1) << bshift) - 1;
  const int64_t ns = *nseg;
  for (int64_t si = warp; si < ns; si += nw) {
    const int64_t s = seg[si];
    const int64_t e = seg_end(keys, s, nrec, bshift);
    const int64_t row = (int64_t)(keys[s] >> bshift);
    const int64_t ro = off[row];
    int del = 0;
    for (int64_t i = s + lane; i < e; i += 32) {
      if (pos[i] >= 0) {
        const int64_t nv = oldw[i] + delta[i];
        if (nv == 0) {
          col[ro + pos[i]] = -1;
          ++del;
        } else {
          w[ro + pos[i]] = (WT)nv;
        }
      }
    }
    del = warp_sum_i32(del);
    del = __shfl_sync(0xffffffffu, del, 0);
    __syncwarp();
    int32_t rl = len[row];
    if (del > 0) {  // stable in-place compaction of the row
      int32_t out = 0;
      for (int32_t base = 0; base < rl; base += 32) {
        const int32_t k = base + lane;
        int32_t c = -1;
        WT x = 0;
        if (k < rl) {
          c = col[ro + k];
          x = w[ro + k];
        }
        const bool keep = c >= 0;
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        __syncwarp();
        if (keep) {
          const int32_t o = out + __popc(bal & ((1u << lane) - 1u));
          col[ro + o] = c;
          w[ro + o] = x;
        }
        out += __popc(bal);
        __syncwarp();
      }
      rl = out;
    }
    // append inserts in record order
    int32_t top = rl;
    for (int64_t b = s; b < e; b += 32) {
      const int64_t i = b + lane;
      bool ins = false;
      int64_t nv = 0;
      if (i < e && pos[i] < 0) {
        nv = delta[i];
        ins = nv > 0;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, ins);
      if (ins) {
        const int32_t o = top + __popc(bal & ((1u << lane) - 1u));
        col[ro + o] = (int32_t)(keys[i] & cmask);
        w[ro + o] = (WT)nv;
      }
      top += __popc(bal);
    }
    __syncwarp();
    if (lane == 0) len[row] = top;
  }
}

// ---------------------------------------------------------------- build
__global__ void k_count_rows(const u64* keys, int64_t nrec, int bshift, int32_t* cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrec; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[keys[i] >> bshift], 1);
}

__global__ void k_caps(const int32_t* cnt, int64_t n, int32_t* cap, int slack_pct) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = cnt[v];
    int64_t c = d + (d * slack_pct) / 100 + (d ? 2 : 0);
    c = (c + 1) & ~(int64_t)1;
    cap[v] = (int32_t)c;
  }
}

template <class WT>
__global__ void k_scatter_build(const u64* keys, const int64_t* vals, int64_t nrec, int bshift, const int64_t* rs,
                                const int64_t* off, int32_t* col, WT* w) {
  const u64 cmask = (((u64)1) << bshift) - 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrec; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = (int64_t)(keys[i] >> bshift);
    const int64_t p = off[row] + (i - rs[row]);
    col[p] = (int32_t)(keys[i] & cmask);
    w[p] = (WT)vals[i];
  }
}

__global__ void k_i32_to_i64(const int32_t* a, int64_t* b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

}  // namespace

// ---------------------------------------------------------------- host side
template <class WT>
void csr_build(SlackCSR<WT>& g, int64_t n, const u64* keys, const int64_t* vals, int64_t nrec, int bshift,
               int slack_pct, CsrScratch& S, Prims& P, cudaStream_t s) {
  g.n = n;
  g.off.exact(n + 1);
  g.len.exact(n + 1);
  g.cap.exact(n + 1);
  CK(cudaMemsetAsync(g.len.p, 0, sizeof(int32_t) * (size_t)(n + 1), s));
  if (nrec > 0) {
    k_count_rows<<<grid_for(nrec, 256), 256, 0, s>>>(keys, nrec, bshift, g.len.p);
    CKL("k_count_rows");
  }
  k_caps<<<grid_for(n, 256), 256, 0, s>>>(g.len.p, n, g.cap.p, slack_pct);
  CKL("k_caps");
  S.rs.reserve(n + 1, s);
  S.tmp64.reserve(n + 1, s);
  k_i32_to_i64<<<grid_for(n, 256), 256, 0, s>>>(g.len.p, S.tmp64.p, n);
  CKL("k_i32_to_i64");
  scan_exclusive(S.tmp64.p, S.rs.p, n, P, s, false);
  k_i32_to_i64<<<grid_for(n, 256), 256, 0, s>>>(g.cap.p, S.tmp64.p, n);
  CKL("k_i32_to_i64");
  const int64_t total = scan_exclusive(S.tmp64.p, g.off.p, n, P, s, true);
  const int64_t pool = total + total / 8 + 1024;
  g.col.release();
  g.w.release();
  g.col.exact(pool);
  g.w.exact(pool);
  g.pool_top = total;
  if (nrec > 0) {
    k_scatter_build<WT><<<grid_for(nrec, 256), 256, 0, s>>>(keys, vals, nrec, bshift, S.rs.p, g.off.p, g.col.p,
                                                            g.w.p);
    CKL("k_scatter_build");
  }
}

template <class WT>
void csr_lookup(const SlackCSR<WT>& g, const u64* keys, int64_t nrec, int bshift, int32_t* pos, int64_t* oldw,
                CsrScratch& S, Prims& P, cudaStream_t s, int32_t* d_nseg) {
  (void)P;
  if (nrec <= 0) return;
  S.seg.reserve(nrec + 1, s);
  CK(cudaMemsetAsync(d_nseg, 0, sizeof(int32_t), s));
  CK(cudaMemsetAsync(pos, 0xff, sizeof(int32_t) * (size_t)nrec, s));
  CK(cudaMemsetAsync(oldw, 0, sizeof(int64_t) * (size_t)nrec, s));
  k_seg_heads<<<grid_for(nrec, 256), 256, 0, s>>>(keys, nrec, bshift, S.seg.p, d_nseg);
  CKL("k_seg_heads");
  k_match<WT><<<grid_for(nrec * 32, 256), 256, 0, s>>>(g.off.p, g.len.p, g.col.p, g.w.p, keys, nrec, bshift,
                                                      S.seg.p, d_nseg, pos, oldw);
  CKL("k_match");
}

template <class WT>
void csr_apply(SlackCSR<WT>& g, const u64* keys, const int64_t* delta, int64_t nrec, int bshift, CsrScratch& S,
               Prims& P, cudaStream_t s, DevScalars* d_sc) {
  if (nrec <= 0) return;
  S.pos.reserve(nrec + 1, s);
  S.oldw.reserve(nrec + 1, s);
  S.newcap.reserve(nrec + 1, s);
  int32_t* d_nseg = &d_sc->cnt[C_SEG];
  csr_lookup<WT>(g, keys, nrec, bshift, S.pos.p, S.oldw.p, S, P, s, d_nseg);
  CK(cudaMemsetAsync(&d_sc->need, 0, sizeof(int64_t), s));
  CK(cudaMemsetAsync(&d_sc->cnt[C_Z], 0, sizeof(int32_t), s));
  const int gw = grid_for(nrec * 32, 256);
  k_plan<<<gw, 256, 0, s>>>(g.len.p, g.cap.p, keys, delta, nrec, bshift, S.seg.p, d_nseg, S.pos.p, S.oldw.p,
                            S.newcap.p, &d_sc->need, &d_sc->cnt[C_Z]);
  CKL("k_plan");
  int64_t need = 0;
  int32_t bad = 0;
  CK(cudaMemcpyAsync(&need, &d_sc->need, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&bad, &d_sc->cnt[C_Z], sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (bad) ldl_throw(LDL_E_INVALID, "internal: adjacency update would make a weight negative");
  if (need > 0) {
    if (g.pool_top + need > g.col.cap) {
      int64_t nc = (g.pool_top + need) + (g.pool_top + need) / 4 + 4096;
      // grow the pool keeping its contents
      int32_t* c2 = (int32_t*)dalloc(sizeof(int32_t) * (size_t)nc);
      WT* w2 = (WT*)dalloc(sizeof(WT) * (size_t)nc);
      CK(cudaMemcpyAsync(c2, g.col.p, sizeof(int32_t) * (size_t)g.pool_top, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(w2, g.w.p, sizeof(WT) * (size_t)g.pool_top, cudaMemcpyDeviceToDevice, s));
      CK(cudaStreamSynchronize(s));
      dfree(g.col.p);
      dfree(g.w.p);
      g.col.p = c2;
      g.col.cap = nc;
      g.w.p = w2;
      g.w.cap = nc;
    }
    CK(cudaMemcpyAsync(&d_sc->pool_top, &g.pool_top, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    k_relocate<WT><<<gw, 256, 0, s>>>(g.off.p, g.len.p, g.cap.p, g.col.p, g.w.p, keys, bshift, S.seg.p, d_nseg,
                                      S.newcap.p, &d_sc->pool_top);
    CKL("k_relocate");
    g.pool_top += need;
  }
  k_write<WT><<<gw, 256, 0, s>>>(g.off.p, g.len.p, g.col.p, g.w.p, keys, delta, nrec, bshift, S.seg.p, d_nseg,
                                 S.pos.p, S.oldw.p);
  CKL("k_write");
}

template void csr_build<int32_t>(SlackCSR<int32_t>&, int64_t, const u64*, const int64_t*, int64_t, int, int,
                                 CsrScratch&, Prims&, cudaStream_t);
template void csr_build<int64_t>(SlackCSR<int64_t>&, int64_t, const u64*, const int64_t*, int64_t, int, int,
                                 CsrScratch&, Prims&, cudaStream_t);
template void csr_lookup<int32_t>(const SlackCSR<int32_t>&, const u64*, int64_t, int, int32_t*, int64_t*,
                                  CsrScratch&, Prims&, cudaStream_t, int32_t*);
template void csr_lookup<int64_t>(const SlackCSR<int64_t>&, const u64*, int64_t, int, int32_t*, int64_t*,
                                  CsrScratch&, Prims&, cudaStream_t, int32_t*);
template void csr_apply<int32_t>(SlackCSR<int32_t>&, const u64*, const int64_t*, int64_t, int, CsrScratch&, Prims&,
                                 cudaStream_t, DevScalars*);
template void csr_apply<int64_t>(SlackCSR<int64_t>&, const u64*, const int64_t*, int64_t, int, CsrScratch&, Prims&,
                                 cudaStream_t, DevScalars*);
