// Device-resident CSR with per-row slack (Sec. III-A keeps adjacency at
// every level; inserts go into the row's slack, deletes shrink the row, a row
// out of slack moves to the end of the pool).
//
// Every row is kept sorted by neighbour id.  Records are (key, delta) pairs
// with key = row << bshift | col, sorted by key and unique.  Matching a record
// is a binary search in its row (one thread per record); a row that gains or
// loses entries is rebuilt by a flattened scatter in which every kept entry
// and every inserted entry computes its own destination, so hub rows spread
// over the whole GPU instead of one warp.
#include "csr.cuh"
#include "prims.cuh"

namespace {

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

constexpr int TPB = 256;

// binary search of col in a sorted row: returns the lower bound index
__device__ inline int32_t row_lower_bound(const int32_t* col, int64_t off, int32_t len, int32_t c) {
  int32_t lo = 0, hi = len;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (col[off + mid] < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}

template <class WT>
__global__ void k_lookup(const int64_t* off, const int32_t* len, const int32_t* col, const WT* w, const u64* keys,
                         int64_t nrec, int bshift, int32_t* pos, int32_t* lb, int64_t* oldw) {
  const u64 cmask = (((u64)1) << bshift) - 1;
  GRID_STRIDE(i, nrec) {
    const int64_t row = (int64_t)(keys[i] >> bshift);
    const int32_t c = (int32_t)(keys[i] & cmask);
    const int64_t o = off[row];
    const int32_t l = len[row];
    const int32_t p = row_lower_bound(col, o, l, c);
    const bool found = p < l && col[o + p] == c;
    pos[i] = found ? p : -1;
    if (lb) lb[i] = p;
    oldw[i] = found ? (int64_t)w[o + p] : 0;
  }
}

// per record: insert / delete flags and segment heads (row changes)
__global__ void k_rec_flags(const u64* keys, const int64_t* delta, int64_t nrec, int bshift, const int32_t* pos,
                            const int64_t* oldw, int32_t* fins, int32_t* fdel, int32_t* fhead, int32_t* err) {
  GRID_STRIDE(i, nrec) {
    const bool found = pos[i] >= 0;
    const int64_t nv = (found ? oldw[i] : 0) + delta[i];
    if (nv < 0 || (!found && nv == 0)) atomicExch(err, 1);
    fins[i] = (!found && nv > 0) ? 1 : 0;
    fdel[i] = (found && nv == 0) ? 1 : 0;
    fhead[i] = (i == 0 || (keys[i] >> bshift) != (keys[i - 1] >> bshift)) ? 1 : 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    fins[nrec] = 0;
    fdel[nrec] = 0;
    fhead[nrec] = 0;
  }
}

// endpoints of the entries a record removes (rows below t.rows)
__global__ void k_track_del(const u64* keys, const int32_t* fdel, int64_t nrec, int bshift, DelTrack t) {
  const u64 cmask = (((u64)1) << bshift) - 1;
  GRID_STRIDE(i, nrec) {
    if (!fdel[i]) continue;
    const int64_t row = (int64_t)(keys[i] >> bshift);
    if (row >= t.rows) continue;
    const int32_t col = (int32_t)(keys[i] & cmask);
    // an arc between two different refined communities cannot disconnect
    // either; a parentless endpoint may have just left its community (an
    // emptied node), so such arcs are kept
    if (t.par && (row == col || (t.par[row] >= 0 && t.par[col] >= 0 && t.par[row] != t.par[col]))) continue;
    stamp_add(t.stamp, t.ep, (int32_t)row, t.list, t.cnt);
    stamp_add(t.stamp, t.ep, col, t.list, t.cnt);
  }
}

__global__ void k_seg_info(const u64* keys, int64_t nrec, int bshift, const int32_t* fhead, const int64_t* segid,
                           int64_t* seg_start, int64_t* seg_row) {
  GRID_STRIDE(i, nrec) {
    if (fhead[i]) {
      seg_start[segid[i]] = i;
      seg_row[segid[i]] = (int64_t)(keys[i] >> bshift);
    }
  }
}

// Per segment: new length, whether the row is rebuilt, relocation size.
__global__ void k_plan(const int64_t* nsegp, int64_t nrec, const int64_t* seg_start, const int64_t* seg_row,
                       const int64_t* pins, const int64_t* pdel, const int32_t* len, const int32_t* cap,
                       int32_t* newcap, int64_t* scratch_len, int64_t* work_len, int64_t* need) {
  const int64_t nseg = *nsegp;
  GRID_STRIDE(s, nseg) {
    const int64_t a = seg_start[s];
    const int64_t b = s + 1 < nseg ? seg_start[s + 1] : nrec;
    const int64_t row = seg_row[s];
    const int64_t ins = pins[b] - pins[a], del = pdel[b] - pdel[a];
    const int64_t l = len[row];
    const int64_t nl = l - del + ins;
    const bool rewrite = ins > 0 || del > 0;
    int32_t nc = 0;
    if (nl > cap[row]) {
      int64_t want = nl + (nl >> 1) + 4;
      want = (want + 3) & ~(int64_t)3;
      nc = (int32_t)want;
      atomic_add_i64(need, want);
    }
    newcap[s] = nc;
    scratch_len[s] = rewrite ? l : 0;
    work_len[s] = rewrite ? l + ins : 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    scratch_len[nseg] = 0;
    work_len[nseg] = 0;
  }
}

// weight updates in place; deleted entries get weight 0 (live weights are >= 1)
template <class WT>
__global__ void k_update(const int64_t* off, const u64* keys, const int64_t* delta, int64_t nrec, int bshift,
                         const int32_t* pos, const int64_t* oldw, WT* w) {
  GRID_STRIDE(i, nrec) {
    if (pos[i] < 0) continue;
    const int64_t row = (int64_t)(keys[i] >> bshift);
    w[off[row] + pos[i]] = (WT)(oldw[i] + delta[i]);
  }
}

// ---- undo log (batches that may be rolled back)
// Row entries: row, old offset, length and capacity, and where its old
// contents went in the content log (-1: not rewritten by this update).
__global__ void k_log_rows(int64_t nseg, const int64_t* seg_row, const int64_t* off, const int32_t* len,
                           const int32_t* cap, const int64_t* slen, const int64_t* soff, int64_t c0, int64_t* lrow,
                           int64_t* loff, int32_t* llen, int32_t* lcap, int64_t* lsrc) {
  GRID_STRIDE(s, nseg) {
    const int64_t row = seg_row[s];
    lrow[s] = row;
    loff[s] = off[row];
    llen[s] = len[row];
    lcap[s] = cap[row];
    lsrc[s] = slen[s] > 0 ? c0 + soff[s] : -1;
  }
}

// Weight entries: pool position of each record's entry (-1: absent) and
// the weight it holds before the update.
template <class WT>
__global__ void k_log_weights(const u64* keys, int64_t nrec, int bshift, const int64_t* off, const int32_t* pos,
                              const int64_t* oldw, int64_t* lpos, WT* lold) {
  GRID_STRIDE(i, nrec) {
    lpos[i] = pos[i] >= 0 ? off[(int64_t)(keys[i] >> bshift)] + pos[i] : -1;
    lold[i] = (WT)oldw[i];
  }
}

// Rollback of one row chunk: offsets, lengths and capacities come back; a
// rewritten row's old contents go back where they were when they lie in the
// batch's first pool below its first free slot (anything else was written
// into space that held no data of the state being restored).
template <class WT>
__global__ void k_undo_rows(int64_t nr, const int64_t* lrow, const int64_t* loff, const int32_t* llen,
                            const int32_t* lcap, const int64_t* lsrc, const int32_t* lcol, const WT* lw,
                            int64_t* off, int32_t* len, int32_t* cap, int32_t* col, WT* w, int restore_content,
                            int64_t top0) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < nr; i += nw) {
    const int64_t row = lrow[i], o = loff[i], src = lsrc[i];
    const int32_t l = llen[i];
    if (lane == 0) {
      off[row] = o;
      len[row] = l;
      cap[row] = lcap[i];
    }
    if (restore_content && src >= 0 && o + l <= top0)
      for (int32_t k = lane; k < l; k += 32) {
        col[o + k] = lcol[src + k];
        w[o + k] = lw[src + k];
      }
  }
}

template <class WT>
__global__ void k_undo_weights(int64_t nw, const int64_t* lpos, const WT* lold, WT* w, int64_t top0) {
  GRID_STRIDE(i, nw) {
    const int64_t p = lpos[i];
    if (p >= 0 && p < top0) w[p] = lold[i];
  }
}

__device__ inline int64_t find_seg(const int64_t* pre, int64_t nseg, int64_t t) {
  // last s with pre[s] <= t (pre is an exclusive scan, pre[0] = 0)
  int64_t lo = 0, hi = nseg;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (pre[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// last s in [lo, hi] with pre[s] <= t
__device__ inline int64_t seg_in(const int64_t* pre, int64_t lo, int64_t hi, int64_t t) {
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Items [0, total) split into segments by the exclusive scan pre.  Each warp
// takes runs of SEG_RUN consecutive items: two warp-uniform searches bound the
// run's segments, and each item then searches only that narrow range.
constexpr int SEG_RUN = 256;
#define FOR_SEG_ITEMS(t, s, pre, nseg, total)                                                       \
  const int64_t warp_ = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;                     \
  const int64_t nwarps_ = ((int64_t)gridDim.x * blockDim.x) >> 5;                                   \
  for (int64_t c0_ = warp_ * SEG_RUN; c0_ < (total); c0_ += nwarps_ * SEG_RUN) {                   \
    const int64_t c1_ = min(c0_ + SEG_RUN, (int64_t)(total)) - 1;                                   \
    const int64_t slo_ = find_seg(pre, nseg, c0_), shi_ = find_seg(pre, nseg, c1_);                 \
    for (int64_t t = c0_ + (threadIdx.x & 31); t <= c1_; t += 32) {                                 \
      const int64_t s = seg_in(pre, slo_, shi_, t);
#define END_SEG_ITEMS \
  }                   \
  }

template <class WT>
__global__ void k_copy_scratch(const int64_t* off, const int64_t* seg_row, int64_t nseg, const int64_t* soff,
                               int64_t total, const int32_t* col, const WT* w, int32_t* scol, WT* sw) {
  FOR_SEG_ITEMS(t, s, soff, nseg, total)
    const int64_t row = seg_row[s];
    const int64_t k = t - soff[s];
    scol[t] = col[off[row] + k];
    sw[t] = w[off[row] + k];
  END_SEG_ITEMS
}

__global__ void k_relocate(int64_t nseg, const int64_t* seg_row, const int32_t* newcap, int64_t* off, int32_t* cap,
                           int64_t* pool_top) {
  GRID_STRIDE(s, nseg) {
    const int32_t nc = newcap[s];
    if (nc == 0) continue;
    const int64_t row = seg_row[s];
    off[row] = (int64_t)atomicAdd((unsigned long long*)pool_top, (unsigned long long)nc);
    cap[row] = nc;
  }
}

// Rebuild of rows with inserts or deletes: item t is either a kept old entry
// (from scratch) or an inserted record; each computes its sorted position.
template <class WT>
__global__ void k_scatter_rows(int64_t nseg, int64_t nrec, const int64_t* seg_start, const int64_t* seg_row,
                               const int64_t* woff, const int64_t* soff, int64_t total, const int32_t* scol,
                               const WT* sw, const u64* keys, const int64_t* delta, const int32_t* lb,
                               const int32_t* fins, const int64_t* pins, const int64_t* pdel, int bshift,
                               const int64_t* off, int32_t* col, WT* w) {
  const u64 cmask = (((u64)1) << bshift) - 1;
  FOR_SEG_ITEMS(t, s, woff, nseg, total)
    const int64_t a = seg_start[s];
    const int64_t b = s + 1 < nseg ? seg_start[s + 1] : nrec;
    const int64_t row = seg_row[s];
    const int64_t lold = (woff[s + 1] - woff[s]) - (pins[b] - pins[a]);
    const int64_t k = t - woff[s];
    if (k < lold) {
      const int64_t i = k;
      const WT x = sw[soff[s] + i];
      if (x == 0) continue;  // deleted
      const int32_t c = scol[soff[s] + i];
      // records of this segment with a smaller column
      int64_t lo = a, hi = b;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int32_t)(keys[mid] & cmask) < c) lo = mid + 1; else hi = mid;
      }
      const int64_t dst = i - (pdel[lo] - pdel[a]) + (pins[lo] - pins[a]);
      col[off[row] + dst] = c;
      w[off[row] + dst] = x;
    } else {
      const int64_t q = k - lold;  // q-th insert of the segment
      int64_t lo = a, hi = b - 1;
      while (lo < hi) {  // first J with pins[J] - pins[a] >= q and fins[J]
        const int64_t mid = (lo + hi) >> 1;
        if (pins[mid + 1] - pins[a] <= q) lo = mid + 1; else hi = mid;
      }
      const int64_t J = lo;
      const int64_t dst = (int64_t)lb[J] - (pdel[J] - pdel[a]) + q;
      col[off[row] + dst] = (int32_t)(keys[J] & cmask);
      w[off[row] + dst] = (WT)delta[J];
      (void)fins;
    }
  END_SEG_ITEMS
}

__global__ void k_set_len(int64_t nseg, int64_t nrec, const int64_t* seg_start, const int64_t* seg_row,
                          const int64_t* pins, const int64_t* pdel, int32_t* len) {
  GRID_STRIDE(s, nseg) {
    const int64_t a = seg_start[s];
    const int64_t b = s + 1 < nseg ? seg_start[s + 1] : nrec;
    const int64_t row = seg_row[s];
    len[row] = (int32_t)(len[row] - (pdel[b] - pdel[a]) + (pins[b] - pins[a]));
  }
}

// compaction: every live entry is one item (rows located through the scan of
// the row lengths), copied to its row's new offset (the scan of the caps)
template <class WT>
__global__ void k_compact_rows(int64_t n, const int64_t* off, const int64_t* lpre, int64_t total,
                               const int64_t* noff, const int32_t* col, const WT* w, int32_t* ncol, WT* nw) {
  FOR_SEG_ITEMS(t, v, lpre, n, total)
    const int64_t k = t - lpre[v];
    ncol[noff[v] + k] = col[off[v] + k];
    nw[noff[v] + k] = w[off[v] + k];
  END_SEG_ITEMS
}

// ---------------------------------------------------------------- build
__global__ void k_count_rows(const u64* keys, int64_t nrec, int bshift, int32_t* cnt) {
  GRID_STRIDE(i, nrec) atomicAdd(&cnt[keys[i] >> bshift], 1);
}

__global__ void k_caps(const int32_t* cnt, int64_t n, int32_t* cap, int slack_pct) {
  GRID_STRIDE(v, n) {
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
  GRID_STRIDE(i, nrec) {
    const int64_t row = (int64_t)(keys[i] >> bshift);
    const int64_t p = off[row] + (i - rs[row]);
    col[p] = (int32_t)(keys[i] & cmask);
    w[p] = (WT)vals[i];
  }
}

__global__ void k_i32_to_i64(const int32_t* a, int64_t* b, int64_t n) {
  GRID_STRIDE(i, n) b[i] = a[i];
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
    k_count_rows<<<grid_for(nrec, TPB), TPB, 0, s>>>(keys, nrec, bshift, g.len.p);
    CKL("k_count_rows");
  }
  k_caps<<<grid_for(n, TPB), TPB, 0, s>>>(g.len.p, n, g.cap.p, slack_pct);
  CKL("k_caps");
  S.rs.reserve(n + 1, s);
  S.tmp64.reserve(n + 1, s);
  k_i32_to_i64<<<grid_for(n, TPB), TPB, 0, s>>>(g.len.p, S.tmp64.p, n);
  CKL("k_i32_to_i64");
  scan_exclusive(S.tmp64.p, S.rs.p, n, P, s, false);
  k_i32_to_i64<<<grid_for(n, TPB), TPB, 0, s>>>(g.cap.p, S.tmp64.p, n);
  CKL("k_i32_to_i64");
  const int64_t total = scan_exclusive(S.tmp64.p, g.off.p, n, P, s, true);
  const int64_t pool = total + total / 8 + 1024;
  g.col.release();
  g.w.release();
  g.col.exact(pool);
  g.w.exact(pool);
  g.pool_top = total;
  if (nrec > 0) {
    k_scatter_build<WT><<<grid_for(nrec, TPB), TPB, 0, s>>>(keys, vals, nrec, bshift, S.rs.p, g.off.p, g.col.p, g.w.p);
    CKL("k_scatter_build");
  }
}

template <class WT>
void csr_lookup(const SlackCSR<WT>& g, const u64* keys, int64_t nrec, int bshift, int32_t* pos, int64_t* oldw,
                CsrScratch& S, Prims& P, cudaStream_t s, int32_t* d_nseg) {
  (void)P;
  (void)S;
  (void)d_nseg;
  if (nrec <= 0) return;
  k_lookup<WT><<<grid_for(nrec, TPB), TPB, 0, s>>>(g.off.p, g.len.p, g.col.p, g.w.p, keys, nrec, bshift, pos, nullptr,
                                                   oldw);
  CKL("k_lookup");
}

// Copy every row into a fresh pool of `cap_total + extra` slots.
template <class WT>
static void compact_pool(SlackCSR<WT>& g, int64_t extra, CsrScratch& S, Prims& P, cudaStream_t s) {
  const int64_t n = g.n;
  S.tmp64.reserve(n + 1, s);
  S.rs.reserve(n + 1, s);
  k_i32_to_i64<<<grid_for(n, TPB), TPB, 0, s>>>(g.cap.p, S.tmp64.p, n);
  CKL("k_i32_to_i64");
  const int64_t total = scan_exclusive(S.tmp64.p, S.rs.p, n, P, s, true);  // new offsets
  // the same headroom again: rows that outgrow their slack move to the pool's
  // end, so a level whose rows churn refills it quickly
  const int64_t pool = 2 * (total + extra) + 4096;
  int32_t* c2 = (int32_t*)dalloc(sizeof(int32_t) * (size_t)pool);
  WT* w2 = (WT*)dalloc(sizeof(WT) * (size_t)pool);
  const int64_t live = scan_exclusive_i32(g.len.p, S.tmp64.p, n, P, s, true);
  if (live > 0) {
    k_compact_rows<WT><<<grid_for((live + 7) / 8, TPB), TPB, 0, s>>>(n, g.off.p, S.tmp64.p, live, S.rs.p, g.col.p,
                                                                     g.w.p, c2, w2);
    CKL("k_compact_rows");
  }
  if (g.logging) {  // the offset table as it was, for a rollback
    g.lofs.reserve(g.otop + n, s, true);
    CK(cudaMemcpyAsync(g.lofs.p + g.otop, g.off.p, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    g.events.push_back({true, 0, 0, 0, 0, g.otop, g.col.p});
    g.otop += n;
  }
  CK(cudaMemcpyAsync(g.off.p, S.rs.p, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  if (g.logging) {
    g.retired.emplace_back(g.col.p, g.w.p);  // freed when the batch commits
  } else {
    dfree(g.col.p);
    dfree(g.w.p);
  }
  g.col.p = c2;
  g.col.cap = pool;
  g.w.p = w2;
  g.w.cap = pool;
  g.pool_top = total;
}

template <class WT>
void csr_apply(SlackCSR<WT>& g, const u64* keys, const int64_t* delta, int64_t nrec, int bshift, CsrScratch& S,
               Prims& P, cudaStream_t s, DevScalars* d_sc, const DelTrack* trk) {
  if (nrec <= 0) return;
  S.pos.reserve(nrec + 1, s);
  S.lb.reserve(nrec + 1, s);
  S.oldw.reserve(nrec + 1, s);
  S.fins.reserve(nrec + 1, s);
  S.fdel.reserve(nrec + 1, s);
  S.fhead.reserve(nrec + 1, s);
  S.pins.reserve(nrec + 1, s);
  S.pdel.reserve(nrec + 1, s);
  S.segid.reserve(nrec + 1, s);
  const int gr = grid_for(nrec, TPB);
  k_lookup<WT><<<gr, TPB, 0, s>>>(g.off.p, g.len.p, g.col.p, g.w.p, keys, nrec, bshift, S.pos.p, S.lb.p, S.oldw.p);
  CKL("k_lookup");
  CK(cudaMemsetAsync(&d_sc->cnt[C_Z], 0, sizeof(int32_t), s));
  k_rec_flags<<<gr, TPB, 0, s>>>(keys, delta, nrec, bshift, S.pos.p, S.oldw.p, S.fins.p, S.fdel.p, S.fhead.p,
                                 &d_sc->cnt[C_Z]);
  CKL("k_rec_flags");
  if (trk) {
    k_track_del<<<gr, TPB, 0, s>>>(keys, S.fdel.p, nrec, bshift, *trk);
    CKL("k_track_del");
  }
  scan_exclusive_i32_to(S.fins.p, S.pins.p, nrec + 1, nullptr, nrec + 1, nullptr, P, s);
  scan_exclusive_i32_to(S.fdel.p, S.pdel.p, nrec + 1, nullptr, nrec + 1, nullptr, P, s);
  // the segment count stays on the device: segment arrays are sized for one
  // segment per record, and the plan and its scans read the count there
  scan_exclusive_i32_to(S.fhead.p, S.segid.p, nrec, nullptr, nrec, &d_sc->seg_n, P, s);
  S.seg.reserve(nrec + 1, s);
  S.segrow.reserve(nrec + 1, s);
  S.newcap.reserve(nrec + 1, s);
  S.slen.reserve(nrec + 2, s);
  S.wlen.reserve(nrec + 2, s);
  S.soff.reserve(nrec + 2, s);
  S.woff.reserve(nrec + 2, s);
  k_seg_info<<<gr, TPB, 0, s>>>(keys, nrec, bshift, S.fhead.p, S.segid.p, S.seg.p, S.segrow.p);
  CKL("k_seg_info");
  CK(cudaMemsetAsync(&d_sc->need, 0, sizeof(int64_t), s));
  k_plan<<<gr, TPB, 0, s>>>(&d_sc->seg_n, nrec, S.seg.p, S.segrow.p, S.pins.p, S.pdel.p, g.len.p, g.cap.p,
                            S.newcap.p, S.slen.p, S.wlen.p, &d_sc->need);
  CKL("k_plan");
  scan_exclusive_to(S.slen.p, S.soff.p, 1, &d_sc->seg_n, nrec + 1, &d_sc->seg_stot, P, s);
  scan_exclusive_to(S.wlen.p, S.woff.p, 1, &d_sc->seg_n, nrec + 1, &d_sc->seg_wtot, P, s);
  static_assert(offsetof(DevScalars, seg_stot) == offsetof(DevScalars, seg_n) + 8 &&
                    offsetof(DevScalars, seg_wtot) == offsetof(DevScalars, seg_n) + 16,
                "adjacent totals");
  int64_t tot[4] = {0, 0, 0, 0};  // need, nseg, scratch total, rebuild total
  int32_t bad = 0;
  const HostRead rr[3] = {{&d_sc->need, &tot[0], sizeof(int64_t)}, {&d_sc->seg_n, &tot[1], 3 * sizeof(int64_t)},
                          {&d_sc->cnt[C_Z], &bad, sizeof(int32_t)}};
  P.read(rr, 3, s);
  if (bad) ldl_throw(LDL_E_INVALID, "internal: adjacency update would make a weight negative");
  const int64_t need = tot[0], nseg = tot[1], stotal = tot[2], wtotal = tot[3];
  const int gs = grid_for(nseg, TPB);
  if (g.pool_top + need > g.col.cap) compact_pool<WT>(g, need, S, P, s);
  DBuf<WT>& sw = S.template sw_of<WT>();
  if (g.logging) {
    // everything a rollback needs, reserved and written before any change
    g.lrow.reserve(g.rtop + nseg + 1, s, true);
    g.loff.reserve(g.rtop + nseg + 1, s, true);
    g.lsrc.reserve(g.rtop + nseg + 1, s, true);
    g.llen.reserve(g.rtop + nseg + 1, s, true);
    g.lcap.reserve(g.rtop + nseg + 1, s, true);
    g.lpos.reserve(g.wtop + nrec + 1, s, true);
    g.lold.reserve(g.wtop + nrec + 1, s, true);
    g.lcol.reserve(g.ctop + stotal + 1, s, true);
    g.lw.reserve(g.ctop + stotal + 1, s, true);
    if (nseg > 0) {
      k_log_rows<<<gs, TPB, 0, s>>>(nseg, S.segrow.p, g.off.p, g.len.p, g.cap.p, S.slen.p, S.soff.p, g.ctop,
                                    g.lrow.p + g.rtop, g.loff.p + g.rtop, g.llen.p + g.rtop, g.lcap.p + g.rtop,
                                    g.lsrc.p + g.rtop);
      CKL("k_log_rows");
    }
    k_log_weights<WT><<<gr, TPB, 0, s>>>(keys, nrec, bshift, g.off.p, S.pos.p, S.oldw.p, g.lpos.p + g.wtop,
                                         g.lold.p + g.wtop);
    CKL("k_log_weights");
    g.events.push_back({false, g.rtop, nseg, g.wtop, nrec, 0, g.col.p});
    g.rtop += nseg;
    g.wtop += nrec;
  }
  k_update<WT><<<gr, TPB, 0, s>>>(g.off.p, keys, delta, nrec, bshift, S.pos.p, S.oldw.p, g.w.p);
  CKL("k_update");
  if (wtotal > 0) {
    // the rows to rebuild, as they are before the rewrite (weights already
    // updated): while a batch is logged they go straight into the undo log,
    // which the rebuild then reads
    int32_t* scol = nullptr;
    WT* swp = nullptr;
    if (g.logging) {
      scol = g.lcol.p + g.ctop;
      swp = g.lw.p + g.ctop;
      g.ctop += stotal;
    } else {
      S.scol.reserve(stotal + 1, s);
      sw.reserve(stotal + 1, s);
      scol = S.scol.p;
      swp = sw.p;
    }
    if (stotal > 0) {
      k_copy_scratch<WT><<<grid_for((stotal + 7) / 8, TPB), TPB, 0, s>>>(g.off.p, S.segrow.p, nseg, S.soff.p, stotal,
                                                                         g.col.p, g.w.p, scol, swp);
      CKL("k_copy_scratch");
    }
    if (need > 0) {
      CK(cudaMemcpyAsync(&d_sc->pool_top, &g.pool_top, sizeof(int64_t), cudaMemcpyHostToDevice, s));
      k_relocate<<<gs, TPB, 0, s>>>(nseg, S.segrow.p, S.newcap.p, g.off.p, g.cap.p, &d_sc->pool_top);
      CKL("k_relocate");
      g.pool_top += need;
    }
    k_scatter_rows<WT><<<grid_for((wtotal + 7) / 8, TPB), TPB, 0, s>>>(nseg, nrec, S.seg.p, S.segrow.p, S.woff.p, S.soff.p,
                                                             wtotal, scol, swp, keys, delta, S.lb.p, S.fins.p,
                                                             S.pins.p, S.pdel.p, bshift, g.off.p, g.col.p, g.w.p);
    CKL("k_scatter_rows");
    k_set_len<<<gs, TPB, 0, s>>>(nseg, nrec, S.seg.p, S.segrow.p, S.pins.p, S.pdel.p, g.len.p);
    CKL("k_set_len");
  }
}

template <class WT>
void csr_txn_begin(SlackCSR<WT>& g) {
  g.logging = true;
  g.col0 = g.col.p;
  g.w0 = g.w.p;
  g.cap0 = g.col.cap;
  g.top0 = g.pool_top;
  g.retired.clear();
  g.events.clear();
  g.rtop = g.wtop = g.ctop = g.otop = 0;
}

template <class WT>
void csr_txn_commit(SlackCSR<WT>& g, cudaStream_t s) {
  if (!g.retired.empty()) {
    CK(cudaStreamSynchronize(s));
    for (auto& x : g.retired) {
      dfree(x.first);
      dfree(x.second);
    }
  }
  g.retired.clear();
  g.events.clear();
  g.logging = false;
}

template <class WT>
cudaError_t csr_txn_rollback(SlackCSR<WT>& g, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  // undo in reverse order; contents go back only into the batch's first pool
  for (size_t k = g.events.size(); k-- > 0 && e == cudaSuccess;) {
    const auto& ev = g.events[k];
    if (ev.offsets) {
      e = cudaMemcpyAsync(g.off.p, g.lofs.p + ev.o0, sizeof(int64_t) * (size_t)g.n, cudaMemcpyDeviceToDevice, s);
      continue;
    }
    const int restore = ev.col == g.col0 ? 1 : 0;
    if (ev.nr > 0) {
      const int grid = (int)std::min<int64_t>((ev.nr + 7) / 8, 4096);
      k_undo_rows<WT><<<grid, TPB, 0, s>>>(ev.nr, g.lrow.p + ev.r0, g.loff.p + ev.r0, g.llen.p + ev.r0,
                                           g.lcap.p + ev.r0, g.lsrc.p + ev.r0, g.lcol.p, g.lw.p, g.off.p, g.len.p,
                                           g.cap.p, g.col0, g.w0, restore, g.top0);
      g_launches.fetch_add(1, std::memory_order_relaxed);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess && restore && ev.nw > 0) {
      const int grid = (int)std::min<int64_t>((ev.nw + TPB - 1) / TPB, 4096);
      k_undo_weights<WT><<<grid, TPB, 0, s>>>(ev.nw, g.lpos.p + ev.w0, g.lold.p + ev.w0, g.w0, g.top0);
      g_launches.fetch_add(1, std::memory_order_relaxed);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  // back to the first pool; pools made during the batch go
  auto drop = [&](int32_t* cp, WT* wp) {
    if (cp != g.col0) dfree(cp);
    if (wp != g.w0) dfree(wp);
  };
  drop(g.col.p, g.w.p);
  for (auto& x : g.retired) drop(x.first, x.second);
  g.retired.clear();
  g.col.p = g.col0;
  g.w.p = g.w0;
  g.col.cap = g.w.cap = g.cap0;
  g.pool_top = g.top0;
  g.events.clear();
  g.logging = false;
  return e;
}

template void csr_txn_begin<int32_t>(SlackCSR<int32_t>&);
template void csr_txn_begin<int64_t>(SlackCSR<int64_t>&);
template void csr_txn_commit<int32_t>(SlackCSR<int32_t>&, cudaStream_t);
template void csr_txn_commit<int64_t>(SlackCSR<int64_t>&, cudaStream_t);
template cudaError_t csr_txn_rollback<int32_t>(SlackCSR<int32_t>&, cudaStream_t);
template cudaError_t csr_txn_rollback<int64_t>(SlackCSR<int64_t>&, cudaStream_t);

template void csr_build<int32_t>(SlackCSR<int32_t>&, int64_t, const u64*, const int64_t*, int64_t, int, int,
                                 CsrScratch&, Prims&, cudaStream_t);
template void csr_build<int64_t>(SlackCSR<int64_t>&, int64_t, const u64*, const int64_t*, int64_t, int, int,
                                 CsrScratch&, Prims&, cudaStream_t);
template void csr_lookup<int32_t>(const SlackCSR<int32_t>&, const u64*, int64_t, int, int32_t*, int64_t*,
                                  CsrScratch&, Prims&, cudaStream_t, int32_t*);
template void csr_lookup<int64_t>(const SlackCSR<int64_t>&, const u64*, int64_t, int, int32_t*, int64_t*,
                                  CsrScratch&, Prims&, cudaStream_t, int32_t*);
template void csr_apply<int32_t>(SlackCSR<int32_t>&, const u64*, const int64_t*, int64_t, int, CsrScratch&, Prims&,
                                 cudaStream_t, DevScalars*, const DelTrack*);
template void csr_apply<int64_t>(SlackCSR<int64_t>&, const u64*, const int64_t*, int64_t, int, CsrScratch&, Prims&,
                                 cudaStream_t, DevScalars*, const DelTrack*);
