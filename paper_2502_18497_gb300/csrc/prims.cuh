// Declarations of the device primitives (prims.cu).
#pragma once
#include "common.cuh"

struct Prims {  // scratch owned by a context
  DBuf<int64_t> bsum, hist, pos, usum;
  DBuf<int32_t> flag;
  DBuf<u64> lb_st;       // look-back scan: per-tile state words
  DBuf<int32_t> lb_ctl;  // look-back scan: 256 epoch tile counters, then the error flag
  uint32_t lb_ep = 0;
  // how totals reach the host (nullptr: a copy and a stream synchronisation)
  HostReadFn rd = nullptr;
  void* rd_owner = nullptr;
  void read(const HostRead* r, int n, cudaStream_t s) {
    if (rd) {
      rd(rd_owner, r, n);
      return;
    }
    for (int i = 0; i < n; ++i) CK(cudaMemcpyAsync(r[i].dst, r[i].src, (size_t)r[i].bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  void release() {
    bsum.release(); hist.release(); pos.release(); usum.release();
    flag.release(); lb_st.release(); lb_ctl.release();
    lb_ep = 0;
  }
};

// out[i] = sum of in[0..i); returns the total when want_total (synchronises).
int64_t scan_exclusive(const int64_t* in, int64_t* out, int64_t n, Prims& P, cudaStream_t s, bool want_total);
int64_t scan_exclusive_i32(const int32_t* in, int64_t* out, int64_t n, Prims& P, cudaStream_t s, bool want_total);
// The same without a host read: the length is n, or *n_dev + n when n_dev is
// given (then n_max bounds it and sizes the launch); the total is written to
// total_dev (device) when that is not null.
void scan_exclusive_to(const int64_t* in, int64_t* out, int64_t n, const int64_t* n_dev, int64_t n_max,
                       int64_t* total_dev, Prims& P, cudaStream_t s);
void scan_exclusive_i32_to(const int32_t* in, int64_t* out, int64_t n, const int64_t* n_dev, int64_t n_max,
                           int64_t* total_dev, Prims& P, cudaStream_t s);
// Exclusive scan (n_hint + 1 entries) of the chunk counts of the listed nodes:
// entry i < *nlist is ceil(la[v] / chunk) + ceil(lb[v] / chunk) for v =
// list[i] (at least 1), later entries 0.  No host read.
void scan_chunk_counts(const int32_t* list, const int32_t* nlist, int64_t n_hint, const int32_t* la,
                       const int32_t* lb, int32_t chunk, int64_t* out, Prims& P, cudaStream_t s);
// Device flag set when a scan's bounded look-back wait gave up (nullptr
// before the first multi-tile scan).
int32_t* scan_error_flag(Prims& P);
// Runs a scan whose first tile is never published; true when the waiting tile
// gave up and raised the error flag (a check of the bounded wait).
bool scan_wait_gives_up(cudaStream_t s);

// Stable LSD radix sort of n (key, value) pairs on the low `bits` key bits,
// 8 bits per pass.  The sorted data ends in (keys, vals); the pointers are
// swapped with (tk, tv) as the passes ping-pong.
// Only key bits [lo_bit, bits) are sorted on (the order of keys equal there is kept).
void radix_sort_pairs(u64*& keys, u64*& vals, u64*& tk, u64*& tv, int64_t n, int bits, Prims& P, cudaStream_t s,
                      int lo_bit = 0);

// Sorted keys -> unique keys with the int64 sum of their values, zero sums
// dropped, order kept.  Returns the number of output pairs (synchronises).
int64_t reduce_by_key(const u64* keys, const u64* vals, int64_t n, u64* okeys, int64_t* ovals, Prims& P,
                      cudaStream_t s);

// flag[i] = 1 where keys[i] differs from keys[i-1] (or i == 0)
void heads_launch(const u64* keys, int64_t n, int32_t* flag, cudaStream_t s);

template <class T>
inline void swap_buf(DBuf<T>& a, DBuf<T>& b) {
  DBuf<T> t = a;
  a = b;
  b = t;
}

// Sort the first n pairs of (k, v) in place (by DBuf identity) using (tk, tv).
inline void sort_pairs(DBuf<u64>& k, DBuf<u64>& v, DBuf<u64>& tk, DBuf<u64>& tv, int64_t n, int bits, Prims& P,
                       cudaStream_t s, int lo_bit = 0) {
  tk.reserve(n, s);
  tv.reserve(n, s);
  u64 *kp = k.p, *vp = v.p, *tkp = tk.p, *tvp = tv.p;
  radix_sort_pairs(kp, vp, tkp, tvp, n, bits, P, s, lo_bit);
  if (kp != k.p) {
    swap_buf(k, tk);
    swap_buf(v, tv);
  }
}

inline int bits_for(int64_t n) {  // bits to hold values in [0, n)
  int b = 0;
  while (((int64_t)1 << b) < n) ++b;
  return b;
}
