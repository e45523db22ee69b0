// Declarations of the slack-CSR operations (csr.cu).
#pragma once
#include "common.cuh"
#include "prims.cuh"

struct CsrScratch {
  DBuf<int64_t> seg, segrow, oldw, rs, tmp64, pins, pdel, segid, slen, wlen, soff, woff;
  DBuf<int32_t> pos, lb, newcap, fins, fdel, fhead, scol, sw32;
  DBuf<int64_t> sw64;
  template <class WT>
  DBuf<WT>& sw_of();
  void release() {
    DBuf<int64_t>* a[] = {&seg, &segrow, &oldw, &rs, &tmp64, &pins, &pdel, &segid, &slen, &wlen, &soff, &woff,
                          &sw64};
    for (auto* b : a) b->release();
    DBuf<int32_t>* c[] = {&pos, &lb, &newcap, &fins, &fdel, &fhead, &scol, &sw32};
    for (auto* b : c) b->release();
  }
};
template <>
inline DBuf<int32_t>& CsrScratch::sw_of<int32_t>() { return sw32; }
template <>
inline DBuf<int64_t>& CsrScratch::sw_of<int64_t>() { return sw64; }

// Build g over rows [0,n) from sorted unique records (key = row<<bshift|col,
// vals = weights), with slack_pct percent spare capacity per row.
template <class WT>
void csr_build(SlackCSR<WT>& g, int64_t n, const u64* keys, const int64_t* vals, int64_t nrec, int bshift,
               int slack_pct, CsrScratch& S, Prims& P, cudaStream_t s);

// For each sorted unique record key: pos[i] = entry index in its row (or -1)
// and oldw[i] = current weight (or 0).  d_nseg is a device counter.
template <class WT>
void csr_lookup(const SlackCSR<WT>& g, const u64* keys, int64_t nrec, int bshift, int32_t* pos, int64_t* oldw,
                CsrScratch& S, Prims& P, cudaStream_t s, int32_t* d_nseg);

// Where csr_apply records the endpoints (row and column) of the entries it
// removes, for records whose row is below `rows`: a dedup stamp with its
// epoch, a list and its device counter.
struct DelTrack {
  int32_t* stamp;
  int32_t ep;
  int32_t* list;
  int32_t* cnt;
  int64_t rows;
  const int32_t* par;  // with it, arcs between two different parents are not recorded
};

// Batch transactions on a CSR (see SlackCSR's undo log): begin logging,
// commit (free pools replaced during the batch), or roll back to the state
// at begin.  Rollback only copies (no allocation) and synchronises s.
template <class WT>
void csr_txn_begin(SlackCSR<WT>& g);
template <class WT>
void csr_txn_commit(SlackCSR<WT>& g, cudaStream_t s);
template <class WT>
cudaError_t csr_txn_rollback(SlackCSR<WT>& g, cudaStream_t s);

// Add delta to each record's entry: absent entries are inserted, entries that
// reach zero are removed (their endpoints go to *trk when given).
// Synchronises once (pool growth decision).
template <class WT>
void csr_apply(SlackCSR<WT>& g, const u64* keys, const int64_t* delta, int64_t nrec, int bshift, CsrScratch& S,
               Prims& P, cudaStream_t s, DevScalars* d_sc, const DelTrack* trk = nullptr);
