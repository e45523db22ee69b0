// Load-balanced iteration over the rows of a node list.
//
// Every listed node is split into chunks of CH adjacency entries (out-row
// chunks first, then in-row chunks); a node with empty rows still gets one
// chunk so that per-node work has a place to run.  An exclusive scan of the
// chunk counts maps a global chunk id back to (node, row, range) by binary
// search, so a hub row is spread over many warps instead of one.
#pragma once
#include "ctx.cuh"

constexpr int CH = 256;

struct ChunkMap {
  const int32_t* list;   // nodes
  const int64_t* pre;    // exclusive scan of chunk counts, length n_hint + 1
  int64_t n_hint;        // list capacity used for the scan
  const int32_t* len_a;  // first row lengths (out)
  const int32_t* len_b;  // second row lengths (in) or nullptr
};

struct Chunk {
  int64_t idx;    // position in the list
  int32_t v;      // node
  int32_t first;  // 1 for the node's first chunk
  int32_t row;    // 0: first row, 1: second row, -1: none
  int32_t k0, k1; // entry range in that row
};

__device__ inline Chunk chunk_of(const ChunkMap& m, int64_t c) {
  int64_t lo = 0, hi = m.n_hint;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (m.pre[mid] <= c) lo = mid; else hi = mid;
  }
  Chunk r;
  r.idx = lo;
  r.v = m.list[lo];
  const int64_t j = c - m.pre[lo];
  r.first = j == 0;
  const int32_t la = m.len_a[r.v];
  const int32_t lb = m.len_b ? m.len_b[r.v] : 0;
  const int64_t ca = (la + CH - 1) / CH;
  if (j < ca) {
    r.row = 0;
    r.k0 = (int32_t)(j * CH);
    r.k1 = min(la, r.k0 + CH);
  } else if (lb > 0) {
    r.row = 1;
    r.k0 = (int32_t)((j - ca) * CH);
    r.k1 = min(lb, r.k0 + CH);
  } else {
    r.row = -1;
    r.k0 = r.k1 = 0;
  }
  return r;
}

// Builds m.pre for `list` (device count *nlist <= n_hint); returns the map.
// The total chunk count is left at pre[n_hint] on the device (no sync).
ChunkMap chunk_map(ldl_ctx& c, const int32_t* list, const int32_t* nlist, int64_t n_hint, const int32_t* len_a,
                   const int32_t* len_b);
