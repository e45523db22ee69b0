// Chunk maps for load-balanced row iteration (see chunks.cuh).
#include "chunks.cuh"
#include "prims.cuh"


ChunkMap chunk_map(ldl_ctx& c, const int32_t* list, const int32_t* nlist, int64_t n_hint, const int32_t* len_a,
                   const int32_t* len_b) {
  // the chunk counts are computed inside the scan
  c.chunk_pre.reserve(n_hint + 2, c.s);
  scan_chunk_counts(list, nlist, n_hint, len_a, len_b, CH, c.chunk_pre.p, c.P, c.s);
  return ChunkMap{list, c.chunk_pre.p, n_hint, len_a, len_b};
}
