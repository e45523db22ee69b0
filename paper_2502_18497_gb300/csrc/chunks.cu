// Chunk maps for load-balanced row iteration (see chunks.cuh).
#include "chunks.cuh"
#include "prims.cuh"

namespace {

__global__ void k_chunk_counts(const int32_t* list, const int32_t* nlist, int64_t n_hint, const int32_t* la,
                               const int32_t* lb, int64_t* cnt) {
  const int32_t n = *nlist;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n_hint; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = 0;
    if (i < n && i < n_hint) {
      const int32_t v = list[i];
      c = (la[v] + CH - 1) / CH + (lb ? (lb[v] + CH - 1) / CH : 0);
      if (c == 0) c = 1;
    }
    cnt[i] = c;
  }
}

}  // namespace

ChunkMap chunk_map(ldl_ctx& c, const int32_t* list, const int32_t* nlist, int64_t n_hint, const int32_t* len_a,
                   const int32_t* len_b) {
  c.chunk_cnt.reserve(n_hint + 2, c.s);
  c.chunk_pre.reserve(n_hint + 2, c.s);
  k_chunk_counts<<<grid_for(n_hint + 1, 256), 256, 0, c.s>>>(list, nlist, n_hint, len_a, len_b, c.chunk_cnt.p);
  CKL("k_chunk_counts");
  scan_exclusive(c.chunk_cnt.p, c.chunk_pre.p, n_hint + 1, c.P, c.s, false);
  return ChunkMap{list, c.chunk_pre.p, n_hint, len_a, len_b};
}
