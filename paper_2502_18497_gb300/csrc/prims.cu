// Device primitives: exclusive scan, stable LSD radix sort of (key, value)
// pairs, and reduce-by-key of sorted pairs.  Hand-written; no library sort.
#include <cooperative_groups.h>

#include <algorithm>

#include "prims.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 4;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

__device__ inline int64_t block_excl_scan_i64(int64_t v, int64_t* total) {
  __shared__ int64_t wsum[SC_THREADS / WARP];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = v;
  for (int d = 1; d < 32; d <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t s = lane < SC_THREADS / WARP ? wsum[lane] : 0;
    for (int d = 1; d < 32; d <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= d) s += y;
    }
    if (lane < SC_THREADS / WARP) wsum[lane] = s;
  }
  __syncthreads();
  int64_t before = wid ? wsum[wid - 1] : 0;
  *total = wsum[SC_THREADS / WARP - 1];
  __syncthreads();
  return before + x - v;
}

// Scan inputs: an array, or the chunk count of each node of a list
// (chunks.cuh: ceil(len / chunk) per row, at least 1 per listed node, 0 past
// the list's device-side count).
template <class T>
struct ArrayIn {
  const T* p;
  __device__ int64_t operator()(int64_t i) const { return (int64_t)p[i]; }
};

struct ChunkCountIn {
  const int32_t* list;
  const int32_t* nlist;
  int64_t n_hint;
  const int32_t* la;
  const int32_t* lb;
  int32_t chunk;
  __device__ int64_t operator()(int64_t i) const {
    if (i >= n_hint || i >= *nlist) return 0;
    const int32_t v = list[i];
    const int64_t c = (la[v] + chunk - 1) / chunk + (lb ? (lb[v] + chunk - 1) / chunk : 0);
    return c > 0 ? c : 1;
  }
};

// whole input in one tile: scan and total in one launch
template <class In>
__global__ void k_scan_one(In in, int64_t* out, int64_t n, const int64_t* n_dev, int64_t* total) {
  if (n_dev) n += *n_dev;
  const int64_t base = (int64_t)threadIdx.x * SC_ITEMS;
  int64_t loc[SC_ITEMS];
  int64_t s = 0;
  for (int k = 0; k < SC_ITEMS; ++k) {
    int64_t i = base + k;
    loc[k] = i < n ? in(i) : 0;
    s += loc[k];
  }
  int64_t tot;
  int64_t pre = block_excl_scan_i64(s, &tot);
  for (int k = 0; k < SC_ITEMS; ++k) {
    int64_t i = base + k;
    if (i < n) out[i] = pre;
    pre += loc[k];
  }
  if (threadIdx.x == 0 && total) *total = tot;
}

// Single-pass scan with decoupled look-back.  Tiles are claimed in order
// from a counter, so a tile only waits on tiles claimed before it, and every
// tile publishes its own aggregate before it waits: the waits always end.
// A tile's state word packs (value << 10 | epoch << 2 | status) with status
// 1 = tile aggregate, 2 = inclusive prefix; words of another epoch (an
// earlier scan) read as not ready.  Inputs are non-negative counts below
// 2^53.  The wait is bounded all the same: past LB_SPINS polls the tile sets
// *err and carries on (the host turns the flag into LDL_E_TIMEOUT).
constexpr int LB_ITEMS = 8;
constexpr int LB_TILE = SC_THREADS * LB_ITEMS;
constexpr uint32_t LB_SPINS = 1u << 20;

template <class In>
__global__ void __launch_bounds__(SC_THREADS) k_scan_lb(In in, int64_t* out, int64_t n, const int64_t* n_dev,
                                                        u64* st, int32_t* ctr, uint32_t ep, int64_t* total,
                                                        int32_t* err) {
  __shared__ int64_t s_tile, s_pre;
  if (n_dev) n += *n_dev;  // launched for an upper bound; tiles past n leave at once
  if (threadIdx.x == 0) s_tile = atomicAdd(ctr, 1);
  __syncthreads();
  const int64_t tile = s_tile;
  if (tile * LB_TILE >= n && tile > 0) return;
  const int64_t base = tile * LB_TILE + (int64_t)threadIdx.x * LB_ITEMS;
  int64_t loc[LB_ITEMS];
  int64_t sum = 0;
  for (int k = 0; k < LB_ITEMS; ++k) {
    const int64_t i = base + k;
    loc[k] = i < n ? in(i) : 0;
    sum += loc[k];
  }
  int64_t agg;
  const int64_t pre = block_excl_scan_i64(sum, &agg);
  if (threadIdx.x < 32) {
    // warp 0 looks back over 32 predecessors at a time: it sums aggregates
    // until the nearest inclusive prefix, waiting only for tiles before it
    const int lane = threadIdx.x;
    const u64 tag = (u64)(ep & 255u) << 2;
    int64_t acc = 0;
    if (tile > 0) {
      if (lane == 0) atomicExch((unsigned long long*)&st[tile], ((u64)agg << 10) | tag | 1u);
      uint32_t spins = 0;
      for (int64_t j0 = tile - 1;;) {
        const int64_t j = j0 - lane;
        u64 x = 0;
        if (j >= 0) x = *(volatile const u64*)&st[j];
        const bool ready = j < 0 || (((x >> 2) & 255u) == (ep & 255u) && (x & 3u) != 0);
        const unsigned rmask = __ballot_sync(0xffffffffu, ready);
        const unsigned pmask = __ballot_sync(0xffffffffu, j >= 0 && ready && (x & 3u) == 2u);
        const int nr = rmask == 0xffffffffu ? 32 : __ffs(~rmask) - 1;  // nearest tile not ready
        const int fp = pmask ? __ffs(pmask) - 1 : 32;                  // nearest inclusive prefix
        if (fp < nr || nr == 32) {
          const int upto = fp < 32 ? fp : 31;
          const int64_t v = (j >= 0 && lane <= upto) ? (int64_t)(x >> 10) : 0;
          acc += warp_sum_i64(v);
          acc = __shfl_sync(0xffffffffu, acc, 0);
          if (fp < 32) break;
          j0 -= 32;
          continue;
        }
        if (++spins > LB_SPINS) {
          if (lane == 0) atomicExch(err, 1);
          break;
        }
        __nanosleep(32);
      }
    }
    if (lane == 0) {
      atomicExch((unsigned long long*)&st[tile], ((u64)(acc + agg) << 10) | tag | 2u);
      s_pre = acc;
      if ((tile + 1) * LB_TILE >= n && total) *total = acc + agg;
    }
  }
  __syncthreads();
  int64_t p = s_pre + pre;
  for (int k = 0; k < LB_ITEMS; ++k) {
    const int64_t i = base + k;
    if (i < n) out[i] = p;
    p += loc[k];
  }
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
static_assert(RS_THREADS == 256 && SC_THREADS == 256, "one thread per digit");

// Digit histogram of tile b (RS_TILE keys from b * RS_TILE) into column b
// of ghist (digit-major: ghist[d * nb + b]).
__device__ inline void rs_hist_tile(const u64* keys, int64_t n, int shift, int64_t nb, int64_t* ghist, int64_t b) {
  __shared__ uint32_t h[256];
  for (int i = threadIdx.x; i < 256; i += RS_THREADS) h[i] = 0;
  const int lane = threadIdx.x & 31;
  const int64_t base = b * RS_TILE;
  int d[RS_ITEMS];
  for (int k = 0; k < RS_ITEMS; ++k) {  // all loads in flight before any shuffle
    const int64_t i = base + (int64_t)k * RS_THREADS + threadIdx.x;
    d[k] = i < n ? (int)((keys[i] >> shift) & 255) : 256;
  }
  __syncthreads();
  for (int k = 0; k < RS_ITEMS; ++k) {
    // one shared atomic per distinct digit of the warp (skewed digits collide)
    const unsigned peers = __match_any_sync(0xffffffffu, d[k]);
    if (d[k] < 256 && lane == __ffs(peers) - 1) atomicAdd(&h[d[k]], (uint32_t)__popc(peers));
  }
  __syncthreads();
  for (int x = threadIdx.x; x < 256; x += RS_THREADS) ghist[(int64_t)x * nb + b] = h[x];
  __syncthreads();  // h is reset by the block's next tile
}

__global__ void k_rs_hist(const u64* keys, int64_t n, int shift, int64_t nb, int64_t* ghist) {
  rs_hist_tile(keys, n, shift, nb, ghist, blockIdx.x);
}

// One block per digit: exclusive scan of the digit's tile counts in place
// (8 consecutive counts per thread per step), and the digit's total.
__device__ inline void rs_dscan_digit(int64_t* ghist, int64_t nb, int64_t* dtot, int d) {
  constexpr int IT = 8;
  int64_t* row = ghist + (int64_t)d * nb;
  int64_t carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += SC_THREADS * IT) {
    const int64_t base = b0 + (int64_t)threadIdx.x * IT;
    int64_t v[IT];
    int64_t sum = 0;
    for (int k = 0; k < IT; ++k) {
      v[k] = base + k < nb ? row[base + k] : 0;
      sum += v[k];
    }
    int64_t total;
    int64_t ex = carry + block_excl_scan_i64(sum, &total);
    for (int k = 0; k < IT; ++k) {
      if (base + k < nb) row[base + k] = ex;
      ex += v[k];
    }
    carry += total;
  }
  if (threadIdx.x == 0) dtot[d] = carry;
}

__global__ void __launch_bounds__(SC_THREADS) k_rs_dscan(int64_t* ghist, int64_t nb, int64_t* dtot) {
  rs_dscan_digit(ghist, nb, dtot, blockIdx.x);
}

// One tile of RS_TILE pairs per block.  Each warp ranks a contiguous sub-tile
// of RS_ITEMS * 32 pairs (rounds of 32, stable), the block turns the warp
// counts into digit-sorted positions inside the tile, the tile is staged in
// shared memory in digit order, and consecutive threads then write
// consecutive output slots of each digit.  The global start of (digit d,
// tile b) is the exclusive prefix of the digit totals dtot at d plus the
// per-digit scanned tile count goff[d * nb + b].
__device__ inline void rs_scatter_tile(const u64* keys, const u64* vals, u64* okeys, u64* ovals, int64_t n, int shift,
                                       int64_t nb, const int64_t* goff, const int64_t* dtot, int64_t b) {
  constexpr int NW = RS_THREADS / WARP;
  __shared__ int32_t whist[NW][256];  // per-warp digit counts, then per-warp exclusive bases
  __shared__ int32_t tstart[256];     // tile-local start of each digit
  __shared__ int64_t gstart[256];     // global start of each digit for this tile
  __shared__ u64 sk[RS_TILE];
  __shared__ u64 sv[RS_TILE];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t base = b * RS_TILE;
  const int tile_n = (int)min((int64_t)RS_TILE, n - base);
  for (int d = lane; d < 256; d += 32) whist[wid][d] = 0;
  {
    int64_t total;
    const int64_t dbase = block_excl_scan_i64(dtot[tid], &total);  // RS_THREADS == 256 digits
    gstart[tid] = dbase + goff[(int64_t)tid * nb + b];
  }
  u64 key[RS_ITEMS], val[RS_ITEMS];
  int rk[RS_ITEMS];
  for (int k = 0; k < RS_ITEMS; ++k) {
    const int li = wid * (RS_ITEMS * 32) + k * 32 + lane;
    const bool valid = li < tile_n;
    key[k] = valid ? keys[base + li] : 0;
    val[k] = valid ? vals[base + li] : 0;
  }
  for (int k = 0; k < RS_ITEMS; ++k) {
    const int li = wid * (RS_ITEMS * 32) + k * 32 + lane;
    const int d = li < tile_n ? (int)((key[k] >> shift) & 255) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int before = d < 256 ? whist[wid][d] : 0;
    rk[k] = before + __popc(peers & ((1u << lane) - 1u));
    __syncwarp();
    if (d < 256 && lane == __ffs(peers) - 1) whist[wid][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // thread d: exclusive scan of digit d over the warps, then over the digits
  int cnt = 0;
  {
    const int d = tid;  // RS_THREADS == 256
    for (int w = 0; w < NW; ++w) {
      const int c = whist[w][d];
      whist[w][d] = cnt;
      cnt += c;
    }
  }
  int64_t total;
  const int64_t ds = block_excl_scan_i64(cnt, &total);
  tstart[tid] = (int32_t)ds;
  __syncthreads();
  for (int k = 0; k < RS_ITEMS; ++k) {
    const int li = wid * (RS_ITEMS * 32) + k * 32 + lane;
    if (li < tile_n) {
      const int d = (int)((key[k] >> shift) & 255);
      const int p = tstart[d] + whist[wid][d] + rk[k];
      sk[p] = key[k];
      sv[p] = val[k];
    }
  }
  __syncthreads();
  for (int j = tid; j < tile_n; j += RS_THREADS) {
    const u64 k = sk[j];
    const int d = (int)((k >> shift) & 255);
    const int64_t p = gstart[d] + (j - tstart[d]);
    okeys[p] = k;
    ovals[p] = sv[j];
  }
  __syncthreads();  // the tile buffers are reused by the caller's next tile
}

__global__ void __launch_bounds__(RS_THREADS, 4) k_rs_scatter(const u64* keys, const u64* vals, u64* okeys,
                                                              u64* ovals, int64_t n, int shift, int64_t nb,
                                                              const int64_t* goff, const int64_t* dtot) {
  rs_scatter_tile(keys, vals, okeys, ovals, n, shift, nb, goff, dtot, blockIdx.x);
}

// The whole multi-tile sort in one cooperative launch (all nb tiles'
// blocks co-resident): per 8-bit pass the tile histograms, the per-digit
// scans over tiles and the scatter, separated by grid barriers, ping-ponging
// between (keys, vals) and (tk, tv).  Replaces three launches per pass.
__global__ void __launch_bounds__(RS_THREADS, 4) k_rs_coop(u64* keys, u64* vals, u64* tk, u64* tv, int64_t n,
                                                           int lo_bit, int bits, int64_t nb, int64_t* ghist,
                                                           int64_t* dtot) {
  cg::grid_group grid = cg::this_grid();
  u64 *ik = keys, *iv = vals, *ok = tk, *ov = tv;
  for (int shift = lo_bit; shift < bits; shift += 8) {
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) rs_hist_tile(ik, n, shift, nb, ghist, b);
    grid.sync();
    for (int d = blockIdx.x; d < 256; d += gridDim.x) rs_dscan_digit(ghist, nb, dtot, d);
    grid.sync();
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) rs_scatter_tile(ik, iv, ok, ov, n, shift, nb, ghist, dtot, b);
    grid.sync();
    u64* t = ik; ik = ok; ok = t;
    t = iv; iv = ov; ov = t;
  }
}

// Whole sort in one block (n <= RS_TILE).  Each thread holds RS_ITEMS pairs
// in registers across the passes: per 8-bit pass every warp ranks its
// contiguous sub-tile (rounds of 32, stable), the block turns the per-warp
// digit counts into positions, the pairs are placed in shared memory in
// digit order and read back in the same warp-contiguous layout.
__global__ void __launch_bounds__(RS_THREADS) k_rs_small(u64* keys, u64* vals, int n, int lo_bit, int bits) {
  constexpr int NW = RS_THREADS / WARP;
  __shared__ int32_t whist[NW][256];
  __shared__ int32_t tstart[256];
  __shared__ u64 sk[RS_TILE];
  __shared__ u64 sv[RS_TILE];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  u64 key[RS_ITEMS], val[RS_ITEMS];
  for (int k = 0; k < RS_ITEMS; ++k) {
    const int li = wid * (RS_ITEMS * 32) + k * 32 + lane;
    key[k] = li < n ? keys[li] : 0;
    val[k] = li < n ? vals[li] : 0;
  }
  for (int shift = lo_bit; shift < bits; shift += 8) {
    for (int d = lane; d < 256; d += 32) whist[wid][d] = 0;
    __syncwarp();
    int rk[RS_ITEMS];
    for (int k = 0; k < RS_ITEMS; ++k) {
      const int li = wid * (RS_ITEMS * 32) + k * 32 + lane;
      const int d = li < n ? (int)((key[k] >> shift) & 255) : 256;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const int before = d < 256 ? whist[wid][d] : 0;
      rk[k] = before + __popc(peers & ((1u << lane) - 1u));
      __syncwarp();
      if (d < 256 && lane == __ffs(peers) - 1) whist[wid][d] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    int cnt = 0;
    for (int w = 0; w < NW; ++w) {  // thread = digit (RS_THREADS == 256)
      const int c = whist[w][tid];
      whist[w][tid] = cnt;
      cnt += c;
    }
    int64_t total;
    tstart[tid] = (int32_t)block_excl_scan_i64(cnt, &total);
    __syncthreads();
    for (int k = 0; k < RS_ITEMS; ++k) {
      const int li = wid * (RS_ITEMS * 32) + k * 32 + lane;
      if (li < n) {
        const int d = (int)((key[k] >> shift) & 255);
        const int p = tstart[d] + whist[wid][d] + rk[k];
        sk[p] = key[k];
        sv[p] = val[k];
      }
    }
    __syncthreads();
    for (int k = 0; k < RS_ITEMS; ++k) {
      const int li = wid * (RS_ITEMS * 32) + k * 32 + lane;
      if (li < n) {
        key[k] = sk[li];
        val[k] = sv[li];
      }
    }
    __syncthreads();  // whist, tstart and the staging buffers are rewritten next pass
  }
  for (int k = 0; k < RS_ITEMS; ++k) {
    const int li = wid * (RS_ITEMS * 32) + k * 32 + lane;
    if (li < n) {
      keys[li] = key[k];
      vals[li] = val[k];
    }
  }
}

// Whole sort in one thread-block cluster of CS_CL blocks (n <= CS_CL *
// CS_TILE): block c holds the pairs at positions [c * CS_TILE, (c+1) *
// CS_TILE), CS_ITEMS per thread in registers.  Per 8-bit pass every warp
// ranks its contiguous sub-tile (stable), each block publishes its digit
// counts in shared memory, and after a cluster barrier every block reads all
// blocks' counts (distributed shared memory) to place each of its pairs at
// its global position: digit start + counts of lower blocks + counts of
// lower warps + rank.  The pair is stored into the shared memory of the block
// that owns that position; after a second barrier each block reloads its
// slice.  The pairs never leave the chip between passes.
constexpr int CS_THREADS = 512;
constexpr int CS_ITEMS = 12;
constexpr int CS_TILE = CS_THREADS * CS_ITEMS;  // 6144 pairs, 96 KB per block
constexpr int CS_CL = 8;
constexpr int CS_NW = CS_THREADS / WARP;
constexpr int CS_MAX = CS_CL * CS_TILE;

__global__ void __cluster_dims__(CS_CL, 1, 1) __launch_bounds__(CS_THREADS, 1)
    k_rs_cluster(u64* keys, u64* vals, int n, int lo_bit, int bits) {
  extern __shared__ u64 cs_smem[];
  u64* sk = cs_smem;
  u64* sv = cs_smem + CS_TILE;
  __shared__ int32_t whist[CS_NW][256];
  __shared__ int32_t hist[256];   // this block's digit counts, read by the whole cluster
  __shared__ int32_t s_tot[256];  // cluster-wide digit counts
  __shared__ int32_t tpos[256];   // global start of (digit, this block)
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int base = c * CS_TILE;
  const int tile_n = max(0, min(CS_TILE, n - base));
  u64 key[CS_ITEMS], val[CS_ITEMS];
  for (int k = 0; k < CS_ITEMS; ++k) {
    const int li = wid * (CS_ITEMS * 32) + k * 32 + lane;
    key[k] = li < tile_n ? keys[base + li] : 0;
    val[k] = li < tile_n ? vals[base + li] : 0;
  }
  for (int shift = lo_bit; shift < bits; shift += 8) {
    for (int d = lane; d < 256; d += 32) whist[wid][d] = 0;
    __syncwarp();
    int rk[CS_ITEMS];
    for (int k = 0; k < CS_ITEMS; ++k) {
      const int li = wid * (CS_ITEMS * 32) + k * 32 + lane;
      const int d = li < tile_n ? (int)((key[k] >> shift) & 255) : 256;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const int before = d < 256 ? whist[wid][d] : 0;
      rk[k] = before + __popc(peers & ((1u << lane) - 1u));
      __syncwarp();
      if (d < 256 && lane == __ffs(peers) - 1) whist[wid][d] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    if (tid < 256) {  // thread = digit: exclusive prefix over the warps
      int cnt = 0;
      for (int w = 0; w < CS_NW; ++w) {
        const int x = whist[w][tid];
        whist[w][tid] = cnt;
        cnt += x;
      }
      hist[tid] = cnt;
    }
    cl.sync();  // every block's counts are published
    if (tid < 256) {
      int tot = 0, lower = 0;
      for (int b = 0; b < CS_CL; ++b) {
        const int x = cl.map_shared_rank(hist, b)[tid];
        tot += x;
        if (b < c) lower += x;
      }
      s_tot[tid] = tot;
      tpos[tid] = lower;
    }
    __syncthreads();
    if (wid == 0) {  // digit starts: exclusive scan of the totals, 8 digits per lane
      int v[8], sum = 0;
      for (int j = 0; j < 8; ++j) {
        v[j] = s_tot[lane * 8 + j];
        sum += v[j];
      }
      int incl = sum;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      int run = incl - sum;
      for (int j = 0; j < 8; ++j) {
        tpos[lane * 8 + j] += run;
        run += v[j];
      }
    }
    __syncthreads();
    for (int k = 0; k < CS_ITEMS; ++k) {
      const int li = wid * (CS_ITEMS * 32) + k * 32 + lane;
      if (li < tile_n) {
        const int d = (int)((key[k] >> shift) & 255);
        const int p = tpos[d] + whist[wid][d] + rk[k];
        const int owner = p / CS_TILE, slot = p - owner * CS_TILE;
        cl.map_shared_rank(sk, owner)[slot] = key[k];
        cl.map_shared_rank(sv, owner)[slot] = val[k];
      }
    }
    cl.sync();  // every pair is in place; counts and staging are reused next pass
    for (int k = 0; k < CS_ITEMS; ++k) {
      const int li = wid * (CS_ITEMS * 32) + k * 32 + lane;
      if (li < tile_n) {
        key[k] = sk[li];
        val[k] = sv[li];
      }
    }
  }
  for (int k = 0; k < CS_ITEMS; ++k) {
    const int li = wid * (CS_ITEMS * 32) + k * 32 + lane;
    if (li < tile_n) {
      keys[base + li] = key[k];
      vals[base + li] = val[k];
    }
  }
}

// ---------------------------------------------------------------- reduce by key
__global__ void k_heads(const u64* keys, int64_t n, int32_t* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

// Segment sums of sorted keys: each thread takes RBK_RUN consecutive pairs.
// A segment that starts and ends inside the run is stored; a segment that
// crosses a run boundary is added atomically at its head (usum is zeroed
// first).  The head of a run's leading partial segment is found by a binary
// search for the first equal key.
constexpr int RBK_RUN = 8;
__global__ void k_segsum(const u64* keys, const u64* vals, int64_t n, int64_t* usum) {
  const int64_t nt = (n + RBK_RUN - 1) / RBK_RUN;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nt; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = r * RBK_RUN, i1 = min(i0 + RBK_RUN, n);
    int64_t head = i0;
    if (i0 > 0 && keys[i0 - 1] == keys[i0]) {
      int64_t lo = 0, hi = i0;
      const u64 k = keys[i0];
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < k) lo = mid + 1; else hi = mid;
      }
      head = lo;
    }
    int64_t acc = 0;
    for (int64_t i = i0; i < i1; ++i) {
      if (i > i0 && keys[i] != keys[i - 1]) {
        if (head < i0) atomic_add_i64(&usum[head], acc);
        else usum[head] = acc;
        head = i;
        acc = 0;
      }
      acc += (int64_t)vals[i];
    }
    const bool open_end = i1 < n && keys[i1] == keys[i1 - 1];
    if (head < i0 || open_end) atomic_add_i64(&usum[head], acc);
    else usum[head] = acc;
  }
}

// flag = segment head with a nonzero sum
__global__ void k_nonzero_heads(const u64* keys, const int64_t* usum, int64_t n, int32_t* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || keys[i] != keys[i - 1]) && usum[i] != 0;
}

__global__ void k_compact_pairs(const u64* ukeys, const int64_t* usum, int64_t nu, const int32_t* flag,
                                const int64_t* pos, u64* okeys, int64_t* ovals) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nu; i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) {
      okeys[pos[i]] = ukeys[i];
      ovals[pos[i]] = usum[i];
    }
}

}  // namespace

// ---------------------------------------------------------------- host wrappers
// Look-back state for the next multi-tile scan of n items: the tile words,
// this scan's epoch (1..255) and its tile counter.  When the epoch wraps, or
// the state grows, everything is cleared so that no stale word matches.
static uint32_t lb_begin(Prims& P, int64_t n, cudaStream_t s) {
  const int64_t tiles = (n + LB_TILE - 1) / LB_TILE;
  if (P.lb_ctl.cap == 0) {
    P.lb_ctl.exact(257);  // 256 epoch counters + the error flag
    CK(cudaMemsetAsync(P.lb_ctl.p, 0, sizeof(int32_t) * 257, s));
    P.lb_ep = 0;
  }
  bool clear = false;
  if (tiles > P.lb_st.cap) {
    P.lb_st.reserve(tiles, s);
    clear = true;
  }
  if (++P.lb_ep > 255) clear = true;
  if (clear) {
    CK(cudaMemsetAsync(P.lb_st.p, 0, sizeof(u64) * (size_t)P.lb_st.cap, s));
    CK(cudaMemsetAsync(P.lb_ctl.p, 0, sizeof(int32_t) * 256, s));
    P.lb_ep = 1;
  }
  return P.lb_ep;
}

// n items, or (n_dev != nullptr) *n_dev + n items with n_max an upper bound;
// the total goes to total_dev (device) when given.
template <class In>
static void scan_launch(In in, int64_t* out, int64_t n, const int64_t* n_dev, int64_t n_max, int64_t* total_dev,
                        Prims& P, cudaStream_t s) {
  if (n_max <= SC_TILE) {
    k_scan_one<In><<<1, SC_THREADS, 0, s>>>(in, out, n, n_dev, total_dev);
    CKL("k_scan_one");
  } else {
    const uint32_t ep = lb_begin(P, n_max, s);
    const int64_t tiles = (n_max + LB_TILE - 1) / LB_TILE;
    k_scan_lb<In><<<(unsigned)tiles, SC_THREADS, 0, s>>>(in, out, n, n_dev, P.lb_st.p, P.lb_ctl.p + ep, ep,
                                                         total_dev, P.lb_ctl.p + 256);
    CKL("k_scan_lb");
  }
}

template <class T>
static int64_t scan_t(const T* in, int64_t* out, int64_t n, Prims& P, cudaStream_t s, bool want_total) {
  if (n <= 0) return 0;
  P.bsum.reserve(2, s);
  scan_launch(ArrayIn<T>{in}, out, n, nullptr, n, P.bsum.p + 1, P, s);
  if (!want_total) return -1;
  int64_t tot = 0;
  const HostRead r{P.bsum.p + 1, &tot, sizeof(int64_t)};
  P.read(&r, 1, s);
  return tot;
}

int64_t scan_exclusive(const int64_t* in, int64_t* out, int64_t n, Prims& P, cudaStream_t s, bool want_total) {
  return scan_t<int64_t>(in, out, n, P, s, want_total);
}

int64_t scan_exclusive_i32(const int32_t* in, int64_t* out, int64_t n, Prims& P, cudaStream_t s, bool want_total) {
  return scan_t<int32_t>(in, out, n, P, s, want_total);
}

void scan_exclusive_to(const int64_t* in, int64_t* out, int64_t n, const int64_t* n_dev, int64_t n_max,
                       int64_t* total_dev, Prims& P, cudaStream_t s) {
  if (n_max <= 0) return;
  scan_launch(ArrayIn<int64_t>{in}, out, n, n_dev, n_max, total_dev, P, s);
}

void scan_exclusive_i32_to(const int32_t* in, int64_t* out, int64_t n, const int64_t* n_dev, int64_t n_max,
                           int64_t* total_dev, Prims& P, cudaStream_t s) {
  if (n_max <= 0) return;
  scan_launch(ArrayIn<int32_t>{in}, out, n, n_dev, n_max, total_dev, P, s);
}

void scan_chunk_counts(const int32_t* list, const int32_t* nlist, int64_t n_hint, const int32_t* la,
                       const int32_t* lb, int32_t chunk, int64_t* out, Prims& P, cudaStream_t s) {
  scan_launch(ChunkCountIn{list, nlist, n_hint, la, lb, chunk}, out, n_hint + 1, nullptr, n_hint + 1, nullptr, P, s);
}

int32_t* scan_error_flag(Prims& P) { return P.lb_ctl.cap ? P.lb_ctl.p + 256 : nullptr; }

bool scan_wait_gives_up(cudaStream_t s) {
  // Two tiles; the tile counter starts at 1 and one block runs, so tile 1
  // waits on tile 0, which nothing publishes: the bounded wait must give up.
  Prims P;
  const int64_t n = 2 * LB_TILE;
  int32_t bad = 0;
  int64_t *in = nullptr, *out = nullptr;
  try {
    in = (int64_t*)dalloc(sizeof(int64_t) * (size_t)n);
    out = (int64_t*)dalloc(sizeof(int64_t) * (size_t)(n + 1));
    CK(cudaMemsetAsync(in, 0, sizeof(int64_t) * (size_t)n, s));
    const uint32_t ep = lb_begin(P, n, s);
    const int32_t one = 1;
    CK(cudaMemcpyAsync(P.lb_ctl.p + ep, &one, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    k_scan_lb<ArrayIn<int64_t>><<<1, SC_THREADS, 0, s>>>(ArrayIn<int64_t>{in}, out, n, nullptr, P.lb_st.p, P.lb_ctl.p + ep, ep, out + n,
                                                P.lb_ctl.p + 256);
    CKL("k_scan_lb");
    CK(cudaMemcpyAsync(&bad, P.lb_ctl.p + 256, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  } catch (...) {
    if (in) dfree(in);
    if (out) dfree(out);
    P.release();
    throw;
  }
  dfree(in);
  dfree(out);
  P.release();
  return bad != 0;
}

void radix_sort_pairs(u64*& keys, u64*& vals, u64*& tk, u64*& tv, int64_t n, int bits, Prims& P, cudaStream_t s,
                      int lo_bit) {
  if (n <= 1 || bits <= lo_bit) return;
  if (n <= RS_TILE) {
    k_rs_small<<<1, RS_THREADS, 0, s>>>(keys, vals, (int)n, lo_bit, bits);
    CKL("k_rs_small");
    return;
  }
  if (n <= CS_MAX) {  // one cluster, the pairs kept on chip
    const int smem = 2 * CS_TILE * (int)sizeof(u64);
    static thread_local int cs_attr_dev = -1;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (cs_attr_dev != dev) {
      CK(cudaFuncSetAttribute(k_rs_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      cs_attr_dev = dev;
    }
    k_rs_cluster<<<CS_CL, CS_THREADS, smem, s>>>(keys, vals, (int)n, lo_bit, bits);
    CKL("k_rs_cluster");
    return;
  }
  const int64_t nb = (n + RS_TILE - 1) / RS_TILE;
  P.hist.reserve(256 * nb + 1, s);
  P.bsum.reserve(256, s);
  // up to a few hundred tiles: one cooperative launch for all passes
  static thread_local int coop_per_sm = -1;
  if (coop_per_sm < 0) CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&coop_per_sm, k_rs_coop, RS_THREADS, 0));
  const int64_t coop_max = (int64_t)coop_per_sm * device_sms();
  if (nb <= coop_max && nb <= 1024) {
    const int grid = (int)std::max<int64_t>(nb, std::min<int64_t>(256, coop_max));
    int64_t n_ = n, nb_ = nb;
    int lo_ = lo_bit, bits_ = bits;
    int64_t *gh = P.hist.p, *dt = P.bsum.p;
    void* args[] = {&keys, &vals, &tk, &tv, &n_, &lo_, &bits_, &nb_, &gh, &dt};
    CK(cudaLaunchCooperativeKernel((const void*)k_rs_coop, dim3(grid), dim3(RS_THREADS), args, 0, s));
    CKL("k_rs_coop");
    for (int shift = lo_bit; shift < bits; shift += 8) {  // where the result ended up
      u64* t = keys; keys = tk; tk = t;
      t = vals; vals = tv; tv = t;
    }
    return;
  }
  for (int shift = lo_bit; shift < bits; shift += 8) {
    k_rs_hist<<<(unsigned)nb, RS_THREADS, 0, s>>>(keys, n, shift, nb, P.hist.p);
    CKL("k_rs_hist");
    k_rs_dscan<<<256, SC_THREADS, 0, s>>>(P.hist.p, nb, P.bsum.p);
    CKL("k_rs_dscan");
    k_rs_scatter<<<(unsigned)nb, RS_THREADS, 0, s>>>(keys, vals, tk, tv, n, shift, nb, P.hist.p, P.bsum.p);
    CKL("k_rs_scatter");
    u64* t = keys; keys = tk; tk = t;
    t = vals; vals = tv; tv = t;
  }
}

void heads_launch(const u64* keys, int64_t n, int32_t* flag, cudaStream_t s) {
  if (n <= 0) return;
  k_heads<<<grid_for(n, 256), 256, 0, s>>>(keys, n, flag);
  CKL("k_heads");
}

int64_t reduce_by_key(const u64* keys, const u64* vals, int64_t n, u64* okeys, int64_t* ovals, Prims& P,
                      cudaStream_t s) {
  if (n <= 0) return 0;
  P.flag.reserve(n + 1, s);
  P.pos.reserve(n + 1, s);
  P.usum.reserve(n + 1, s);
  // a segment crossing a run boundary is summed atomically into a zeroed slot
  CK(cudaMemsetAsync(P.usum.p, 0, sizeof(int64_t) * (size_t)n, s));
  k_segsum<<<grid_for((n + RBK_RUN - 1) / RBK_RUN, 256), 256, 0, s>>>(keys, vals, n, P.usum.p);
  CKL("k_segsum");
  const int g = grid_for(n, 256);
  k_nonzero_heads<<<g, 256, 0, s>>>(keys, P.usum.p, n, P.flag.p);
  CKL("k_nonzero_heads");
  const int64_t nz = scan_exclusive_i32(P.flag.p, P.pos.p, n, P, s, true);
  k_compact_pairs<<<g, 256, 0, s>>>(keys, P.usum.p, n, P.flag.p, P.pos.p, okeys, ovals);
  CKL("k_compact_pairs");
  return nz;
}
