// Device primitives: exclusive scan, stable LSD radix sort of (key, value)
// pairs, and reduce-by-key of sorted pairs.  Hand-written; no library sort.
#include "prims.cuh"

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

template <class T>
__global__ void k_scan_tile(const T* in, int64_t* out, int64_t n, int64_t* bsum) {
  const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
  int64_t loc[SC_ITEMS];
  int64_t s = 0;
  for (int k = 0; k < SC_ITEMS; ++k) {
    int64_t i = base + k;
    loc[k] = i < n ? (int64_t)in[i] : 0;
    s += loc[k];
  }
  int64_t tot;
  int64_t pre = block_excl_scan_i64(s, &tot);
  for (int k = 0; k < SC_ITEMS; ++k) {
    int64_t i = base + k;
    if (i < n) out[i] = pre;
    pre += loc[k];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// whole input in one tile: scan and total in one launch
template <class T>
__global__ void k_scan_one(const T* in, int64_t* out, int64_t n, int64_t* total) {
  const int64_t base = (int64_t)threadIdx.x * SC_ITEMS;
  int64_t loc[SC_ITEMS];
  int64_t s = 0;
  for (int k = 0; k < SC_ITEMS; ++k) {
    int64_t i = base + k;
    loc[k] = i < n ? (int64_t)in[i] : 0;
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

__global__ void k_scan_bsums(int64_t* bsum, int64_t nb, int64_t* total) {
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += SC_THREADS) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < nb ? bsum[i] : 0;
    int64_t tot;
    int64_t pre = block_excl_scan_i64(v, &tot);
    if (i < nb) bsum[i] = carry + pre;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_add(int64_t* out, int64_t n, const int64_t* bsum) {
  const int64_t base = (int64_t)blockIdx.x * SC_TILE;
  const int64_t add = bsum[blockIdx.x];
  for (int k = threadIdx.x; k < SC_TILE; k += SC_THREADS) {
    int64_t i = base + k;
    if (i < n) out[i] += add;
  }
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

__global__ void k_rs_hist(const u64* keys, int64_t n, int shift, int64_t nb, int64_t* ghist) {
  __shared__ uint32_t h[256];
  for (int i = threadIdx.x; i < 256; i += RS_THREADS) h[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int k = 0; k < RS_ITEMS; ++k) {
    int64_t i = base + (int64_t)k * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += RS_THREADS) ghist[(int64_t)d * nb + blockIdx.x] = h[d];
}

// goff holds tile-local exclusive prefixes of the digit-major histogram and
// gbs the scanned tile sums: the global offset of entry i is
// goff[i] + gbs[i / SC_TILE] (the scan's final add pass is folded in here).
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const u64* keys, const u64* vals, u64* okeys,
                                                           u64* ovals, int64_t n, int shift, int64_t nb,
                                                           const int64_t* goff, const int64_t* gbs) {
  __shared__ int64_t run[256];
  __shared__ int32_t tot[256];
  __shared__ int32_t wcnt[RS_THREADS / WARP][257];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int d = tid; d < 256; d += RS_THREADS) {
    const int64_t i = (int64_t)d * nb + blockIdx.x;
    run[d] = goff[i] + gbs[i / SC_TILE];
  }
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  __syncthreads();
  for (int ch = 0; ch < RS_ITEMS; ++ch) {
    const int64_t i = base + (int64_t)ch * RS_THREADS + tid;
    const bool valid = i < n;
    const u64 key = valid ? keys[i] : 0;
    const u64 val = valid ? vals[i] : 0;
    const int d = valid ? (int)((key >> shift) & 255) : 256;
    for (int x = lane; x < 257; x += 32) wcnt[wid][x] = 0;
    __syncwarp();
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (rank == 0) wcnt[wid][d] = __popc(peers);
    __syncthreads();
    if (tid < 256) {
      int acc = 0;
      for (int w = 0; w < RS_THREADS / WARP; ++w) {
        int c = wcnt[w][tid];
        wcnt[w][tid] = acc;
        acc += c;
      }
      tot[tid] = acc;
    }
    __syncthreads();
    if (valid) {
      const int64_t pos = run[d] + wcnt[wid][d] + rank;
      okeys[pos] = key;
      ovals[pos] = val;
    }
    __syncthreads();
    if (tid < 256) run[tid] += tot[tid];
    __syncthreads();
  }
}

// Whole sort in one block (n <= RS_TILE): every pass in shared memory.
__global__ void __launch_bounds__(RS_THREADS) k_rs_small(u64* keys, u64* vals, int n, int lo_bit, int bits) {
  extern __shared__ u64 sm[];
  u64* kb[2] = {sm, sm + RS_TILE};
  u64* vb[2] = {sm + 2 * RS_TILE, sm + 3 * RS_TILE};
  __shared__ int32_t hist[256];
  __shared__ int64_t run[256];
  __shared__ int32_t tot[256];
  __shared__ int32_t wcnt[RS_THREADS / WARP][257];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int i = tid; i < n; i += RS_THREADS) {
    kb[0][i] = keys[i];
    vb[0][i] = vals[i];
  }
  int cur = 0;
  for (int shift = lo_bit; shift < bits; shift += 8) {
    for (int d = tid; d < 256; d += RS_THREADS) hist[d] = 0;
    __syncthreads();
    for (int i = tid; i < n; i += RS_THREADS) atomicAdd(&hist[(kb[cur][i] >> shift) & 255], 1);
    __syncthreads();
    if (tid == 0) {
      int64_t acc = 0;
      for (int d = 0; d < 256; ++d) {
        run[d] = acc;
        acc += hist[d];
      }
    }
    __syncthreads();
    for (int ch = 0; ch * RS_THREADS < n; ++ch) {
      const int i = ch * RS_THREADS + tid;
      const bool valid = i < n;
      const u64 key = valid ? kb[cur][i] : 0;
      const u64 val = valid ? vb[cur][i] : 0;
      const int d = valid ? (int)((key >> shift) & 255) : 256;
      for (int x = lane; x < 257; x += 32) wcnt[wid][x] = 0;
      __syncwarp();
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const int rank = __popc(peers & ((1u << lane) - 1u));
      if (rank == 0) wcnt[wid][d] = __popc(peers);
      __syncthreads();
      if (tid < 256) {
        int acc = 0;
        for (int w = 0; w < RS_THREADS / WARP; ++w) {
          int cc = wcnt[w][tid];
          wcnt[w][tid] = acc;
          acc += cc;
        }
        tot[tid] = acc;
      }
      __syncthreads();
      if (valid) {
        const int64_t pos = run[d] + wcnt[wid][d] + rank;
        kb[cur ^ 1][pos] = key;
        vb[cur ^ 1][pos] = val;
      }
      __syncthreads();
      if (tid < 256) run[tid] += tot[tid];
      __syncthreads();
    }
    cur ^= 1;
  }
  for (int i = tid; i < n; i += RS_THREADS) {
    keys[i] = kb[cur][i];
    vals[i] = vb[cur][i];
  }
}

// ---------------------------------------------------------------- reduce by key
__global__ void k_heads(const u64* keys, int64_t n, int32_t* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_segsum(const u64* keys, const u64* vals, int64_t n, const int64_t* pos, const int32_t* flag,
                         u64* ukeys, int64_t* usum) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t s = pos[i] + flag[i] - 1;  // segment index
    if (flag[i]) ukeys[s] = keys[i];
    atomic_add_i64(&usum[s], (int64_t)vals[i]);
  }
}

__global__ void k_nonzero(const int64_t* usum, int64_t nu, int32_t* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nu; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = usum[i] != 0;
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
int64_t scan_exclusive(const int64_t* in, int64_t* out, int64_t n, Prims& P, cudaStream_t s, bool want_total) {
  if (n <= 0) return 0;
  int64_t nb = (n + SC_TILE - 1) / SC_TILE;
  P.bsum.reserve(nb + 1, s);
  if (nb == 1) {
    k_scan_one<int64_t><<<1, SC_THREADS, 0, s>>>(in, out, n, P.bsum.p + 1);
    CKL("k_scan_one");
    if (!want_total) return -1;
    int64_t tot = 0;
    CK(cudaMemcpyAsync(&tot, P.bsum.p + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return tot;
  }
  k_scan_tile<int64_t><<<(unsigned)nb, SC_THREADS, 0, s>>>(in, out, n, P.bsum.p);
  CKL("k_scan_tile");
  k_scan_bsums<<<1, SC_THREADS, 0, s>>>(P.bsum.p, nb, P.bsum.p + nb);
  CKL("k_scan_bsums");
  k_scan_add<<<(unsigned)nb, SC_THREADS, 0, s>>>(out, n, P.bsum.p);
  CKL("k_scan_add");
  if (!want_total) return -1;
  int64_t tot = 0;
  CK(cudaMemcpyAsync(&tot, P.bsum.p + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return tot;
}

int64_t scan_exclusive_i32(const int32_t* in, int64_t* out, int64_t n, Prims& P, cudaStream_t s, bool want_total) {
  if (n <= 0) return 0;
  int64_t nb = (n + SC_TILE - 1) / SC_TILE;
  P.bsum.reserve(nb + 1, s);
  if (nb == 1) {
    k_scan_one<int32_t><<<1, SC_THREADS, 0, s>>>(in, out, n, P.bsum.p + 1);
    CKL("k_scan_one");
    if (!want_total) return -1;
    int64_t tot = 0;
    CK(cudaMemcpyAsync(&tot, P.bsum.p + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return tot;
  }
  k_scan_tile<int32_t><<<(unsigned)nb, SC_THREADS, 0, s>>>(in, out, n, P.bsum.p);
  CKL("k_scan_tile32");
  k_scan_bsums<<<1, SC_THREADS, 0, s>>>(P.bsum.p, nb, P.bsum.p + nb);
  CKL("k_scan_bsums");
  k_scan_add<<<(unsigned)nb, SC_THREADS, 0, s>>>(out, n, P.bsum.p);
  CKL("k_scan_add");
  if (!want_total) return -1;
  int64_t tot = 0;
  CK(cudaMemcpyAsync(&tot, P.bsum.p + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return tot;
}

void radix_sort_pairs(u64*& keys, u64*& vals, u64*& tk, u64*& tv, int64_t n, int bits, Prims& P, cudaStream_t s,
                      int lo_bit) {
  if (n <= 1 || bits <= lo_bit) return;
  if (n <= RS_TILE) {
    const int smem = 4 * RS_TILE * (int)sizeof(u64);
    CK(cudaFuncSetAttribute(k_rs_small, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_rs_small<<<1, RS_THREADS, smem, s>>>(keys, vals, (int)n, lo_bit, bits);
    CKL("k_rs_small");
    return;
  }
  const int64_t nb = (n + RS_TILE - 1) / RS_TILE;
  P.hist.reserve(256 * nb + 1, s);
  P.hoff.reserve(256 * nb + 1, s);
  for (int shift = lo_bit; shift < bits; shift += 8) {
    k_rs_hist<<<(unsigned)nb, RS_THREADS, 0, s>>>(keys, n, shift, nb, P.hist.p);
    CKL("k_rs_hist");
    const int64_t hn = 256 * nb, hb = (hn + SC_TILE - 1) / SC_TILE;
    P.bsum.reserve(hb + 1, s);
    k_scan_tile<int64_t><<<(unsigned)hb, SC_THREADS, 0, s>>>(P.hist.p, P.hoff.p, hn, P.bsum.p);
    CKL("k_scan_tile");
    k_scan_bsums<<<1, SC_THREADS, 0, s>>>(P.bsum.p, hb, nullptr);
    CKL("k_scan_bsums");
    k_rs_scatter<<<(unsigned)nb, RS_THREADS, 0, s>>>(keys, vals, tk, tv, n, shift, nb, P.hoff.p, P.bsum.p);
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
  P.ukeys.reserve(n + 1, s);
  P.usum.reserve(n + 1, s);
  const int g = grid_for(n, 256);
  k_heads<<<g, 256, 0, s>>>(keys, n, P.flag.p);
  CKL("k_heads");
  int64_t nu = scan_exclusive_i32(P.flag.p, P.pos.p, n, P, s, true);
  CK(cudaMemsetAsync(P.usum.p, 0, sizeof(int64_t) * (size_t)nu, s));
  k_segsum<<<g, 256, 0, s>>>(keys, vals, n, P.pos.p, P.flag.p, P.ukeys.p, P.usum.p);
  CKL("k_segsum");
  const int g2 = grid_for(nu, 256);
  k_nonzero<<<g2, 256, 0, s>>>(P.usum.p, nu, P.flag.p);
  CKL("k_nonzero");
  int64_t nz = scan_exclusive_i32(P.flag.p, P.pos.p, nu, P, s, true);
  k_compact_pairs<<<g2, 256, 0, s>>>(P.ukeys.p, P.usum.p, nu, P.flag.p, P.pos.p, okeys, ovals);
  CKL("k_compact_pairs");
  return nz;
}
