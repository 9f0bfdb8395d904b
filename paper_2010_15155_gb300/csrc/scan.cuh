// Device-wide exclusive scan with a device-resident length (graph-friendly: fixed grids).
#pragma once
#include "common.cuh"

namespace kafmm {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class T>
__device__ inline T block_excl_scan(T v, T* sm, T& total) {
  // sm: [SCAN_THREADS / 32] scratch
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm[w] = x;
  __syncthreads();
  if (w == 0) {
    T s = lane < (int)(blockDim.x >> 5) ? sm[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    sm[lane] = s;
  }
  __syncthreads();
  T base = w > 0 ? sm[w - 1] : T(0);
  total = sm[(blockDim.x >> 5) - 1];
  __syncthreads();
  return base + x - v;
}

// Phase 1: per-tile sums. len = *d_len if d_len else n.
template <class T>
__global__ void k_scan_tiles(const T* in, int64_t n, const int* d_len, T* tile_sum) {
  __shared__ T sm[32];
  int64_t len = d_len ? (int64_t)*d_len : n;
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  if (base >= len) {
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = 0;
    return;
  }
  T s = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + threadIdx.x * SCAN_ITEMS + k;
    if (i < len) s += in[i];
  }
  T total;
  block_excl_scan<T>(s, sm, total);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

// Phase 2: scan of tile sums (one block, loops over chunks) + total.
template <class T>
__global__ void k_scan_sums(T* tile_sum, int ntiles, T* d_total) {
  __shared__ T sm[32];
  T carry = 0;
  for (int base = 0; base < ntiles; base += blockDim.x) {
    int i = base + threadIdx.x;
    T v = i < ntiles ? tile_sum[i] : T(0);
    T total;
    T e = block_excl_scan<T>(v, sm, total);
    if (i < ntiles) tile_sum[i] = carry + e;
    carry += total;
  }
  if (threadIdx.x == 0 && d_total) *d_total = carry;
}

// Phase 3: exclusive scan inside tiles plus the tile offset.
template <class T>
__global__ void k_scan_apply(const T* in, int64_t n, const int* d_len, const T* tile_sum, T* out) {
  __shared__ T sm[32];
  int64_t len = d_len ? (int64_t)*d_len : n;
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  if (base >= len) return;
  T v[SCAN_ITEMS];
  T s = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + threadIdx.x * SCAN_ITEMS + k;
    v[k] = i < len ? in[i] : T(0);
    s += v[k];
  }
  T total;
  T e = block_excl_scan<T>(s, sm, total) + tile_sum[blockIdx.x];
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + threadIdx.x * SCAN_ITEMS + k;
    if (i < len) out[i] = e;
    e += v[k];
  }
}

// One block scans up to SCAN_SMALL elements in one launch: warp w owns the contiguous chunk
// [512 w, 512 (w + 1)), read and written in rows of 32 consecutive elements (coalesced); each row
// is scanned across the lanes with a running carry, then the warps' totals are scanned.
// len = *d_len if d_len else n.
constexpr int SCAN_SMALL_ITEMS = 16;
constexpr int64_t SCAN_SMALL = (int64_t)SCAN_THREADS * SCAN_SMALL_ITEMS;
template <class T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_small(const T* in, int64_t n, const int* d_len,
                                                             T* out, T* d_total) {
  __shared__ T wsum[32];
  int64_t len = d_len ? (int64_t)*d_len : n;
  if (len > n) len = n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t chunk = (int64_t)w * 32 * SCAN_SMALL_ITEMS;
  T ex[SCAN_SMALL_ITEMS];
  T carry = 0;
#pragma unroll
  for (int k = 0; k < SCAN_SMALL_ITEMS; ++k) {
    const int64_t i = chunk + 32 * k + lane;
    const T v = i < len ? in[i] : T(0);
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    ex[k] = carry + x - v;
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) wsum[w] = carry;
  __syncthreads();
  if (w == 0) {
    const T t = lane < (int)(blockDim.x >> 5) ? wsum[lane] : T(0);
    T x = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    wsum[lane] = x - t;   // exclusive offsets of the warps
    if (lane == 31 && d_total) *d_total = x;
  }
  __syncthreads();
  const T off = wsum[w];
#pragma unroll
  for (int k = 0; k < SCAN_SMALL_ITEMS; ++k) {
    const int64_t i = chunk + 32 * k + lane;
    if (i < len) out[i] = off + ex[k];
  }
}

// Exclusive scan of in[0..len) into out (in-place allowed); *d_total receives the sum.
// cap bounds len; scratch needs (cap / SCAN_TILE + 1) elements.
template <class T>
inline void scan_excl(const T* in, T* out, int64_t cap, const int* d_len, T* scratch, T* d_total,
                      cudaStream_t st) {
  if (cap <= SCAN_SMALL) {
    KL k_scan_small<T><<<1, SCAN_THREADS, 0, st>>>(in, cap, d_len, out, d_total);
    return;
  }
  int ntiles = (int)((cap + SCAN_TILE - 1) / SCAN_TILE);
  if (ntiles < 1) ntiles = 1;
  KL k_scan_tiles<T><<<ntiles, SCAN_THREADS, 0, st>>>(in, cap, d_len, scratch);
  KL k_scan_sums<T><<<1, SCAN_THREADS, 0, st>>>(scratch, ntiles, d_total);
  KL k_scan_apply<T><<<ntiles, SCAN_THREADS, 0, st>>>(in, cap, d_len, scratch, out);
}

}  // namespace kafmm
