// Octree construction on the device: Morton keys, LSD radix sort, level-by-level
// refinement and the U/V/W/X interaction lists of kernel-independent FMM (Sec. II; the
// refinement rule of Sec. III with a configurable leaf size).
#include <algorithm>
#include <cmath>

#include "plan.cuh"
#include "scan.cuh"

namespace kafmm {

// ---------------------------------------------------------------------------------------
// Morton keys.  Cell I = clamp(floor((p - origin) / L * 2^20), 0, 2^20 - 1) per axis in FP64.
// When L is a power of two, inv_L = 1 / L is exact and the product equals the quotient.
template <class T>
__global__ void k_keys(const T* __restrict__ pts, int64_t n, double ox, double oy, double oz,
                       double L, double inv_L, uint64_t* __restrict__ key, uint32_t* __restrict__ idx,
                       unsigned* status) {
  const double s = (double)(1 << MAX_LEVEL);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d[3] = {(double)pts[3 * i] - ox, (double)pts[3 * i + 1] - oy, (double)pts[3 * i + 2] - oz};
    double u[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = inv_L > 0.0 ? d[c] * inv_L : d[c] / L;
    uint32_t c[3];
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      ok = ok && (u[d] >= 0.0) && (u[d] < 1.0);
      double f = floor(u[d] * s);
      f = f < 0.0 ? 0.0 : (f > s - 1.0 ? s - 1.0 : f);
      c[d] = ok ? (uint32_t)f : 0u;
    }
    if (!ok) atomicOr(status, (unsigned)ST_DOMAIN);
    key[i] = morton3(c[0], c[1], c[2]);
    idx[i] = (uint32_t)i;
  }
}

// ---------------------------------------------------------------------------------------
// LSD radix sort of (u64 key, u32 value), 8-bit digits, stable.  Tile of 4096 keys per block
// (8 warps x 32 lanes x 16 rounds); ranks inside a warp come from __match_any_sync.
constexpr int RS_THREADS = 256, RS_ROUNDS = 16, RS_WARPS = RS_THREADS / 32;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;

// Problem of caller index v: the largest k < nprob with off[k] <= v (empty problems skipped).
__device__ inline uint32_t problem_of(const int64_t* __restrict__ off, int nprob, uint32_t v) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= (int64_t)v)
      lo = mid;
    else
      hi = mid - 1;
  }
  return (uint32_t)lo;
}

// Digit of one element: bits [shift, shift + 8) of the Morton key, or of the element's
// problem index when poff is given (the passes that group a batch by problem).
__device__ inline unsigned radix_digit(uint64_t k, uint32_t v, int shift, const int64_t* poff,
                                       int nprob) {
  if (poff) return (problem_of(poff, nprob, v) >> shift) & 255u;
  return (unsigned)((k >> shift) & 255);
}

__global__ void k_radix_hist(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                             int64_t n, int shift, const int64_t* __restrict__ poff, int nprob,
                             uint32_t* __restrict__ hist, int nblk) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int k = 0; k < RS_ROUNDS; ++k) {
    int64_t i = base + k * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&cnt[radix_digit(keys[i], poff ? vals[i] : 0u, shift, poff, nprob)], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_radix_scatter(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n,
                                int shift, const int64_t* __restrict__ poff, int nprob,
                                const uint32_t* __restrict__ hist, int nblk) {
  __shared__ uint32_t wcnt[RS_WARPS][256];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = lane; d < 256; d += 32) wcnt[w][d] = 0;
  __syncwarp();
  int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * 32 * RS_ROUNDS;
  uint64_t k[RS_ROUNDS];
  uint32_t v[RS_ROUNDS], rk[RS_ROUNDS];
  unsigned dg[RS_ROUNDS];
  unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    int64_t i = base + r * 32 + lane;
    bool valid = i < n;
    k[r] = valid ? kin[i] : 0ull;
    v[r] = valid ? vin[i] : 0u;
    unsigned d = valid ? radix_digit(k[r], v[r], shift, poff, nprob) : 256u;
    dg[r] = d;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int leader = __ffs(peers) - 1;
    uint32_t cur = 0;
    if (lane == leader && valid) cur = wcnt[w][d];
    cur = __shfl_sync(0xffffffffu, cur, leader);
    rk[r] = cur + __popc(peers & lt);
    __syncwarp();
    if (lane == leader && valid) wcnt[w][d] = cur + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {  // exclusive scan over warps per digit, plus the global base of this block
    int d = threadIdx.x;
    uint32_t run = hist[(int64_t)d * nblk + blockIdx.x];
    for (int ww = 0; ww < RS_WARPS; ++ww) {
      uint32_t t = wcnt[ww][d];
      wcnt[ww][d] = run;
      run += t;
    }
  }
  __syncthreads();
  for (int r = 0; r < RS_ROUNDS; ++r) {
    int64_t i = base + r * 32 + lane;
    if (i < n) {
      unsigned d = dg[r];
      uint32_t pos = wcnt[w][d] + rk[r];
      kout[pos] = k[r];
      vout[pos] = v[r];
    }
  }
}

// Stable LSD passes over (keys, vals), ping-pong through (k2, v2): one pass per entry of
// shifts, the 8-bit digit of the key at that bit (an entry s >= 64: bits [s - 64, s - 56) of the
// problem index of the element's caller index).  An odd number of passes ends with a copy back,
// so the result is always in (keys, vals).
static void radix_passes(uint64_t* keys, uint32_t* vals, uint64_t* k2, uint32_t* v2, uint32_t* hist,
                         int64_t n, const int64_t* poff, int nprob, const int* shifts, int npass, cudaStream_t st) {
  if (n <= 1 || npass <= 0) return;
  int nblk = (int)((n + RS_TILE - 1) / RS_TILE);
  uint64_t *ka = keys, *kb = k2;
  uint32_t *va = vals, *vb = v2;
  for (int pass = 0; pass < npass; ++pass) {
    const bool by_prob = shifts[pass] >= 64;
    const int shift = by_prob ? shifts[pass] - 64 : shifts[pass];
    const int64_t* po = by_prob ? poff : nullptr;
    KL k_radix_hist<<<nblk, RS_THREADS, 0, st>>>(ka, va, n, shift, po, nprob, hist, nblk);
    scan_excl<uint32_t>(hist, hist, (int64_t)256 * nblk, nullptr, hist + 256 * (int64_t)nblk, nullptr, st);
    KL k_radix_scatter<<<nblk, RS_THREADS, 0, st>>>(ka, va, kb, vb, n, shift, po, nprob, hist, nblk);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (npass & 1) {  // the result sits in (k2, v2)
    cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
  }
}

// The low 2 x key_passes digits of the keys (for short keys), unconditionally.
static void radix_sort(uint64_t* keys, uint32_t* vals, uint64_t* k2, uint32_t* v2, uint32_t* hist,
                       int64_t n, cudaStream_t st, int key_passes) {
  int shifts[8];
  for (int i = 0; i < key_passes; ++i) shifts[i] = 8 * i;
  radix_passes(keys, vals, k2, v2, hist, n, nullptr, 1, shifts, key_passes, st);
}

// The Morton keys are first sorted on their top 32 bits (bits 28-59: the cells of levels 1-10
// in order).  That order is all the refinement reads unless a level-10 cell would split, i.e.
// holds more than q points (sources and targets); k_deep_check looks for a run of q + 1 equal
// level-10 cells, the host reads its flag with the level counts, and then the full sort on all
// 60 bits runs and the tree is built again (a stable LSD sort from scratch: the first order only
// breaks ties, which index order breaks the same way).  With separate targets each set is
// checked against q / 2, which bounds the sum.
constexpr int TOP_SHIFTS[4] = {28, 36, 44, 52};
constexpr int FULL_SHIFTS[8] = {0, 8, 16, 24, 32, 40, 48, 56};
constexpr int CELL10_SHIFT = 3 * (MAX_LEVEL - 10);

__global__ void k_deep_check(const uint64_t* __restrict__ key, int64_t n, int run, int* flag) {
  bool deep = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i + run < n; i += (int64_t)gridDim.x * blockDim.x)
    deep = deep || (key[i] >> CELL10_SHIFT) == (key[i + run] >> CELL10_SHIFT);
  if (__any_sync(0xffffffffu, deep) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// Dense starts of the cells of levels 1-DENSE_LV in the sorted keys of one point set (a single
// problem): start[cell_off(l) + cell] = first sorted index in the cell, 0x7f7f7f7f when empty.
constexpr int DENSE_LV = 5;
constexpr int DENSE_N = ((1 << (3 * (DENSE_LV + 1))) - 8) / 7;
__host__ __device__ constexpr int dense_off(int l) { return ((1 << (3 * l)) - 8) / 7; }

__global__ void k_cell_starts(const uint64_t* __restrict__ key, int64_t n, int* __restrict__ start) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = key[i], kp = i > 0 ? key[i - 1] : ~0ull;
#pragma unroll
    for (int l = 1; l <= DENSE_LV; ++l) {
      const int sh = 3 * (MAX_LEVEL - l);
      if (i == 0 || (k >> sh) != (kp >> sh)) start[dense_off(l) + (int)(k >> sh)] = (int)i;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Level-by-level refinement.  Level l holds up to cap[l] boxes at bld_* + cap_off[l].
struct BuildArgs {
  uint64_t* key;
  int *sb, *se, *tb, *te, *parent, *child, *cnt, *nch, *choff, *cb, *ctb, *prob;
  const uint64_t* skey;
  const uint64_t* tkey;
  const int64_t* soff;   // [nprob + 1] source offsets of the problems
  const int64_t* toff;   // [nprob + 1] target offsets
  const int* dstart_s;   // dense cell starts of levels 1-DENSE_LV (sources, targets) when dense
  const int* dstart_t;
  int same, q, nprob, dense;
  int64_t cap_off[MAX_LEVELS + 1];
  int cap[MAX_LEVELS];
};

__device__ inline int lower_bound_prefix(const uint64_t* k, int lo, int hi, uint64_t want, int sh) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if ((k[mid] >> sh) < want)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Level 0: one root per problem, holding that problem's slice of the sorted points.
__global__ void k_root(BuildArgs a) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.nprob; k += gridDim.x * blockDim.x) {
    a.key[k] = 0;
    a.sb[k] = (int)a.soff[k];
    a.se[k] = (int)a.soff[k + 1];
    a.tb[k] = a.same ? (int)a.soff[k] : (int)a.toff[k];
    a.te[k] = a.same ? (int)a.soff[k + 1] : (int)a.toff[k + 1];
    a.parent[k] = -1;
    a.prob[k] = k;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (int l = 0; l < MAX_LEVELS; ++l) a.cnt[l] = l == 0 ? a.nprob : 0;
}

// Loads of the refinement: plain, or L2-only (ld.global.cg) inside the cooperative kernel,
// whose phases read what other blocks wrote earlier in the same launch (an L1 line could still
// hold an older copy of a neighbouring entry).
template <bool CG, class V>
__device__ __forceinline__ V rd(const V* p) {
  if constexpr (CG)
    return __ldcg(p);
  else
    return *p;
}

// One warp per box: a box with more than q points splits; lanes 0-7 find the start of child o in
// the sorted source keys and lanes 8-15 in the target keys (binary searches in parallel, so
// the root's eight searches over all points are one chain of dependent loads, not eight; the
// top levels read their child boundaries from the dense cell-start tables).
template <bool CG>
__device__ void split_box(const BuildArgs& a, int lv, int i, int lane) {
  const int64_t g = a.cap_off[lv] + i;
  const int sh = 3 * (MAX_LEVEL - lv - 1);
  const int sb = rd<CG>(a.sb + g), se = rd<CG>(a.se + g), tb = rd<CG>(a.tb + g), te = rd<CG>(a.te + g);
  const int count = (se - sb) + (a.same ? 0 : (te - tb));
  int nch = 0;
  if (count > a.q && lv < MAX_LEVEL) {   // warp-uniform
    const uint64_t k = rd<CG>(a.key + g);
    int v = 0;
    if (a.dense && lv < DENSE_LV) {
      // child o starts at the first non-empty child o' >= o (suffix minimum over the 8 cell
      // starts of each set), else at the end of the box
      v = 0x7f7f7f7f;
      const int base = dense_off(lv + 1) + (int)(k * 8);
      if (lane < 8)
        v = a.dstart_s[base + lane];
      else if (lane < 16 && !a.same)
        v = a.dstart_t[base + lane - 8];
#pragma unroll
      for (int d = 1; d < 8; d <<= 1) {
        const int w = __shfl_down_sync(0xffffffffu, v, d, 8);
        if ((lane & 7) + d < 8) v = min(v, w);
      }
      v = min(v, lane < 8 ? se : te);
    } else if (lane < 8) {
      v = lower_bound_prefix(a.skey, sb, se, k * 8 + lane, sh);
    } else if (lane < 16 && !a.same) {
      v = lower_bound_prefix(a.tkey, tb, te, k * 8 + (lane - 8), sh);
    }
    int cb[9], ctb[9];
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      cb[o] = __shfl_sync(0xffffffffu, v, o);
      ctb[o] = __shfl_sync(0xffffffffu, v, 8 + o);
      if (a.same) ctb[o] = cb[o];
    }
    cb[8] = se;
    ctb[8] = a.same ? se : te;
    if (lane < 9) {
      a.cb[g * 9 + lane] = cb[lane];
      a.ctb[g * 9 + lane] = ctb[lane];
    }
#pragma unroll
    for (int o = 0; o < 8; ++o)
      nch += ((cb[o + 1] - cb[o]) + (a.same ? 0 : (ctb[o + 1] - ctb[o]))) > 0;
  }
  if (lane == 0) a.nch[g] = nch;
}

__global__ void k_split(BuildArgs a, int lv, unsigned* status) {
  const int n = a.cnt[lv];
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += gridDim.x * wpb) split_box<false>(a, lv, i, lane);
}

__global__ void k_level_total(BuildArgs a, int lv, const int* total, unsigned* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int t = *total;
    if (lv + 1 < MAX_LEVELS) {
      if (t > a.cap[lv + 1]) {
        atomicOr(status, (unsigned)ST_OVERFLOW);
        t = a.cap[lv + 1];
      }
      a.cnt[lv + 1] = t;
    }
  }
}

// Children of box i of level lv, numbered from j (the exclusive prefix of the child counts).
template <bool CG>
__device__ void emit_box(const BuildArgs& a, int lv, int i, int j) {
  const int64_t o0 = a.cap_off[lv], o1 = a.cap_off[lv + 1];
  const int cap1 = a.cap[lv + 1 < MAX_LEVELS ? lv + 1 : lv];
  const int64_t g = o0 + i;
  const int nch = rd<CG>(a.nch + g);
  const uint64_t k = rd<CG>(a.key + g);
  const int prob = rd<CG>(a.prob + g);
  for (int o = 0; o < 8; ++o) {
    int c = -1;
    if (nch > 0) {
      const int b0 = rd<CG>(a.cb + g * 9 + o), b1 = rd<CG>(a.cb + g * 9 + o + 1);
      const int t0 = rd<CG>(a.ctb + g * 9 + o), t1 = rd<CG>(a.ctb + g * 9 + o + 1);
      const int cnt = (b1 - b0) + (a.same ? 0 : (t1 - t0));
      if (cnt > 0 && j < cap1) {
        const int64_t h = o1 + j;
        a.key[h] = k * 8 + o;
        a.sb[h] = b0;
        a.se[h] = b1;
        a.tb[h] = a.same ? b0 : t0;
        a.te[h] = a.same ? b1 : t1;
        a.parent[h] = i;
        a.prob[h] = prob;
        c = j;
        ++j;
      }
    }
    a.child[g * 8 + o] = c;
  }
}

__global__ void k_emit(BuildArgs a, int lv) {
  const int n = a.cnt[lv];
  const int64_t o0 = a.cap_off[lv];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    emit_box<false>(a, lv, i, a.choff[o0 + i]);
}

// Grid barrier of the cooperative refinement: arrival counter and generation, the wait bounded
// by %globaltimer (ST_TIMEOUT in *status and false when the other blocks did not arrive).
__device__ bool refine_barrier(unsigned* count, unsigned* gen, unsigned* status, unsigned long long limit_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned g = *(volatile unsigned*)gen;
    __threadfence();
    if (atomicAdd(count, 1u) + 1u == gridDim.x) {
      *(volatile unsigned*)count = 0u;
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*(volatile unsigned*)gen == g) {
        if (global_ns() - t0 > limit_ns) {
          atomicOr(status, (unsigned)ST_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// The whole refinement in one cooperative launch: the roots, then per level (until one is
// empty) split (warp per box), the exclusive scan of the child counts (block b scans a
// contiguous chunk; its offset is the sum of the earlier blocks' totals), the next level's count
// (clamped to its capacity, ST_OVERFLOW otherwise) and the children (thread per box of the
// block's own chunk), with grid barriers between the phases.  sync: [count, generation];
// bsum: one total per block.  A barrier that times out ends every block (ST_TIMEOUT).
__global__ void __launch_bounds__(256) k_refine(BuildArgs a, int* bsum, unsigned* sync, unsigned* status,
                                                unsigned long long limit_ns) {
  __shared__ int s_part[32];
  __shared__ int s_off, s_tot;
  const int G = gridDim.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  if (blockIdx.x == 0) {
    for (int k = threadIdx.x; k < a.nprob; k += blockDim.x) {
      a.key[k] = 0;
      a.sb[k] = (int)a.soff[k];
      a.se[k] = (int)a.soff[k + 1];
      a.tb[k] = a.same ? (int)a.soff[k] : (int)a.toff[k];
      a.te[k] = a.same ? (int)a.soff[k + 1] : (int)a.toff[k + 1];
      a.parent[k] = -1;
      a.prob[k] = k;
    }
    for (int l = threadIdx.x; l < MAX_LEVELS; l += blockDim.x) a.cnt[l] = l == 0 ? a.nprob : 0;
  }
  if (!refine_barrier(sync, sync + 1, status, limit_ns)) return;
  for (int lv = 0; lv < MAX_LEVEL; ++lv) {
    const int n = __ldcg(a.cnt + lv);
    if (n == 0) break;   // uniform: every block read the count after the same barrier
    const int64_t o0 = a.cap_off[lv];
    for (int i = blockIdx.x * wpb + w; i < n; i += G * wpb) split_box<true>(a, lv, i, lane);
    if (!refine_barrier(sync, sync + 1, status, limit_ns)) return;
    // exclusive scan of the child counts over this block's chunk
    const int chunk = (n + G - 1) / G;
    const int lo = min(n, blockIdx.x * chunk), hi = min(n, lo + chunk);
    int carry = 0;
    for (int base = lo; base < hi; base += blockDim.x) {
      const int i = base + threadIdx.x;
      const int v = i < hi ? __ldcg(a.nch + o0 + i) : 0;
      int x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) s_part[w] = x;
      __syncthreads();
      if (w == 0) {
        const int t = lane < wpb ? s_part[lane] : 0;
        int xx = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, xx, o);
          if (lane >= o) xx += y;
        }
        s_part[lane] = xx - t;   // exclusive warp offsets
        if (lane == 31) s_tot = xx;
      }
      __syncthreads();
      if (i < hi) a.choff[o0 + i] = carry + s_part[w] + x - v;
      carry += s_tot;
      __syncthreads();
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = carry;
    if (!refine_barrier(sync, sync + 1, status, limit_ns)) return;
    // this block's offset, and (last block) the next level's count
    int before = 0, all = 0;
    for (int b = threadIdx.x; b < G; b += blockDim.x) {
      const int t = __ldcg(bsum + b);
      all += t;
      if (b < blockIdx.x) before += t;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      before += __shfl_down_sync(0xffffffffu, before, o);
      all += __shfl_down_sync(0xffffffffu, all, o);
    }
    if (lane == 0) s_part[w] = before;
    __syncthreads();
    if (threadIdx.x == 0) {
      int sbf = 0;
      for (int q = 0; q < wpb; ++q) sbf += s_part[q];
      s_off = sbf;
    }
    __syncthreads();
    if (lane == 0) s_part[w] = all;
    __syncthreads();
    if (threadIdx.x == 0 && blockIdx.x == G - 1 && lv + 1 < MAX_LEVELS) {
      int t = 0;
      for (int q = 0; q < wpb; ++q) t += s_part[q];
      if (t > a.cap[lv + 1]) {
        atomicOr(status, (unsigned)ST_OVERFLOW);
        t = a.cap[lv + 1];
      }
      a.cnt[lv + 1] = t;
    }
    const int off = s_off;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) emit_box<true>(a, lv, i, off + __ldcg(a.choff + o0 + i));
    if (!refine_barrier(sync, sync + 1, status, limit_ns)) return;
  }
}

struct Layout {
  int lvl_start[MAX_LEVELS + 1];
  int64_t cap_off[MAX_LEVELS + 1];
};

__global__ void k_compact(BuildArgs a, Layout lay, int nbox, uint64_t* key, int8_t* level,
                          int* parent, int* child, int* sb, int* se, int* tb, int* te,
                          int8_t* leaf, int* prob) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nbox; g += gridDim.x * blockDim.x) {
    int lv = 0;
    while (lv + 1 < MAX_LEVELS && g >= lay.lvl_start[lv + 1]) ++lv;
    int i = g - lay.lvl_start[lv];
    int64_t h = lay.cap_off[lv] + i;
    key[g] = a.key[h];
    prob[g] = a.prob[h];
    level[g] = (int8_t)lv;
    parent[g] = lv > 0 ? lay.lvl_start[lv - 1] + a.parent[h] : -1;
    sb[g] = a.sb[h];
    se[g] = a.se[h];
    tb[g] = a.tb[h];
    te[g] = a.te[h];
    bool lf = true;
    for (int o = 0; o < 8; ++o) {
      int c = (lv + 1 < MAX_LEVELS) ? a.child[h * 8 + o] : -1;
      child[g * 8 + o] = c >= 0 ? lay.lvl_start[lv + 1] + c : -1;
      lf = lf && c < 0;
    }
    leaf[g] = lf ? 1 : 0;
  }
}

// ---------------------------------------------------------------------------------------
// Lists.
__device__ inline void anchor_of(uint64_t k, int& x, int& y, int& z) {
  x = (int)compact3(k);
  y = (int)compact3(k >> 1);
  z = (int)compact3(k >> 2);
}

// Box of problem pb at level lv with anchor (ax, ay, az), or -1.  A level is ordered by
// (problem, Morton key).
__device__ inline int find_box(const TreeView& t, int lv, int pb, int ax, int ay, int az) {
  if (lv >= t.nlevels) return -1;
  uint64_t k = morton3((uint32_t)ax, (uint32_t)ay, (uint32_t)az);
  int lo = t.lvl_start[lv], hi = t.lvl_start[lv + 1], end = hi;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    int pm = t.prob[mid];
    if (pm < pb || (pm == pb && t.key[mid] < k))
      lo = mid + 1;
    else
      hi = mid;
  }
  return (lo < end && t.prob[lo] == pb && t.key[lo] == k) ? lo : -1;
}

// Deepest existing box of problem pb at level <= lv that contains cell (lv, a).  The roots
// always exist: root of problem pb is box pb.
__device__ inline int deepest_box(const TreeView& t, int lv, int pb, int ax, int ay, int az) {
  int top = lv < t.nlevels - 1 ? lv : t.nlevels - 1;
  for (int l = top; l >= 0; --l) {
    int sh = lv - l;
    int b = find_box(t, l, pb, ax >> sh, ay >> sh, az >> sh);
    if (b >= 0) return b;
  }
  return pb;
}

// Neighbour cell a + d at level lv along one axis: wraps (periodic along that axis) or reports
// absence.  s: image shift.
__device__ inline bool neighbour(int periodic, int lv, int a, int d, int& c, int& s) {
  int n = 1 << lv;
  c = a + d;
  s = 0;
  if (c < 0 || c >= n) {
    if (!periodic) return false;
    s = c < 0 ? -((-c + n - 1) / n) : c / n;
    c -= s * n;
  }
  return true;
}

// Closed boxes (b at level lb, anchor ab, moved by shift s domains) and (lb2, ab2) intersect?
__device__ inline bool adjacent(int la, int ax, int ay, int az, int sx, int sy, int sz, int lb, int bx,
                                int by, int bz) {
  int64_t wa = 1ll << (MAX_LEVEL - la), wb = 1ll << (MAX_LEVEL - lb), D = 1ll << MAX_LEVEL;
  int64_t a0[3] = {ax * wa + sx * D, ay * wa + sy * D, az * wa + sz * D};
  int64_t b0[3] = {bx * wb, by * wb, bz * wb};
  for (int d = 0; d < 3; ++d)
    if (a0[d] > b0[d] + wb || b0[d] > a0[d] + wa) return false;
  return true;
}

struct ListOut {
  int64_t* u_cnt;  // count mode: counts; fill mode: offsets
  int64_t* w_cnt;
  int64_t* x_cnt;
  int32_t* u_ent;
  int32_t* w_ent;
  int32_t* x_ent;
  int32_t* vtab;   // [nbox][216]
  int8_t* w_flag;
  unsigned long long* near_pairs;
};

// V: same-level boxes at the 189 offsets of the parent's neighbourhood, one thread per
// (box, slot k of the parent's 6^3 neighbourhood).
__global__ void k_vtab(TreeView t, int32_t* __restrict__ vtab) {
  const int64_t total = (int64_t)t.nbox * 216;
  for (int64_t e0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e0 < total;
       e0 += (int64_t)gridDim.x * blockDim.x) {
    int b = (int)(e0 / 216), k = (int)(e0 % 216);
    int lv = t.level[b];
    int ax, ay, az;
    anchor_of(t.key[b], ax, ay, az);
    int ox = k % 6 - 2 - (ax & 1), oy = (k / 6) % 6 - 2 - (ay & 1), oz = k / 36 - 2 - (az & 1);
    int32_t e = LIST_EMPTY;
    bool inner = abs(ox) <= 1 && abs(oy) <= 1 && abs(oz) <= 1;
    if (!inner && (lv >= 2 || (t.periodic && lv >= 1))) {
      int cx, cy, cz, sx, sy, sz;
      if (neighbour(t.periodic & 1, lv, ax, ox, cx, sx) && neighbour(t.periodic & 2, lv, ay, oy, cy, sy) &&
          neighbour(t.periodic & 4, lv, az, oz, cz, sz)) {
        int s = find_box(t, lv, t.prob[b], cx, cy, cz);
        if (s >= 0) e = pack_entry(s, shift_code(sx, sy, sz));
      }
    }
    vtab[e0] = e;
  }
}

// Warp-level exclusive scan of per-lane counts; total in *tot.
__device__ __forceinline__ int64_t warp_excl(int64_t v, int lane, int64_t* tot) {
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  *tot = __shfl_sync(0xffffffffu, x, 31);
  return x - v;
}

// U, W and X lists, one warp per box: lane d < 27 takes neighbour direction d of the box (U and
// W, leaves only), lane d < 27 also direction d of the parent (X, d != 13).  A coarse U or X
// entry reached from several directions is kept by its lowest lane (__match_any_sync); each
// lane's entries go to its place in the box's list by a warp scan of the counts (direction
// order, then descent order within a direction).
template <bool FILL>
__global__ void k_lists(TreeView t, ListOut o) {
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int b = blockIdx.x * wpb + (threadIdx.x >> 5); b < t.nbox; b += gridDim.x * wpb) {
    const int lv = t.level[b];
    const int pb = t.prob[b];
    int ax, ay, az;
    anchor_of(t.key[b], ax, ay, az);
    const bool is_leaf = t.leaf[b] != 0;
    const int ntb = t.te[b] - t.tb[b];
    int64_t nu = 0, nw = 0, nx = 0;
    unsigned long long pairs = 0;
    // ---- U and W (leaves): direction d = lane
    int sx = 0, sy = 0, sz = 0, sc = 13, nb = -1, kind = 0;   // kind 1: coarse leaf, 2: leaf, 3: descend
    if (is_leaf && lane < 27) {
      const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
      int cx, cy, cz;
      if (neighbour(t.periodic & 1, lv, ax, dx, cx, sx) && neighbour(t.periodic & 2, lv, ay, dy, cy, sy) &&
          neighbour(t.periodic & 4, lv, az, dz, cz, sz)) {
        sc = shift_code(sx, sy, sz);
        nb = deepest_box(t, lv, pb, cx, cy, cz);
        const int nl = t.level[nb];
        if (nl < lv)
          kind = t.leaf[nb] ? 1 : 0;   // a coarser box holds the cell: only a leaf is a U neighbour
        else
          kind = t.leaf[nb] ? 2 : 3;
      }
    }
    // coarse entries reached from several directions: the lowest lane keeps it
    const int32_t ce = kind == 1 ? pack_entry(nb, sc) : LIST_EMPTY;
    const unsigned peers = __match_any_sync(0xffffffffu, ce);
    if (kind == 1 && (__ffs(peers) - 1) != lane) kind = 0;
    // two rounds: count, then (FILL) write at the scanned offsets
    int64_t u_base = 0, w_base = 0;
    for (int round = 0; round < (FILL ? 2 : 1); ++round) {
      nu = nw = 0;
      pairs = 0;
      const bool write = FILL && round == 1;
      if (kind == 1 || kind == 2) {
        if (write) o.u_ent[u_base + nu] = pack_entry(nb, sc);
        ++nu;
        pairs += (unsigned long long)ntb * (t.se[nb] - t.sb[nb]);
      } else if (kind == 3) {
        // non-leaf colleague: descend; adjacent leaves -> U, non-adjacent boxes -> W
        int stack[8 * MAX_LEVELS];
        int sp = 0;
        for (int c = 0; c < 8; ++c)
          if (t.child[nb * 8 + c] >= 0) stack[sp++] = t.child[nb * 8 + c];
        while (sp > 0) {
          const int dd = stack[--sp];
          const int dl = t.level[dd];
          int qx, qy, qz;
          anchor_of(t.key[dd], qx, qy, qz);
          if (adjacent(dl, qx, qy, qz, sx, sy, sz, lv, ax, ay, az)) {
            if (t.leaf[dd]) {
              if (write) o.u_ent[u_base + nu] = pack_entry(dd, sc);
              ++nu;
              pairs += (unsigned long long)ntb * (t.se[dd] - t.sb[dd]);
            } else {
              for (int c = 0; c < 8; ++c)
                if (t.child[dd * 8 + c] >= 0 && sp < 8 * MAX_LEVELS) stack[sp++] = t.child[dd * 8 + c];
            }
          } else {
            if (write) {
              o.w_ent[w_base + nw] = pack_entry(dd, sc);
              o.w_flag[dd] = 1;
            }
            ++nw;
          }
        }
      }
      if (FILL && round == 0) {   // this lane's first entry in the box's lists
        int64_t tu, tw;
        u_base = o.u_cnt[b] + warp_excl(nu, lane, &tu);
        w_base = o.w_cnt[b] + warp_excl(nw, lane, &tw);
      }
    }
    // ---- X: coarser leaves adjacent to the parent but not to b; direction d = lane != 13
    int32_t xe = LIST_EMPTY;
    if (lv >= 1 && lane < 27 && lane != 13) {
      const int p = t.parent[b];
      int px_, py_, pz_;
      anchor_of(t.key[p], px_, py_, pz_);
      const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
      int cx, cy, cz, xsx, xsy, xsz;
      if (neighbour(t.periodic & 1, lv - 1, px_, dx, cx, xsx) &&
          neighbour(t.periodic & 2, lv - 1, py_, dy, cy, xsy) &&
          neighbour(t.periodic & 4, lv - 1, pz_, dz, cz, xsz)) {
        const int xb = deepest_box(t, lv - 1, pb, cx, cy, cz);
        if (t.leaf[xb]) {
          const int nl = t.level[xb];
          int qx, qy, qz;
          anchor_of(t.key[xb], qx, qy, qz);
          if (!adjacent(nl, qx, qy, qz, xsx, xsy, xsz, lv, ax, ay, az)) xe = pack_entry(xb, shift_code(xsx, xsy, xsz));
        }
      }
    }
    const unsigned xpeers = __match_any_sync(0xffffffffu, xe);
    nx = (xe != LIST_EMPTY && (__ffs(xpeers) - 1) == lane) ? 1 : 0;
    int64_t tx;
    const int64_t xoff = warp_excl(nx, lane, &tx);
    if (FILL && nx) o.x_ent[o.x_cnt[b] + xoff] = xe;
    // ---- totals
    int64_t tu, tw;
    warp_excl(nu, lane, &tu);
    warp_excl(nw, lane, &tw);
    if (!FILL) {
      if (lane == 0) {
        o.u_cnt[b] = tu;
        o.w_cnt[b] = tw;
        o.x_cnt[b] = tx;
      }
    } else {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, off);
      if (lane == 0 && pairs) atomicAdd(o.near_pairs, pairs);
    }
  }
}

// Gathers the sorted points into the compute type (x, y, z, 0).
template <class Tin, class T4>
__global__ void k_gather_pos(const Tin* __restrict__ pts, const uint32_t* __restrict__ perm, int64_t n,
                             T4* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t j = perm[i];
    T4 v;
    v.x = pts[3 * (int64_t)j];
    v.y = pts[3 * (int64_t)j + 1];
    v.z = pts[3 * (int64_t)j + 2];
    v.w = 0;
    out[i] = v;
  }
}

__global__ void k_leaf_list(const int8_t* leaf, const int* leaf_pos, int nbox, int* leaves) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += gridDim.x * blockDim.x)
    if (leaf[b]) leaves[leaf_pos[b]] = b;
}

// Leaf box of every sorted source point.
__global__ void k_leaf_of(TreeView t, int* __restrict__ leaf_of) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < t.nbox; b += gridDim.x * blockDim.x)
    if (t.leaf[b])
      for (int i = t.sb[b]; i < t.se[b]; ++i) leaf_of[i] = b;
}

// V-list count, largest leaf, and the V slot occupancy of every box as 27 bytes (padded to 32):
// byte g = (gx, gy, gz) in [0,3)^3 is the neighbour of the parent at offset (g - 1), bit
// d = (dx, dy, dz) its child, i.e. slot (2gx + dx) + 6 (2gy + dy) + 36 (2gz + dz) of the 6^3
// table.
// Parent neighbours of box b with V entries (bit g of the result): bytes of its occupancy
// record that are nonzero.
__device__ inline uint32_t vocc_neighbours(const uint4* vocc, int64_t b, uint64_t (&w)[4]) {
  const uint4 a = vocc[2 * b], c = vocc[2 * b + 1];
  w[0] = a.x | (uint64_t)a.y << 32;
  w[1] = a.z | (uint64_t)a.w << 32;
  w[2] = c.x | (uint64_t)c.y << 32;
  w[3] = c.z | (uint64_t)c.w << 32;
  uint32_t m = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    uint64_t x = w[k];
    x |= x >> 4;
    x |= x >> 2;
    x |= x >> 1;
    x &= 0x0101010101010101ull;   // bit 0 of each byte: byte nonzero
    m |= (uint32_t)((x * 0x0102040810204080ull) >> 56) << (8 * k);   // gather to bits 0..7
  }
  return m & ((1u << 27) - 1);
}

__global__ void k_tree_stats(TreeView t, const int32_t* vtab, unsigned long long* out, uint4* vocc,
                             int vmin, int* m2l_cnt, unsigned* m2l_hist) {
  __shared__ unsigned hist[216];
  for (int k = threadIdx.x; k < 216; k += blockDim.x) hist[k] = 0;
  __syncthreads();
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < t.nbox; b += gridDim.x * blockDim.x) {
    unsigned long long nv = 0;
    uint32_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int32_t* vt = vtab + (int64_t)b * 216;
#pragma unroll
    for (int g = 0; g < 27; ++g) {
      const int gx = g % 3, gy = (g / 3) % 3, gz = g / 9;
      uint32_t byte = 0;
#pragma unroll
      for (int d = 0; d < 8; ++d) {
        int k = (2 * gx + (d & 1)) + 6 * (2 * gy + ((d >> 1) & 1)) + 36 * (2 * gz + (d >> 2));
        byte |= (uint32_t)(vt[k] != LIST_EMPTY) << d;
      }
      nv += __popc(byte);
      w[g >> 2] |= byte << (8 * (g & 3));
    }
    vocc[2 * (int64_t)b] = make_uint4(w[0], w[1], w[2], w[3]);
    vocc[2 * (int64_t)b + 1] = make_uint4(w[4], w[5], w[6], w[7]);
    atomicAdd(&out[0], nv);
    if (t.leaf[b]) {
      unsigned long long np = (unsigned long long)max(t.se[b] - t.sb[b], t.te[b] - t.tb[b]);
      atomicMax(&out[1], np);
    }
    // grouped M->L: (box, parent neighbour) pairs of the boxes at levels >= vmin
    uint32_t m = 0;
    if (t.level[b] >= vmin) {
      uint64_t wd[4];
      m = vocc_neighbours(vocc, b, wd);
      const int c = (int)(t.key[b] & 7);
      for (uint32_t r = m; r; r &= r - 1) atomicAdd(&hist[(__ffs(r) - 1) * 8 + c], 1u);
    }
    m2l_cnt[b] = __popc(m);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 216; k += blockDim.x)
    if (hist[k]) atomicAdd(&m2l_hist[k], hist[k]);
}

// Grouped M->L pairs in box order: pair i = (box, neighbour g) has the sort key (g, octant
// class, occupancy byte of g), its partial index i, and its box; comb[b] = (b, first pair,
// count).  Neighbour-major order keeps the 27 offsets of one neighbour (over all classes) in
// L2 while its tiles run: class-major order re-read every operator from DRAM once per class
// (2.4 GB per M->L launch, Stokeslet N = 262144, p = 10).
__global__ void k_m2l_pair_emit(TreeView t, const uint4* vocc, int vmin, const int* base,
                                uint64_t* keys, uint32_t* vals, int* pbox, int4* comb) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < t.nbox; b += gridDim.x * blockDim.x) {
    int n = 0;
    const int first = base[b];
    if (t.level[b] >= vmin) {
      uint64_t w[4];
      const uint32_t m = vocc_neighbours(vocc, b, w);
      const int c = (int)(t.key[b] & 7);
      for (uint32_t r = m; r; r &= r - 1) {
        const int g = __ffs(r) - 1;
        const unsigned byte = (unsigned)(w[g >> 3] >> (8 * (g & 7))) & 255u;
        const int pos = first + n++;
        keys[pos] = (uint64_t)((g * 8 + c) << 8 | byte);
        vals[pos] = (uint32_t)pos;
        pbox[pos] = b;
      }
    }
    comb[b] = make_int4(b, first, n, 0);
  }
}

__global__ void k_m2l_pair_box(const uint32_t* vals, const int* pbox, int64_t n, int* box) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    box[i] = pbox[vals[i]];
}

__global__ void k_i8_to_i32(const int8_t* a, int n, int* b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = a[i];
}

TreeView Tree::view() const {
  TreeView v;
  v.nbox = nbox;
  v.nlevels = nlevels;
  v.periodic = 0;
  v.lvl_start = d_lvl_start.as<int>();
  v.prob = prob.as<int>();
  v.key = key.as<uint64_t>();
  v.level = level.as<int8_t>();
  v.parent = parent.as<int>();
  v.child = child.as<int>();
  v.sb = sb.as<int>();
  v.se = se.as<int>();
  v.tb = tb.as<int>();
  v.te = te.as<int>();
  v.leaf = leaf.as<int8_t>();
  return v;
}

static int grid_for(int64_t n, int threads, int maxb = 152 * 8) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > maxb) b = maxb;
  return (int)b;
}

#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(P, e_, #call); \
  } while (0)

// Keys + permutation of one point set, sorted on the top 32 bits of the keys.
static int sort_top(Plan& P, const void* pts, int64_t n, int dtype, DevBuf& key, DevBuf& perm, DevBuf& k2,
                    DevBuf& v2) {
  Tree& T = P.tree;
  cudaStream_t st = P.stream;
  CK(key.reserve(sizeof(uint64_t) * (n + 1)));
  CK(perm.reserve(sizeof(uint32_t) * (n + 1)));
  CK(k2.reserve(sizeof(uint64_t) * (n + 1)));
  CK(v2.reserve(sizeof(uint32_t) * (n + 1)));
  int64_t nblk = (n + RS_TILE - 1) / RS_TILE + 1;
  CK(T.s_hist.reserve(sizeof(uint32_t) * (256 * nblk + 256 * nblk / SCAN_TILE + 64)));
  if (n == 0) return 0;
  unsigned* status = T.status.as<unsigned>();
  int g = grid_for(n, 256);
  int e = 0;
  const double inv_L = std::frexp(P.L, &e) == 0.5 ? 1.0 / P.L : 0.0;   // exact for a power of two
  if (dtype == KAFMM_F64)
    KL k_keys<double><<<g, 256, 0, st>>>((const double*)pts, n, P.origin[0], P.origin[1], P.origin[2], P.L,
                                       inv_L, key.as<uint64_t>(), perm.as<uint32_t>(), status);
  else
    KL k_keys<float><<<g, 256, 0, st>>>((const float*)pts, n, P.origin[0], P.origin[1], P.origin[2], P.L,
                                      inv_L, key.as<uint64_t>(), perm.as<uint32_t>(), status);
  radix_passes(key.as<uint64_t>(), perm.as<uint32_t>(), k2.as<uint64_t>(), v2.as<uint32_t>(), T.s_hist.as<uint32_t>(),
               n, nullptr, 1, TOP_SHIFTS, 4, st);
  return 0;
}

// The full 60-bit key sort of one point set (stable LSD from the current order: the first
// sort only breaks ties, which index order breaks the same way).
static void sort_full(Plan& P, int64_t n, DevBuf& key, DevBuf& perm, DevBuf& k2, DevBuf& v2) {
  radix_passes(key.as<uint64_t>(), perm.as<uint32_t>(), k2.as<uint64_t>(), v2.as<uint32_t>(),
               P.tree.s_hist.as<uint32_t>(), n, nullptr, 1, FULL_SHIFTS, 8, P.stream);
}

// The problem passes of a batch and the sorted positions in the compute type.
static int sort_finish(Plan& P, const void* pts, int64_t n, int dtype, const int64_t* d_off, int nprob,
                       DevBuf& key, DevBuf& perm, DevBuf& k2, DevBuf& v2, DevBuf& pos) {
  Tree& T = P.tree;
  cudaStream_t st = P.stream;
  uint64_t* kk = key.as<uint64_t>();
  uint32_t* vv = perm.as<uint32_t>();
  if (nprob > 1) {
    const int prob_shifts[2] = {64, 72};
    radix_passes(kk, vv, k2.as<uint64_t>(), v2.as<uint32_t>(), T.s_hist.as<uint32_t>(), n, d_off, nprob,
                 prob_shifts, nprob > 256 ? 2 : 1, st);
  }
  size_t esz = P.fp64() ? sizeof(double4) : sizeof(float4);
  CK(pos.reserve(esz * (n + 1)));
  int g = grid_for(n, 256);
  if (n > 0) {
    if (P.fp64()) {
      if (dtype == KAFMM_F64)
        KL k_gather_pos<double, double4><<<g, 256, 0, st>>>((const double*)pts, vv, n, pos.as<double4>());
      else
        KL k_gather_pos<float, double4><<<g, 256, 0, st>>>((const float*)pts, vv, n, pos.as<double4>());
    } else {
      if (dtype == KAFMM_F64)
        KL k_gather_pos<double, float4><<<g, 256, 0, st>>>((const double*)pts, vv, n, pos.as<float4>());
      else
        KL k_gather_pos<float, float4><<<g, 256, 0, st>>>((const float*)pts, vv, n, pos.as<float4>());
    }
  }
  CK(cudaGetLastError());
  return 0;
}

__global__ void k_clear_bits(unsigned* status, unsigned mask) {
  if (threadIdx.x == 0) *status &= ~mask;
}

int build_tree(Plan& P, const void* y, int64_t ns, const void* x, int64_t nt, int dtype, int n_prob,
               const int64_t* src_off, const int64_t* trg_off) {
  Tree& T = P.tree;
  cudaStream_t st = P.stream;
  T.n_src = ns;
  T.n_trg = nt;
  T.n_prob = n_prob;
  T.src_off.assign(src_off, src_off + n_prob + 1);
  T.trg_off.assign(trg_off, trg_off + n_prob + 1);
  T.same = (x == y) && (ns == nt) && T.src_off == T.trg_off;
  T.dtype_pts = dtype;
  CK(T.status.reserve(64));
  CK(cudaMemsetAsync(T.status.p, 0, 64, st));
  CK(T.d_src_off.reserve(sizeof(int64_t) * (n_prob + 1)));
  CK(T.d_trg_off.reserve(sizeof(int64_t) * (n_prob + 1)));
  CK(cudaMemcpyAsync(T.d_src_off.p, T.src_off.data(), sizeof(int64_t) * (n_prob + 1),
                     cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(T.d_trg_off.p, T.trg_off.data(), sizeof(int64_t) * (n_prob + 1),
                     cudaMemcpyHostToDevice, st));
  cudaEventRecord(P.ev[0], st);

  int rc = sort_top(P, y, ns, dtype, T.src_key, T.src_perm, T.s_keys2, T.s_vals2);
  if (!rc && !T.same) rc = sort_top(P, x, nt, dtype, T.trg_key, T.trg_perm, T.t_keys2, T.t_vals2);
  if (rc) return rc;
  CK(T.sort_flag.reserve(sizeof(int) * 4));
  int* flag = T.sort_flag.as<int>();
  CK(cudaMemsetAsync(flag, 0, sizeof(int) * 4, st));
  {
    const int run = T.same ? P.q : P.q / 2;
    if (ns > 0)
      KL k_deep_check<<<grid_for(ns, 256), 256, 0, st>>>(T.src_key.as<uint64_t>(), ns, run, flag);
    if (!T.same && nt > 0)
      KL k_deep_check<<<grid_for(nt, 256), 256, 0, st>>>(T.trg_key.as<uint64_t>(), nt, run, flag);
  }
  const bool dense = n_prob == 1;

  // per-level capacities: n_prob roots; below, min(n_prob 8^l, 8 * floor(N / (q + 1)) + 8)
  // (only a box with more than q points splits, into at most 8 children)
  int64_t npts = T.same ? ns : ns + nt;
  int64_t per = 8 * (npts / (P.q + 1)) + 8;
  BuildArgs a;
  int64_t off = 0;
  for (int l = 0; l < MAX_LEVELS; ++l) {
    int64_t c = l == 0 ? n_prob : (l < 8 ? std::min<int64_t>(per, (int64_t)n_prob << (3 * l)) : per);
    a.cap[l] = (int)c;
    a.cap_off[l] = off;
    off += c;
  }
  a.cap_off[MAX_LEVELS] = off;
  CK(T.bld_key.reserve(sizeof(uint64_t) * off));
  CK(T.bld_sb.reserve(sizeof(int) * off));
  CK(T.bld_se.reserve(sizeof(int) * off));
  CK(T.bld_tb.reserve(sizeof(int) * off));
  CK(T.bld_te.reserve(sizeof(int) * off));
  CK(T.bld_parent.reserve(sizeof(int) * off));
  CK(T.bld_child.reserve(sizeof(int) * off * 8));
  CK(T.bld_nch.reserve(sizeof(int) * off));
  CK(T.bld_choff.reserve(sizeof(int) * (off + off / SCAN_TILE + 64)));
  CK(T.bld_cb.reserve(sizeof(int) * off * 9));
  CK(T.bld_ctb.reserve(sizeof(int) * off * 9));
  CK(T.bld_cnt.reserve(sizeof(int) * (MAX_LEVELS + 8)));
  CK(T.bld_prob.reserve(sizeof(int) * off));
  if (dense) CK(T.dense_start.reserve(sizeof(int) * 2 * DENSE_N));
  a.key = T.bld_key.as<uint64_t>();
  a.sb = T.bld_sb.as<int>();
  a.se = T.bld_se.as<int>();
  a.tb = T.bld_tb.as<int>();
  a.te = T.bld_te.as<int>();
  a.parent = T.bld_parent.as<int>();
  a.child = T.bld_child.as<int>();
  a.cnt = T.bld_cnt.as<int>();
  a.nch = T.bld_nch.as<int>();
  a.choff = T.bld_choff.as<int>();
  a.cb = T.bld_cb.as<int>();
  a.ctb = T.bld_ctb.as<int>();
  a.prob = T.bld_prob.as<int>();
  a.soff = T.d_src_off.as<int64_t>();
  a.toff = T.d_trg_off.as<int64_t>();
  a.nprob = n_prob;
  a.skey = T.src_key.as<uint64_t>();
  a.tkey = T.same ? a.skey : T.trg_key.as<uint64_t>();
  a.same = T.same ? 1 : 0;
  a.q = P.q;
  a.dense = dense ? 1 : 0;
  a.dstart_s = dense ? T.dense_start.as<int>() : nullptr;
  a.dstart_t = dense ? T.dense_start.as<int>() + DENSE_N : nullptr;
  unsigned* status = T.status.as<unsigned>();
  int* d_total = a.cnt + MAX_LEVELS + 1;

  // cooperative refinement: blocks that fit on the GPU at once, at most two per SM
  int coop_blocks = 0;
  {
    int dev = 0, nsm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_refine, 256, 0) == cudaSuccess)
      coop_blocks = std::min(per_sm, 2) * nsm;
    cudaGetLastError();
  }
  CK(T.bld_sync.reserve(sizeof(int) * (coop_blocks + 16)));

  // The top-32-bit order suffices unless k_deep_check found a level-10 cell that would split;
  // the flag is read back with the level counts, and then the points are sorted on all 60 bits
  // and the tree is built again.
  int cnt[MAX_LEVELS + 1];
  unsigned h_status = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (attempt == 1) {
      KL k_clear_bits<<<1, 32, 0, st>>>(status, ST_OVERFLOW | ST_TIMEOUT);
      sort_full(P, ns, T.src_key, T.src_perm, T.s_keys2, T.s_vals2);
      if (!T.same) sort_full(P, nt, T.trg_key, T.trg_perm, T.t_keys2, T.t_vals2);
    }
    rc = sort_finish(P, y, ns, dtype, T.d_src_off.as<int64_t>(), n_prob, T.src_key, T.src_perm, T.s_keys2,
                     T.s_vals2, T.src_pos);
    if (!rc && !T.same)
      rc = sort_finish(P, x, nt, dtype, T.d_trg_off.as<int64_t>(), n_prob, T.trg_key, T.trg_perm, T.t_keys2,
                       T.t_vals2, T.trg_pos);
    if (rc) return rc;
    // dense cell starts of the top levels (one problem): the refinement of levels 0 to
    // DENSE_LV - 1 reads its child boundaries there instead of searching
    if (dense) {
      CK(cudaMemsetAsync(T.dense_start.p, 0x7f, sizeof(int) * (T.same ? 1 : 2) * DENSE_N, st));
      if (ns > 0)
        KL k_cell_starts<<<grid_for(ns, 256), 256, 0, st>>>(T.src_key.as<uint64_t>(), ns, T.dense_start.as<int>());
      if (!T.same && nt > 0)
        KL k_cell_starts<<<grid_for(nt, 256), 256, 0, st>>>(T.trg_key.as<uint64_t>(), nt,
                                                          T.dense_start.as<int>() + DENSE_N);
    }
    bool coop = false;
    if (coop_blocks > 0) {
      int* bsum = T.bld_sync.as<int>() + 16;
      unsigned* sync = T.bld_sync.as<unsigned>();
      CK(cudaMemsetAsync(sync, 0, sizeof(unsigned) * 2, st));
      unsigned long long limit = P.wait.hard_ns;
      void* args[] = {&a, &bsum, &sync, &status, &limit};
      ++g_launches;
      coop = cudaLaunchCooperativeKernel((const void*)k_refine, dim3(coop_blocks), dim3(256), args, 0, st) ==
             cudaSuccess;
      cudaGetLastError();
    }
    if (coop) {
      CK(cudaMemcpyAsync(cnt, a.cnt, sizeof(int) * MAX_LEVELS, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(&h_status, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    } else {
      // levels in groups of launches: the first covers the depth a uniform tree of these points
      // would have (ceil(log8(points / q)) + 1 levels below the root), later ones 4 levels
      // each; after each group every level's box count and the status are read back at once
      // and the refinement stops when the next level is empty
      KL k_root<<<grid_for(n_prob, 256), 256, 0, st>>>(a);
      int est = 1;
      for (double m = (double)npts / (double)(P.q > 0 ? P.q : 1) / std::max(1, n_prob); m > 1.0 && est < MAX_LEVEL;
           m /= 8.0)
        ++est;
      for (int l0 = 0, group = est + 1;; group = 4) {
        int l1 = std::min(MAX_LEVEL, l0 + group);
        for (int l = l0; l < l1; ++l) {
          int g = grid_for(a.cap[l], 256);
          KL k_split<<<grid_for((int64_t)a.cap[l] * 32, 256), 256, 0, st>>>(a, l, status);
          int* scratch = a.choff + a.cap_off[MAX_LEVELS] + 16;
          scan_excl<int>(a.nch + a.cap_off[l], a.choff + a.cap_off[l], a.cap[l], a.cnt + l, scratch, d_total, st);
          KL k_level_total<<<1, 32, 0, st>>>(a, l, d_total, status);
          KL k_emit<<<g, 256, 0, st>>>(a, l);
        }
        CK(cudaMemcpyAsync(cnt, a.cnt, sizeof(int) * MAX_LEVELS, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&h_status, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (l1 >= MAX_LEVEL || cnt[l1] == 0 || (h_status & (ST_DOMAIN | ST_OVERFLOW))) break;
        l0 = l1;
      }
    }
    int h_flag = 0;
    CK(cudaMemcpyAsync(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h_status & (ST_DOMAIN | ST_TIMEOUT)) break;
    if (!h_flag || attempt == 1) break;
  }
  CK(cudaGetLastError());
  if (h_status & ST_DOMAIN)
    return fail(P, KAFMM_ERR_DOMAIN, "a point lies outside [origin, origin + L)^3 or is not finite");
  if (h_status & ST_TIMEOUT) return fail(P, KAFMM_ERR_TIMEOUT, "octree refinement: a grid barrier timed out");
  if (h_status & ST_OVERFLOW) return fail(P, KAFMM_ERR_NOMEM, "octree level capacity exceeded");

  Layout lay;
  T.nlevels = 0;
  int nb = 0;
  for (int l = 0; l < MAX_LEVELS; ++l) {
    lay.lvl_start[l] = nb;
    T.lvl_start[l] = nb;
    nb += cnt[l];
    if (cnt[l] > 0) T.nlevels = l + 1;
    lay.cap_off[l] = a.cap_off[l];
  }
  lay.lvl_start[MAX_LEVELS] = nb;
  T.lvl_start[MAX_LEVELS] = nb;
  lay.cap_off[MAX_LEVELS] = a.cap_off[MAX_LEVELS];
  T.nbox = nb;

  CK(T.key.reserve(sizeof(uint64_t) * nb));
  CK(T.level.reserve(nb));
  CK(T.parent.reserve(sizeof(int) * nb));
  CK(T.child.reserve(sizeof(int) * nb * 8));
  CK(T.sb.reserve(sizeof(int) * nb));
  CK(T.se.reserve(sizeof(int) * nb));
  CK(T.tb.reserve(sizeof(int) * nb));
  CK(T.te.reserve(sizeof(int) * nb));
  CK(T.leaf.reserve(nb));
  CK(T.prob.reserve(sizeof(int) * nb));
  CK(T.d_lvl_start.reserve(sizeof(int) * (MAX_LEVELS + 1)));
  CK(cudaMemcpyAsync(T.d_lvl_start.p, T.lvl_start, sizeof(int) * (MAX_LEVELS + 1),
                     cudaMemcpyHostToDevice, st));
  KL k_compact<<<grid_for(nb, 256), 256, 0, st>>>(a, lay, nb, T.key.as<uint64_t>(), T.level.as<int8_t>(),
                                              T.parent.as<int>(), T.child.as<int>(), T.sb.as<int>(),
                                              T.se.as<int>(), T.tb.as<int>(), T.te.as<int>(),
                                              T.leaf.as<int8_t>(), T.prob.as<int>());
  // leaf list (box order)
  CK(T.leaves.reserve(sizeof(int) * (2 * nb + nb / SCAN_TILE + 64)));
  int* lpos = T.leaves.as<int>() + nb;
  int* lscratch = lpos + nb;
  int* ltot = lscratch + nb / SCAN_TILE + 8;
  KL k_i8_to_i32<<<grid_for(nb, 256), 256, 0, st>>>(T.leaf.as<int8_t>(), nb, lpos);
  scan_excl<int>(lpos, lpos, nb, nullptr, lscratch, ltot, st);
  KL k_leaf_list<<<grid_for(nb, 256), 256, 0, st>>>(T.leaf.as<int8_t>(), lpos, nb, T.leaves.as<int>());
  CK(T.leaf_of.reserve(sizeof(int) * (ns + 1)));
  KL k_leaf_of<<<grid_for(nb, 128), 128, 0, st>>>(T.view(), T.leaf_of.as<int>());
  CK(cudaMemcpyAsync(&T.nleaf, ltot, sizeof(int), cudaMemcpyDeviceToHost, st));
  cudaEventRecord(P.ev[1], st);

  // ---- lists
  TreeView tv = T.view();
  tv.periodic = periodic_mask(P.bc);
  CK(T.u_off.reserve(sizeof(int64_t) * (nb + 1 + nb / SCAN_TILE + 64)));
  CK(T.w_off.reserve(sizeof(int64_t) * (nb + 1 + nb / SCAN_TILE + 64)));
  CK(T.x_off.reserve(sizeof(int64_t) * (nb + 1 + nb / SCAN_TILE + 64)));
  CK(T.vtab.reserve(sizeof(int32_t) * (int64_t)nb * 216));
  CK(T.w_flag.reserve(nb));
  CK(cudaMemsetAsync(T.w_flag.p, 0, nb, st));
  ListOut lo{};
  lo.u_cnt = T.u_off.as<int64_t>();
  lo.w_cnt = T.w_off.as<int64_t>();
  lo.x_cnt = T.x_off.as<int64_t>();
  // one warp per box (lanes take the neighbour directions), 8 boxes per block
  int g = grid_for((int64_t)nb * 32, 256, 152 * 16);
  KL k_vtab<<<grid_for((int64_t)nb * 216, 256, 152 * 16), 256, 0, st>>>(tv, T.vtab.as<int32_t>());
  KL k_lists<false><<<g, 256, 0, st>>>(tv, lo);
  int64_t tot[3];
  int64_t* sc[3] = {lo.u_cnt, lo.w_cnt, lo.x_cnt};
  for (int k = 0; k < 3; ++k) {
    int64_t* scratch = sc[k] + nb + 2;
    scan_excl<int64_t>(sc[k], sc[k], nb, nullptr, scratch, sc[k] + nb, st);
  }
  for (int k = 0; k < 3; ++k)
    CK(cudaMemcpyAsync(&tot[k], sc[k] + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  T.n_u = tot[0];
  T.n_w = tot[1];
  T.n_x = tot[2];
  CK(T.u_ent.reserve(sizeof(int32_t) * (T.n_u + 1)));
  CK(T.w_ent.reserve(sizeof(int32_t) * (T.n_w + 1)));
  CK(T.x_ent.reserve(sizeof(int32_t) * (T.n_x + 1)));
  lo.u_ent = T.u_ent.as<int32_t>();
  lo.w_ent = T.w_ent.as<int32_t>();
  lo.x_ent = T.x_ent.as<int32_t>();
  lo.vtab = T.vtab.as<int32_t>();
  lo.w_flag = T.w_flag.as<int8_t>();
  lo.near_pairs = (unsigned long long*)(T.status.as<unsigned>() + 8);
  CK(cudaMemsetAsync(lo.near_pairs, 0, 8, st));
  KL k_lists<true><<<g, 256, 0, st>>>(tv, lo);
  CK(cudaGetLastError());
  cudaEventRecord(P.ev[2], st);
  // V entries, the largest leaf, and the pairs of the grouped M->L (count per box, then their
  // offsets by a scan; per (class, neighbour) totals for the tile layout)
  unsigned long long* stats = (unsigned long long*)(T.status.as<unsigned>() + 10);
  CK(cudaMemsetAsync(stats, 0, 16, st));
  CK(T.vocc.reserve(32 * (size_t)(nb + 1)));
  CK(T.m2l_cnt.reserve(sizeof(int) * (nb + 1)));
  CK(T.m2l_base.reserve(sizeof(int) * (nb + 1)));
  CK(T.m2l_meta.reserve(sizeof(int) * (216 + 1 + nb / SCAN_TILE + 64)));
  unsigned* meta = T.m2l_meta.as<unsigned>();   // [0..216) per (neighbour, class), [216] total
  CK(cudaMemsetAsync(meta, 0, sizeof(unsigned) * 217, st));
  const int vmin = periodic_mask(P.bc) ? 1 : 2;
  KL k_tree_stats<<<grid_for(nb, 256), 256, 0, st>>>(tv, T.vtab.as<int32_t>(), stats, T.vocc.as<uint4>(),
                                                   vmin, T.m2l_cnt.as<int>(), meta);
  scan_excl<int>(T.m2l_cnt.as<int>(), T.m2l_base.as<int>(), nb, nullptr,
                 reinterpret_cast<int*>(meta) + 217, reinterpret_cast<int*>(meta) + 216, st);
  // the V entry count, the largest leaf, the near-field pair count and the grouped M->L pair
  // histogram are read back with the work lists (build_worklists), in the same copy
  CK(cudaGetLastError());
  return 0;
}

// Sorted pairs of the grouped M->L: P.m2l_box[i] and P.m2l_part_sorted[i] for the pairs ordered by
// (parent neighbour, octant class, occupancy byte), boxes in box order within equal keys;
// P.m2l_comb[b] = (b, first partial, count) for every box.
int m2l_pairs_sort(Plan& P) {
  Tree& T = P.tree;
  cudaStream_t st = P.stream;
  const int nb = T.nbox;
  const int64_t n = T.m2l_npairs;
  const int vmin = periodic_mask(P.bc) ? 1 : 2;
  CK(P.m2l_keys.reserve(sizeof(uint64_t) * 2 * (n + 1)));
  CK(P.m2l_vals.reserve(sizeof(uint32_t) * 2 * (n + 1)));
  CK(P.m2l_pbox.reserve(sizeof(int) * (n + 1)));
  CK(P.m2l_box.reserve(sizeof(int) * (n + 1)));
  CK(P.m2l_comb.reserve(sizeof(int4) * (nb + 1)));
  const int nblk = (int)((n + RS_TILE - 1) / RS_TILE);
  CK(P.m2l_hist.reserve(sizeof(uint32_t) * (256 * (size_t)nblk + 256 * (size_t)nblk / SCAN_TILE + 64)));
  uint64_t* k1 = P.m2l_keys.as<uint64_t>();
  uint32_t* v1 = P.m2l_vals.as<uint32_t>();
  TreeView tv = T.view();
  KL k_m2l_pair_emit<<<grid_for(nb, 256), 256, 0, st>>>(tv, T.vocc.as<uint4>(), vmin, T.m2l_base.as<int>(), k1,
                                                      v1, P.m2l_pbox.as<int>(), P.m2l_comb.as<int4>());
  // two 8-bit passes over the 16-bit keys (stable): the sorted values are the partial indices
  radix_sort(k1, v1, k1 + n + 1, v1 + n + 1, P.m2l_hist.as<uint32_t>(), n, st, 2);
  KL k_m2l_pair_box<<<grid_for(n, 256), 256, 0, st>>>(v1, P.m2l_pbox.as<int>(), n, P.m2l_box.as<int>());
  P.m2l_part_sorted = v1;
  CK(cudaGetLastError());
  return 0;
}

}  // namespace kafmm
