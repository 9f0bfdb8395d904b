// RPY sphere velocities (Sec. II.B): target assembly u_a = u + a^2/6 lap u (Eq. RPYtrgvel)
// and the post-processing the paper prescribes for overlapping spheres.  The kernel sum
// uses the far form G + b^2/6 lap G for every pair; for pairs in contact (r <= a_i + b_j) the
// far form is replaced by the overlap-regularised pair mobility of unequal spheres (the form
// of Zuk et al. 2014, cited by the paper):
//   |a-b| < r <= a+b :  M = [A I + B rr/r^2] / (6 pi a b),
//        A = (16 r^3 (a+b) - ((a-b)^2 + 3 r^2)^2) / (32 r^3),  B = 3 ((a-b)^2 - r^2)^2 / (32 r^3)
//   r <= |a-b|       :  M = I / (6 pi max(a, b))
// i.e. the pass adds (M_overlap - M_far) f for those pairs (M_far = 0 at r = 0, as the sum
// skips coincident pairs).  With the contact split (FP32 forms, one shared point set) the near
// field leaves out its pairs within r <= b_i + b_j and this pass adds their whole mobility.
// Neighbours come from a dense cell table at a grid level whose cell side is at least the contact
// reach (max(a_max, b_max) + b_max) divided by H, so every contact partner lies in the (2H + 1)^3
// surrounding cells; H = 2 where the grid allows it (about half the candidate pairs of H = 1 in
// dense clusters), and cells farther from the target than the reach are skipped.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "physics.cuh"
#include "plan.cuh"

namespace kafmm {

namespace {

template <class Tin, class T>
__global__ void k_gather_scalar(const Tin* __restrict__ in, const uint32_t* __restrict__ perm, int64_t n,
                                T* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (T)in[perm[i]];
}

template <class Tin, class T>
__global__ void k_gather_fb(const Tin* __restrict__ s, const uint32_t* __restrict__ perm, int64_t n,
                            typename V4<T>::type* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const Tin* p = s + 4 * (int64_t)perm[i];
    typename V4<T>::type v;
    v.x = (T)p[0];
    v.y = (T)p[1];
    v.z = (T)p[2];
    v.w = (T)p[3];
    out[i] = v;
  }
}

template <class T>
__global__ void k_max_radius(const T* __restrict__ a, int64_t n, const typename V4<T>::type* __restrict__ fb,
                             int64_t ns, unsigned* out) {
  float ma = 0.f, mb = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    ma = fmaxf(ma, (float)a[i]);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x)
    mb = fmaxf(mb, (float)fb[i].w);
  atomicMax(out, __float_as_uint(ma));  // non-negative floats order as unsigned ints
  atomicMax(out + 1, __float_as_uint(mb));
}

// cell table: for the cells (Morton code at level g) holding sources, [begin, end) in sorted order
__global__ void k_cell_table(const uint64_t* __restrict__ key, int64_t n, int shift, int* __restrict__ beg,
                             int* __restrict__ end) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t c = key[i] >> shift;
    if (i == 0 || (key[i - 1] >> shift) != c) beg[c] = (int)i;
    if (i == n - 1 || (key[i + 1] >> shift) != c) end[c] = (int)(i + 1);
  }
}

// Whole pair mobility M(r; ai, aj) f (overlap form within contact, far form outside), added to
// acc: for contact pairs the near field left out (one shared point set, FP32 forms).
template <class T>
__device__ inline void pair_full(T r0, T r1, T r2, T ai, T aj, T f0, T f1, T f2, T* acc) {
  T rr = r0 * r0 + r1 * r1 + r2 * r2;
  T rn = sqrt(rr);
  T s = ai + aj, d = fabs(ai - aj);
  const T pi = T(PI);
  T rf = r0 * f0 + r1 * f1 + r2 * f2;
  T A, Bt;   // M f = A f + Bt r
  if (rn > s) {   // far form G + (ai^2 + aj^2)/6 lap G
    T c = ai * ai + aj * aj;
    A = (T(1) + c / (T(3) * rr)) / (T(8) * pi * rn);
    Bt = (T(1) - c / rr) / (T(8) * pi * rn) * rf / rr;
  } else if (rn > d) {
    T r3 = rr * rn, t = d * d + T(3) * rr, e = d * d - rr;
    A = (T(16) * r3 * s - t * t) / (T(32) * r3) / (T(6) * pi * ai * aj);
    Bt = T(3) * e * e / (T(32) * r3) / (T(6) * pi * ai * aj) * rf / rr;
  } else {
    A = T(1) / (T(6) * pi * (ai > aj ? ai : aj));
    Bt = T(0);
  }
  acc[0] += A * f0 + Bt * r0;
  acc[1] += A * f1 + Bt * r1;
  acc[2] += A * f2 + Bt * r2;
}

// Closed leaf boxes A and B (B moved by the image shift s, in domains) intersect: the pair is
// in A's U list.
__device__ inline bool leaves_adjacent(const int8_t* level, const uint64_t* key, int A, int B, int sx, int sy,
                                       int sz) {
  int la = level[A], lb = level[B];
  int64_t wa = 1ll << (MAX_LEVEL - la), wb = 1ll << (MAX_LEVEL - lb), D = 1ll << MAX_LEVEL;
  uint64_t ka = key[A], kb = key[B];
  int64_t a0[3] = {(int64_t)compact3(ka) * wa, (int64_t)compact3(ka >> 1) * wa, (int64_t)compact3(ka >> 2) * wa};
  int64_t b0[3] = {(int64_t)compact3(kb) * wb + sx * D, (int64_t)compact3(kb >> 1) * wb + sy * D,
                   (int64_t)compact3(kb >> 2) * wb + sz * D};
  for (int d = 0; d < 3; ++d)
    if (a0[d] > b0[d] + wb || b0[d] > a0[d] + wa) return false;
  return true;
}

// Pair mobility difference (overlap form minus far form) applied to f, accumulated in acc.
template <class T>
__device__ inline void overlap_delta(T r0, T r1, T r2, T ai, T aj, T f0, T f1, T f2, T* acc) {
  T rr = r0 * r0 + r1 * r1 + r2 * r2;
  T rn = sqrt(rr);
  T s = ai + aj, d = fabs(ai - aj);
  if (rn > s) return;
  const T pi = T(PI);
  T A, B;
  if (rn > d) {
    T r3 = rr * rn, t = d * d + T(3) * rr, e = d * d - rr;
    A = (T(16) * r3 * s - t * t) / (T(32) * r3) / (T(6) * pi * ai * aj);
    B = T(3) * e * e / (T(32) * r3) / (T(6) * pi * ai * aj);
  } else {
    A = T(1) / (T(6) * pi * (ai > aj ? ai : aj));
    B = T(0);
  }
  T rf = r0 * f0 + r1 * f1 + r2 * f2;
  T bo = rr > T(0) ? B * rf / rr : T(0);
  T u0 = A * f0 + bo * r0, u1 = A * f1 + bo * r1, u2 = A * f2 + bo * r2;
  if (rr > T(0)) {  // subtract the far form (what the kernel sum already added)
    T c = ai * ai + aj * aj;
    T Af = (T(1) + c / (T(3) * rr)) / (T(8) * pi * rn);
    T Bf = (T(1) - c / rr) / (T(8) * pi * rn) * rf / rr;
    u0 -= Af * f0 + Bf * r0;
    u1 -= Af * f1 + Bf * r1;
    u2 -= Af * f2 + Bf * r2;
  }
  acc[0] += u0;
  acc[1] += u1;
  acc[2] += u2;
}

// Contact split (one shared point set): the near field left out the U-list pairs with
// r <= b_i + b_j, so those get their whole mobility here; contact pairs in the far-field lists
// keep the overlap-minus-far correction.
struct ContactInfo {
  int on;
  const int* leaf_of;      // [n_src] leaf box of each sorted point
  const int8_t* level;     // box levels
  const uint64_t* key;     // box Morton keys
};

template <class T, class Tio>
__global__ void k_rpy_velocity(const typename V4<T>::type* __restrict__ spos,
                               const typename V4<T>::type* __restrict__ sfb,
                               const typename V4<T>::type* __restrict__ tpos, const T* __restrict__ ta,
                               const uint64_t* __restrict__ tkey, const uint32_t* __restrict__ tperm,
                               int64_t nt, const int* __restrict__ cbeg, const int* __restrict__ cend, int g,
                               int H, double reach, double ox0, double oy0, double oz0, int periodic,
                               double L, int same, const Tio* __restrict__ gin, Tio* __restrict__ ua,
                               ContactInfo ci) {
  const int W = 2 * H + 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt;
       i += (int64_t)gridDim.x * blockDim.x) {
    typename V4<T>::type x = tpos[i];
    T ai = ta[i];
    T bi = ci.on ? sfb[i].w : T(0);   // the target's own source radius (shared point set)
    uint64_t ck = tkey[i] >> (3 * (MAX_LEVEL - g));
    int cx = (int)compact3(ck), cy = (int)compact3(ck >> 1), cz = (int)compact3(ck >> 2);
    int n = 1 << g;
    const double side = L / (double)n;
    // the target in cell units, relative to its own cell's low corner (cells farther than the
    // reach, taken with a margin, hold no contact partner)
    const double fx = ((double)x.x - ox0) / side - cx, fy = ((double)x.y - oy0) / side - cy,
                 fz = ((double)x.z - oz0) / side - cz;
    const double rc = reach / side * (1.0 + 1e-6) + 1e-6;
    T acc[3] = {0, 0, 0};
    for (int d = 0; d < W * W * W; ++d) {
      const int ddx = d % W - H, ddy = (d / W) % W - H, ddz = d / (W * W) - H;
      if (H > 1) {   // distance from the target to the neighbour cell's box, in cell units
        const double ex = ddx > 0 ? ddx - fx : (ddx < 0 ? fx - (ddx + 1) : 0.0);
        const double ey = ddy > 0 ? ddy - fy : (ddy < 0 ? fy - (ddy + 1) : 0.0);
        const double ez = ddz > 0 ? ddz - fz : (ddz < 0 ? fz - (ddz + 1) : 0.0);
        const double mx = ex > 0 ? ex : 0.0, my = ey > 0 ? ey : 0.0, mz = ez > 0 ? ez : 0.0;
        if (mx * mx + my * my + mz * mz > rc * rc) continue;
      }
      int qx = cx + ddx, qy = cy + ddy, qz = cz + ddz;
      // outside the cube: the image cell along a periodic axis (bit 0 = x, 1 = y, 2 = z of
      // periodic), none along an open one
      const int sx = qx < 0 ? -1 : (qx >= n ? 1 : 0);
      const int sy = qy < 0 ? -1 : (qy >= n ? 1 : 0);
      const int sz = qz < 0 ? -1 : (qz >= n ? 1 : 0);
      if ((sx && !(periodic & 1)) || (sy && !(periodic & 2)) || (sz && !(periodic & 4))) continue;
      qx -= sx * n;
      qy -= sy * n;
      qz -= sz * n;
      uint64_t c = morton3((uint32_t)qx, (uint32_t)qy, (uint32_t)qz);
      int b0 = cbeg[c], b1 = cend[c];
      T ox = (T)(sx * L), oy = (T)(sy * L), oz = (T)(sz * L);
      for (int j = b0; j < b1; ++j) {
        if (same && j == (int)i && sx == 0 && sy == 0 && sz == 0) continue;
        typename V4<T>::type y = spos[j], fb = sfb[j];
        T r0 = x.x - (y.x + ox), r1 = x.y - (y.y + oy), r2 = x.z - (y.z + oz);
        // clearly out of contact for both tests below (the overlap form's r <= a_i + b_j and
        // the near field's r <= b_i + b_j, each taken in its own arithmetic): nothing to add
        const T m = (ai > bi ? ai : bi) + fb.w;
        if (r0 * r0 + r1 * r1 + r2 * r2 > m * m * T(1.0001)) continue;
        if (ci.on) {   // the near field's contact test (its own radii, the same arithmetic)
          if (in_contact<T>(x.x, x.y, x.z, y.x, y.y, y.z, ox, oy, oz, bi, fb.w) &&
              leaves_adjacent(ci.level, ci.key, ci.leaf_of[i], ci.leaf_of[j], sx, sy, sz)) {
            pair_full<T>(r0, r1, r2, ai, fb.w, fb.x, fb.y, fb.z, acc);
            continue;
          }
        }
        overlap_delta<T>(r0, r1, r2, ai, fb.w, fb.x, fb.y, fb.z, acc);
      }
    }
    int64_t o = tperm[i];
    const Tio* gg = gin + 6 * o;
    T c6 = ai * ai / T(6);
    for (int k = 0; k < 3; ++k) ua[3 * o + k] = (Tio)((T)gg[k] + c6 * (T)gg[3 + k] + acc[k]);
  }
}

ContactInfo contact_info(const Plan& P) {
  ContactInfo ci;
  ci.on = P.contact_split() ? 1 : 0;
  ci.leaf_of = P.tree.leaf_of.as<int>();
  ci.level = P.tree.level.as<int8_t>();
  ci.key = P.tree.key.as<uint64_t>();
  return ci;
}

int grid_for(int64_t n, int threads, int maxb = 152 * 16) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > maxb) b = maxb;
  return (int)b;
}

#define CK(call)                                           \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(P, e_, #call); \
  } while (0)

template <class T>
int run(Plan& P, const void* s, const void* a, const void* g, void* ua, int dtype) {
  using T4 = typename V4<T>::type;
  Tree& Tr = P.tree;
  cudaStream_t st = P.stream;
  int64_t ns = Tr.n_src, nt = Tr.n_trg;
  const uint32_t* sperm = Tr.src_perm.as<uint32_t>();
  const uint32_t* tperm = Tr.same ? sperm : Tr.trg_perm.as<uint32_t>();
  const uint64_t* skey = Tr.src_key.as<uint64_t>();
  const uint64_t* tkey = Tr.same ? skey : Tr.trg_key.as<uint64_t>();
  DevBuf fb, ta, stat, cb, ce;
  CK(fb.reserve(sizeof(T4) * (ns + 1)));
  CK(ta.reserve(sizeof(T) * (nt + 1)));
  CK(stat.reserve(64));
  CK(cudaMemsetAsync(stat.p, 0, 64, st));
  if (dtype == KAFMM_F64) {
    KL k_gather_fb<double, T><<<grid_for(ns, 256), 256, 0, st>>>((const double*)s, sperm, ns, fb.as<T4>());
    KL k_gather_scalar<double, T><<<grid_for(nt, 256), 256, 0, st>>>((const double*)a, tperm, nt, ta.as<T>());
  } else {
    KL k_gather_fb<float, T><<<grid_for(ns, 256), 256, 0, st>>>((const float*)s, sperm, ns, fb.as<T4>());
    KL k_gather_scalar<float, T><<<grid_for(nt, 256), 256, 0, st>>>((const float*)a, tperm, nt, ta.as<T>());
  }
  KL k_max_radius<T><<<grid_for(std::max(ns, nt), 256), 256, 0, st>>>(ta.as<T>(), nt, fb.as<T4>(), ns,
                                                                       stat.as<unsigned>());
  unsigned h[2];
  CK(cudaMemcpyAsync(h, stat.p, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  float amax, bmax;
  memcpy(&amax, &h[0], 4);
  memcpy(&bmax, &h[1], 4);
  double reach = (std::max((double)amax, (double)bmax) + (double)bmax) * (1.0 + 1e-6) / P.L;
  // cells of at least half the reach and a 5^3 stencil where the grid has at least 5 cells per
  // side (level <= 8), else cells of at least the reach and 3^3
  int lev = 0, H = 1;
  while (lev < 8 && reach > 0 && 1.0 / (double)(1 << (lev + 1)) >= 0.5 * reach) ++lev;
  if (reach > 0 && lev >= 3 && 1.0 / (double)(1 << lev) >= 0.5 * reach) {
    H = 2;
  } else {
    lev = 0;
    while (lev < 8 && reach > 0 && 1.0 / (double)(1 << (lev + 1)) >= reach) ++lev;
  }
  if (reach <= 0) {
    lev = 8;
    H = 1;
  }
  int64_t ncell = 1ll << (3 * lev);
  CK(cb.reserve(sizeof(int) * ncell));
  CK(ce.reserve(sizeof(int) * ncell));
  CK(cudaMemsetAsync(cb.p, 0, sizeof(int) * ncell, st));
  CK(cudaMemsetAsync(ce.p, 0, sizeof(int) * ncell, st));
  if (ns > 0)
    KL k_cell_table<<<grid_for(ns, 256), 256, 0, st>>>(skey, ns, 3 * (MAX_LEVEL - lev), cb.as<int>(), ce.as<int>());
  const T4* spos = Tr.src_pos.as<T4>();
  const T4* tpos = Tr.same ? spos : Tr.trg_pos.as<T4>();
  if (nt > 0) {
    if (dtype == KAFMM_F64)
      KL k_rpy_velocity<T, double><<<grid_for(nt, 128), 128, 0, st>>>(
          spos, fb.as<T4>(), tpos, ta.as<T>(), tkey, tperm, nt, cb.as<int>(), ce.as<int>(), lev, H, reach * P.L,
          P.origin[0], P.origin[1], P.origin[2], periodic_mask(P.bc), P.L, Tr.same ? 1 : 0, (const double*)g,
          (double*)ua, contact_info(P));
    else
      KL k_rpy_velocity<T, float><<<grid_for(nt, 128), 128, 0, st>>>(
          spos, fb.as<T4>(), tpos, ta.as<T>(), tkey, tperm, nt, cb.as<int>(), ce.as<int>(), lev, H, reach * P.L,
          P.origin[0], P.origin[1], P.origin[2], periodic_mask(P.bc), P.L, Tr.same ? 1 : 0, (const float*)g,
          (float*)ua, contact_info(P));
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return 0;
}

// ---------------------------------------------------------------------------------------
// Variant without allocations: the per-call work arrays (gathered forces and radii, the cell
// table, the radius maxima) live in one file-scope device array instead of cudaMalloc'd
// buffers.  Every GPU that loads the library holds the array until the process exits.  Calls
// share it, so two calls that overlap on the GPU race; each call clears what must start at
// zero.  The cell grid is capped at level 6 (a coarser grid than the contact radius asks for
// is still exact, only slower).
constexpr size_t NOALLOC_BYTES = (size_t)32 << 20;   // 32 MiB
constexpr int NOALLOC_MAX_CELL_LEVEL = 6;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Host-side address of the array in the CUDA context current on this thread.  A module's
// device variables live per context, and cudaDeviceReset replaces the device's primary context,
// so the address is looked up once per context (keyed by the driver's context id, which a new
// context never reuses), with that context current.
static unsigned char* noalloc_base(Plan& P, int* rc) {
  typedef CUresult (*CtxCurrentFn)(CUcontext*);
  typedef CUresult (*CtxIdFn)(CUcontext, unsigned long long*);
  static std::mutex mu;
  static CtxCurrentFn ctx_current = nullptr;
  static CtxIdFn ctx_id = nullptr;
  static unsigned long long ids[64] = {0};
  static unsigned char* addr[64] = {nullptr};
  static int n_cached = 0, next_evict = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaSetDevice(dev);   // makes the device's primary context current
  if (e != cudaSuccess) {
    *rc = cuda_fail(P, e, "cudaGetDevice / cudaSetDevice");
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!ctx_current || !ctx_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &f1, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPoint("cuCtxGetId", &f2, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
      cudaGetLastError();
      *rc = fail(P, KAFMM_ERR_CUDA, "cuCtxGetCurrent / cuCtxGetId are unavailable");
      return nullptr;
    }
    ctx_current = reinterpret_cast<CtxCurrentFn>(f1);
    ctx_id = reinterpret_cast<CtxIdFn>(f2);
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (ctx_current(&ctx) != CUDA_SUCCESS || !ctx || ctx_id(ctx, &id) != CUDA_SUCCESS) {
    *rc = fail(P, KAFMM_ERR_CUDA, "no current CUDA context");
    return nullptr;
  }
  for (int i = 0; i < n_cached; ++i)
    if (ids[i] == id) {
      *rc = 0;
      return addr[i];
    }
  void* ptr = nullptr;
  e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || !ptr) {
    *rc = cuda_fail(P, e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress(scratch)");
    return nullptr;
  }
  int slot = n_cached < 64 ? n_cached++ : (next_evict++ % 64);   // a full table reuses slots in turn
  ids[slot] = id;
  addr[slot] = reinterpret_cast<unsigned char*>(ptr);
  *rc = 0;
  return addr[slot];
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <class T>
int run_noalloc(Plan& P, const void* s, const void* a, const void* g, void* ua, int dtype) {
  using T4 = typename V4<T>::type;
  Tree& Tr = P.tree;
  cudaStream_t st = P.stream;
  int64_t ns = Tr.n_src, nt = Tr.n_trg;
  const int64_t ncell_max = 1ll << (3 * NOALLOC_MAX_CELL_LEVEL);
  size_t need = 256 + align256(sizeof(T4) * (ns + 1)) + align256(sizeof(T) * (nt + 1)) +
                2 * align256(sizeof(int) * ncell_max);
  if (need > NOALLOC_BYTES)
    return fail(P, KAFMM_ERR_ARG,
                "kafmm_rpy_velocity_noalloc: %lld sources and %lld targets need %zu bytes of "
                "scratch, more than the fixed %zu bytes (use kafmm_rpy_velocity)",
                (long long)ns, (long long)nt, need, NOALLOC_BYTES);
  int rc = 0;
  unsigned char* base = noalloc_base(P, &rc);
  if (rc) return rc;
  unsigned* stat = reinterpret_cast<unsigned*>(base);
  T4* fb = reinterpret_cast<T4*>(base + 256);
  T* ta = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(fb) + align256(sizeof(T4) * (ns + 1)));
  int* cb = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(ta) + align256(sizeof(T) * (nt + 1)));
  int* ce = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(cb) + align256(sizeof(int) * ncell_max));
  const uint32_t* sperm = Tr.src_perm.as<uint32_t>();
  const uint32_t* tperm = Tr.same ? sperm : Tr.trg_perm.as<uint32_t>();
  const uint64_t* skey = Tr.src_key.as<uint64_t>();
  const uint64_t* tkey = Tr.same ? skey : Tr.trg_key.as<uint64_t>();
  CK(cudaMemsetAsync(stat, 0, 64, st));
  if (dtype == KAFMM_F64) {
    KL k_gather_fb<double, T><<<grid_for(ns, 256), 256, 0, st>>>((const double*)s, sperm, ns, fb);
    KL k_gather_scalar<double, T><<<grid_for(nt, 256), 256, 0, st>>>((const double*)a, tperm, nt, ta);
  } else {
    KL k_gather_fb<float, T><<<grid_for(ns, 256), 256, 0, st>>>((const float*)s, sperm, ns, fb);
    KL k_gather_scalar<float, T><<<grid_for(nt, 256), 256, 0, st>>>((const float*)a, tperm, nt, ta);
  }
  KL k_max_radius<T><<<grid_for(std::max(ns, nt), 256), 256, 0, st>>>(ta, nt, fb, ns, stat);
  unsigned h[2];
  CK(cudaMemcpyAsync(h, stat, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  float amax, bmax;
  memcpy(&amax, &h[0], 4);
  memcpy(&bmax, &h[1], 4);
  double reach = (std::max((double)amax, (double)bmax) + (double)bmax) * (1.0 + 1e-6) / P.L;
  int lev = 0;
  while (lev < NOALLOC_MAX_CELL_LEVEL && reach > 0 && 1.0 / (double)(1 << (lev + 1)) >= reach) ++lev;
  if (reach <= 0) lev = NOALLOC_MAX_CELL_LEVEL;
  int64_t ncell = 1ll << (3 * lev);
  CK(cudaMemsetAsync(cb, 0, sizeof(int) * ncell, st));
  CK(cudaMemsetAsync(ce, 0, sizeof(int) * ncell, st));
  if (ns > 0)
    KL k_cell_table<<<grid_for(ns, 256), 256, 0, st>>>(skey, ns, 3 * (MAX_LEVEL - lev), cb, ce);
  const T4* spos = Tr.src_pos.as<T4>();
  const T4* tpos = Tr.same ? spos : Tr.trg_pos.as<T4>();
  if (nt > 0) {
    if (dtype == KAFMM_F64)
      KL k_rpy_velocity<T, double><<<grid_for(nt, 128), 128, 0, st>>>(
          spos, fb, tpos, ta, tkey, tperm, nt, cb, ce, lev, 1, reach * P.L, P.origin[0], P.origin[1], P.origin[2],
          periodic_mask(P.bc), P.L, Tr.same ? 1 : 0, (const double*)g, (double*)ua, contact_info(P));
    else
      KL k_rpy_velocity<T, float><<<grid_for(nt, 128), 128, 0, st>>>(
          spos, fb, tpos, ta, tkey, tperm, nt, cb, ce, lev, 1, reach * P.L, P.origin[0], P.origin[1], P.origin[2],
          periodic_mask(P.bc), P.L, Tr.same ? 1 : 0, (const float*)g, (float*)ua, contact_info(P));
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return 0;
}

}  // namespace

int rpy_velocity(Plan& P, const void* s, const void* a, const void* g, void* ua, int dtype) {
  return P.fp64() ? run<double>(P, s, a, g, ua, dtype) : run<float>(P, s, a, g, ua, dtype);
}

int rpy_velocity_noalloc(Plan& P, const void* s, const void* a, const void* g, void* ua, int dtype) {
  return P.fp64() ? run_noalloc<double>(P, s, a, g, ua, dtype) : run_noalloc<float>(P, s, a, g, ua, dtype);
}

}  // namespace kafmm
