// The KAFMM evaluation (Sec. II, Fig. kifmmgraph): S->M, M->M, M->L, S->L, L->L, and at the
// leaves L->T, M->T, S->T; CUDA-core kernels in FP32 or FP64.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "physics.cuh"
#include "plan.cuh"

namespace kafmm {

int tc_gemm_launch(Plan& P, int mode, int opset, const int4* tiles, int ntiles, const int* boxlist,
                   const float* in, float* out, int op, int write, cudaStream_t st);
// modes and output kinds of tc_gemm_launch (m2l_tc.cu)
constexpr int TCM_M2L = 0, TCM_M2M = 1, TCM_L2L = 2, TCM_APPLY = 3;
constexpr int TCW_STORE = 0, TCW_ADD = 1, TCW_SCALE = 2;

// ---------------------------------------------------------------------------------------
// Geometry helpers.
template <class T>
__device__ inline void box_centre(const TreeView& t, int b, double L, const double* org, T& cx, T& cy,
                                  T& cz, T& r) {
  int lv = t.level[b];
  uint64_t k = t.key[b];
  double side = L / (double)(1 << lv);
  cx = (T)(org[0] + ((double)compact3(k) + 0.5) * side);
  cy = (T)(org[1] + ((double)compact3(k >> 1) + 0.5) * side);
  cz = (T)(org[2] + ((double)compact3(k >> 2) + 0.5) * side);
  r = (T)(0.5 * side);
}

struct Geo {
  double L;
  double org[3];
};

// ---------------------------------------------------------------------------------------
// Source values to sorted compute-type records (T4 per source; DL: 3 T4).
template <class Tin, class T, int PR>
__global__ void k_prep_src(const Tin* __restrict__ s, const uint32_t* __restrict__ perm, int64_t n,
                           typename V4<T>::type* __restrict__ out) {
  using T4 = typename V4<T>::type;
  constexpr int KS =
      PR == P_LAP ? 1
                  : ((dl_src(PR) || PR == P_LAPQ) ? 9
                                : ((PR == P_RPY_L4 || PR == P_RPY_G || PR == P_REG_G || PR == P_LAPQD || pvel_src(PR))
                                       ? 4
                                       : 3));
  constexpr int NV = ProbInfo<PR>::NV;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const Tin* src = s + (int64_t)perm[i] * KS;
    T v[4 * NV];
#pragma unroll
    for (int k = 0; k < 4 * NV; ++k) v[k] = k < KS ? (T)src[k] : T(0);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      T4 r;
      r.x = v[4 * q];
      r.y = v[4 * q + 1];
      r.z = v[4 * q + 2];
      r.w = v[4 * q + 3];
      out[i * NV + q] = r;
    }
  }
}

// Derivative target values back to the caller's order and dtype, from [p, u, grad p, grad u]
// per sorted target: mode 0 all 16; mode 1 [p, u, lap u] with lap u = grad p (the Stokes
// equation off the sources, mu = 1, which every source and equivalent point's field solves);
// mode 2 the traction sigma_ij = -p delta_ij + d_j u_i + d_i u_j at 3 i + j (Eq. stressdef).
template <class T, class Tout>
__global__ void k_unperm_deriv(const T* __restrict__ g, const uint32_t* __restrict__ perm, int64_t n, int mode,
                               Tout* __restrict__ out) {
  const int kt = mode == 0 ? 16 : (mode == 1 ? 7 : 9);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * kt;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / kt;
    const int k = (int)(e % kt);
    const T* v = g + 16 * i;
    T o;
    if (mode == 2) {
      const int a = k / 3, b = k % 3;
      o = v[7 + 3 * a + b] + v[7 + 3 * b + a] - (a == b ? v[0] : T(0));
    } else {
      o = v[k];   // mode 1: lap u_i = d_i p are entries 4..6
    }
    out[(int64_t)perm[i] * kt + k] = (Tout)o;
  }
}

// Sorted results back to the caller's order and dtype.
template <class T, class Tout>
__global__ void k_unperm(const T* __restrict__ g, const uint32_t* __restrict__ perm, int64_t n, int kt,
                         Tout* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * kt;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / kt;
    int k = (int)(e % kt);
    out[(int64_t)perm[i] * kt + k] = (Tout)g[e];
  }
}

// ---------------------------------------------------------------------------------------
// S->M (leaf sources to the upward check surface) and S->L (X-list sources to the downward
// check surface).  One block per box; check points over threads; sources staged in shared
// memory in local coordinates (relative to the box centre, which is also the reference
// point of the four-channel table).
template <class T, int PR>
struct S2CArgs {
  TreeView t;
  Geo geo;
  const typename V4<T>::type* pos;   // sorted source positions
  const typename V4<T>::type* val;   // sorted source values
  const T* unit;                     // unit surface [n][3]
  const int* boxes;
  const int64_t* x_off;
  const int32_t* x_ent;
  T* check;
  int n, R;
  int mode;                          // 0: S->M (overwrite), 1: S->L over X lists (accumulate)
};

// Check points per thread of k_s2check: each staged source feeds CPT check points.
constexpr int S2C_CPT = 4;

template <class T, int PR>
__global__ void __launch_bounds__(128) k_s2check(S2CArgs<T, PR> a) {
  using T4 = typename V4<T>::type;
  constexpr int C = ProbInfo<PR>::C, D = ProbInfo<PR>::D, NV = ProbInfo<PR>::NV;
  constexpr int CH = 256;
  __shared__ T4 sp[CH], sv[CH * NV];
  int b = a.boxes[blockIdx.x];
  T cx, cy, cz, r;
  box_centre<T>(a.t, b, a.geo.L, a.geo.org, cx, cy, cz, r);
  T alpha = a.mode == 0 ? T(ALPHA_UC) : T(ALPHA_DC);
  int nent = a.mode == 0 ? 1 : (int)(a.x_off[b + 1] - a.x_off[b]);
  // check points i0 + threadIdx.x + 128 u (u < S2C_CPT) of this pass
  for (int i0 = 0; i0 < a.n; i0 += 128 * S2C_CPT) {
    T px[S2C_CPT], py[S2C_CPT], pz[S2C_CPT];
    bool on[S2C_CPT];
    T acc[S2C_CPT][C * D];
#pragma unroll
    for (int u = 0; u < S2C_CPT; ++u) {
      const int i = i0 + threadIdx.x + 128 * u;
      on[u] = i < a.n;
      px[u] = py[u] = pz[u] = 0;
      if (on[u]) {
        px[u] = alpha * r * a.unit[3 * i];
        py[u] = alpha * r * a.unit[3 * i + 1];
        pz[u] = alpha * r * a.unit[3 * i + 2];
      }
#pragma unroll
      for (int k = 0; k < C * D; ++k) acc[u][k] = 0;
    }
    for (int e = 0; e < nent; ++e) {
      int src = b, sc = 13;
      if (a.mode == 1) {
        int32_t ent = a.x_ent[a.x_off[b] + e];
        src = entry_box(ent);
        sc = entry_shift(ent);
      }
      int sx, sy, sz;
      shift_decode(sc, sx, sy, sz);
      T ox = (T)(sx * a.geo.L) - cx, oy = (T)(sy * a.geo.L) - cy, oz = (T)(sz * a.geo.L) - cz;
      int s0 = a.t.sb[src], s1 = a.t.se[src];
      for (int c0 = s0; c0 < s1; c0 += CH) {
        int cn = min(CH, s1 - c0);
        __syncthreads();
        for (int j = threadIdx.x; j < cn; j += blockDim.x) {
          T4 p = a.pos[c0 + j];
          p.x = p.x + ox;  // local source coordinates
          p.y = p.y + oy;
          p.z = p.z + oz;
          sp[j] = p;
#pragma unroll
          for (int qv = 0; qv < NV; ++qv) sv[j * NV + qv] = a.val[(int64_t)(c0 + j) * NV + qv];
        }
        __syncthreads();
        if (!on[0]) continue;
        for (int j = 0; j < cn; ++j) {
          const T4 y = sp[j], v = sv[j * NV];
#pragma unroll
          for (int u = 0; u < S2C_CPT; ++u) {
            if (!on[u]) continue;
            T r0 = px[u] - y.x, r1 = py[u] - y.y, r2 = pz[u] - y.z;
            T* ac = acc[u];
            if (dl_src(PR)) {   // S->M, S->L: the double-layer kernel K, [p, u] (p doubled: 1/(8 pi) below)
              T4 v1 = sv[j * NV + 1], v2 = sv[j * NV + 2];
              T Dm[9] = {v.x, v.y, v.z, v.w, v1.x, v1.y, v1.z, v1.w, v2.x};
              T tmp[4] = {0, 0, 0, 0};
              dl_st<T>(r0, r1, r2, Dm, tmp);
              ac[0] += T(2) * tmp[0];
              ac[1] += tmp[1];
              ac[2] += tmp[2];
              ac[3] += tmp[3];
            } else if (pvel_src(PR)) {   // S->M, S->L: G^P, [p, u] (p doubled: 1/(8 pi) below)
              T tmp[4] = {0, 0, 0, 0};
              pvel_st<T>(r0, r1, r2, v.x, v.y, v.z, v.w, tmp);
              ac[0] += T(2) * tmp[0];
              ac[1] += tmp[1];
              ac[2] += tmp[2];
              ac[3] += tmp[3];
            } else if (PR == P_LAP) {
              lap_st<T>(r0, r1, r2, v.x, ac);
            } else if (PR == P_LAPQ) {   // S->M, S->L: the quadrupole potential
              T4 v1 = sv[j * NV + 1], v2 = sv[j * NV + 2];
              T Qm[9] = {v.x, v.y, v.z, v.w, v1.x, v1.y, v1.z, v1.w, v2.x};
              T tmp[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
              quad_st<T>(r0, r1, r2, Qm, tmp);
              ac[0] += tmp[0];
            } else if (PR == P_LAPQD) {   // S->M, S->L: L for the charge, L^D for the dipole
              T rr = r0 * r0 + r1 * r1 + r2 * r2;
              T ir = inv_r(rr);
              ac[0] += v.x * ir + (v.y * r0 + v.z * r1 + v.w * r2) * ir * ir * ir;
            } else if (PR == P_STK_L4 || PR == P_RPY_L4) {
              T rr = r0 * r0 + r1 * r1 + r2 * r2;
              T ir = inv_r(rr);
              ac[0] += v.x * ir;
              ac[1] += v.y * ir;
              ac[2] += v.z * ir;
              T q4 = y.x * v.x + y.y * v.y + y.z * v.z;  // (y - c) . f
              if (PR == P_RPY_L4) q4 = q4 + v.w * v.w * T(1.0 / 3.0) * (r0 * v.x + r1 * v.y + r2 * v.z) * ir * ir;
              ac[3] += q4 * ir;
            } else if (PR == P_STK_G) {
              stk_st<T>(r0, r1, r2, v.x, v.y, v.z, ac);
            } else if (PR == P_REG_G) {   // S->M, S->L: the regularized kernel (Table tab:ktab_reg)
              reg_st<T>(r0, r1, r2, v.x, v.y, v.z, v.w, ac);
            } else if (PR == P_RPY_G) {
              T tmp[6] = {0, 0, 0, 0, 0, 0};
              rpy_st<T>(r0, r1, r2, v.x, v.y, v.z, v.w, tmp);
              ac[0] += tmp[0];
              ac[1] += tmp[1];
              ac[2] += tmp[2];
            }
          }
        }
      }
    }
    T sc = (PR == P_STK_G || PR == P_RPY_G || PR == P_REG_G || pvel_table(PR))
               ? T(1.0 / (8.0 * PI))
               : T(1.0 / (4.0 * PI));
    T* out = a.check + (int64_t)b * a.R * C;
#pragma unroll
    for (int u = 0; u < S2C_CPT; ++u) {
      if (!on[u]) continue;
      const int i = i0 + threadIdx.x + 128 * u;
#pragma unroll
      for (int d = 0; d < D; ++d)
#pragma unroll
        for (int c = 0; c < C; ++c) {
          int64_t idx = (int64_t)(i * D + d) * C + c;
          T v = acc[u][d * C + c] * sc;
          // StokesPVel check values are stored as [h p, u] (h: box half-width), which makes
          // the translations level-independent (p falls as 1/r^2, u as 1/r)
          if (pvel_table(PR) && d == 0) v *= r;
          if (a.mode == 0)
            out[idx] = v;
          else
            out[idx] += v;
        }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Gather-GEMM engine on CUDA cores: for each output box b of a tile (all of one octant class),
//   out[b] (+)= alpha_b * sum_k Op[op(k)] * shift_k(in[src(b, k)])
// with [R][C] per box.  Modes: M->L over the 216 V slots, M->M over 8 children, L->L from the
// parent, and the check-to-equivalent pseudo-inverses (alpha_b = box half-width).
// GM_APPLY: one operator (args.op) on the box itself; args.scale_r multiplies by the box
// half-width (the level scaling of a pseudo-inverse).
enum GemmMode { GM_M2L = 0, GM_M2M = 1, GM_L2L = 2, GM_APPLY = 3 };

template <class T>
struct GemmArgs {
  TreeView t;
  Geo geo;
  const T* ops;
  const T* in;
  T* out;
  const int4* tiles;   // (offset into boxlist, count, class, unused)
  const int* boxlist;
  const int32_t* vtab;
  int mode, R;
  int op, scale_r;
  int qscale4;         // StokesPVel table: rows 4k+3 (q) of a scaled apply get the half-width again
};

template <int C>
struct GemmShape { static constexpr int NB = 64 / C; };
constexpr int GEMM_BM = 128;   // operator rows per CTA of k_gemm

__device__ inline void m2l_slot_offset(int k, int cls, int& ox, int& oy, int& oz) {
  ox = k % 6 - 2 - (cls & 1);
  oy = (k / 6) % 6 - 2 - ((cls >> 1) & 1);
  oz = k / 36 - 2 - ((cls >> 2) & 1);
}

// Gather-GEMM on the CUDA cores: out[box] (+)= sum over slots of op_slot (R x R) times the
// slot's source column block (R x C, the four-channel block re-referenced to the target
// centre).  A CTA owns 128 rows x 64 columns (64 / C boxes of one octant class); each thread
// an 8 x 4 register tile (8 rows, one box's four channels when C = 4); operator and source
// chunks of BK k-values are double-buffered in shared memory (loads of chunk c + 1 in flight
// while chunk c is multiplied).  FP32 M->L: three-level summation (BK-term chunk -> slot ->
// total), so no single FP32 accumulator runs over all 189 x R terms; the other modes (at most
// 8 slots) sum BK-term chunks into the total.
template <class T, int C, bool M2L>
__global__ void __launch_bounds__(256, M2L ? 1 : 2) k_gemm(GemmArgs<T> a) {
  using T4 = typename V4<T>::type;
  // the per-slot partial level of the summation is kept for the 189-slot M->L sums only; the
  // other modes have at most 8 slots (and run two CTAs per SM in the registers saved)
  constexpr bool THREE = sizeof(T) == 4 && M2L;
  constexpr int NB = GemmShape<C>::NB, BM = GEMM_BM, BN = 64, BK = sizeof(T) == 4 ? 16 : 8, TM = 8,
                TN = 4;
  constexpr int AP = BM + 4, BP = BN + 4;               // padded rows (bank spread, 16 B aligned)
  constexpr int A_PER = BM * BK / 256;                  // operator loads per thread per chunk
  constexpr int B_PER = C == 4 ? (BK * NB + 255) / 256 : BK * NB / 256;
  __shared__ __align__(16) T As[2][BK][AP];
  __shared__ __align__(16) T Bs[2][BK][BP];
  __shared__ int ob[NB], srcb[NB];
  __shared__ T dcx[NB], dcy[NB], dcz[NB], alph[NB];
  const int4 tile = a.tiles[blockIdx.x];
  const int row0 = blockIdx.y * BM;
  const int cls = tile.z;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  if (tid < NB) {
    int b = tid < tile.y ? a.boxlist[tile.x + tid] : -1;
    ob[tid] = b;
    T al = 1;
    if (b >= 0 && a.mode == GM_APPLY && a.scale_r)
      al = (T)(0.5 * a.geo.L / (double)(1 << a.t.level[b]));
    alph[tid] = al;
  }
  __syncthreads();
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0;
  const int nslots = a.mode == GM_M2L ? 216 : (a.mode == GM_M2M ? 8 : 1);
  const int R = a.R;
  const int nch = (R + BK - 1) / BK;
  for (int k = 0; k < nslots; ++k) {
    int op = 0;
    int ox = 0, oy = 0, oz = 0;
    if (a.mode == GM_M2L) {
      m2l_slot_offset(k, cls, ox, oy, oz);
      if (abs(ox) <= 1 && abs(oy) <= 1 && abs(oz) <= 1) continue;
      op = OP_M2L + m2l_index(ox, oy, oz);
    } else if (a.mode == GM_M2M) {
      op = OP_M2M + k;
    } else if (a.mode == GM_L2L) {
      op = OP_L2L + cls;
    } else {
      op = a.op;
    }
    int has = 0;
    if (tid < NB) {
      int b = ob[tid], s = -1;
      T dx = 0, dy = 0, dz = 0;
      if (b >= 0) {
        int lv = a.t.level[b];
        double side = a.geo.L / (double)(1 << lv);
        if (a.mode == GM_M2L) {
          int32_t e = a.vtab[(int64_t)b * 216 + k];
          if (e != LIST_EMPTY) {
            s = entry_box(e);
            dx = (T)(ox * side);
            dy = (T)(oy * side);
            dz = (T)(oz * side);
          }
        } else if (a.mode == GM_M2M) {
          s = a.t.child[b * 8 + k];
          dx = (T)(((k & 1) ? 0.25 : -0.25) * side);
          dy = (T)(((k & 2) ? 0.25 : -0.25) * side);
          dz = (T)(((k & 4) ? 0.25 : -0.25) * side);
        } else if (a.mode == GM_L2L) {
          s = a.t.parent[b];
          dx = (T)(((cls & 1) ? -0.5 : 0.5) * side);
          dy = (T)(((cls & 2) ? -0.5 : 0.5) * side);
          dz = (T)(((cls & 4) ? -0.5 : 0.5) * side);
        } else {
          s = b;
        }
      }
      srcb[tid] = s;
      dcx[tid] = dx;
      dcy[tid] = dy;
      dcz[tid] = dz;
      has = s >= 0;
    }
    if (!__syncthreads_or(has)) continue;
    const T* opp = a.ops + (int64_t)op * R * R;
    T ra[A_PER];
    T4 rb4[C == 4 ? B_PER : 1];
    T rb1[C == 4 ? 1 : B_PER];
    // global -> registers for chunk ch (zero outside R)
    auto load = [&](int ch) {
      int k0 = ch * BK;
#pragma unroll
      for (int q = 0; q < A_PER; ++q) {
        int e = q * 256 + tid;
        int row = e / BK, kk = e % BK;
        int gr = row0 + row, gk = k0 + kk;
        ra[q] = (gr < R && gk < R) ? __ldg(opp + (int64_t)gr * R + gk) : T(0);
      }
      if constexpr (C == 4) {
#pragma unroll
        for (int q = 0; q < B_PER; ++q) {
          int e = q * 256 + tid;
          int kk = e / NB, j = e % NB;
          int gk = k0 + kk;
          int sb = (kk < BK) ? srcb[j] : -1;
          T4 v;
          if (sb >= 0 && gk < R) {
            const T4* src = reinterpret_cast<const T4*>(a.in) + (int64_t)sb * R + gk;
            if constexpr (sizeof(T) == 4)
              v = __ldg(src);
            else
              v = *src;
            v.w = v.w + dcx[j] * v.x + dcy[j] * v.y + dcz[j] * v.z;
          } else {
            v.x = v.y = v.z = v.w = 0;
          }
          rb4[q] = v;
        }
      } else {
#pragma unroll
        for (int q = 0; q < B_PER; ++q) {
          int e = q * 256 + tid;
          int kk = e / NB, j = e % NB;
          int gk = k0 + kk, sb = srcb[j];
          rb1[q] = (sb >= 0 && gk < R) ? __ldg(a.in + (int64_t)sb * R + gk) : T(0);
        }
      }
    };
    auto store = [&](int buf) {
#pragma unroll
      for (int q = 0; q < A_PER; ++q) {
        int e = q * 256 + tid;
        As[buf][e % BK][e / BK] = ra[q];
      }
      if constexpr (C == 4) {
#pragma unroll
        for (int q = 0; q < B_PER; ++q) {
          int e = q * 256 + tid;
          int kk = e / NB, j = e % NB;
          if (kk < BK) *reinterpret_cast<T4*>(&Bs[buf][kk][j * 4]) = rb4[q];
        }
      } else {
#pragma unroll
        for (int q = 0; q < B_PER; ++q) {
          int e = q * 256 + tid;
          Bs[buf][e / NB][e % NB] = rb1[q];
        }
      }
    };
    T part[THREE ? TM : 1][THREE ? TN : 1];
    if constexpr (THREE) {
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) part[i][j] = 0;
    }
    load(0);
    store(0);
    __syncthreads();
    for (int ch = 0; ch < nch; ++ch) {
      const int buf = ch & 1;
      if (ch + 1 < nch) load(ch + 1);
      T chunk[TM][TN];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) chunk[i][j] = 0;
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T av[TM], bv[TN];
        if constexpr (sizeof(T) == 4) {
          float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * TM]);
          float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * TM + 4]);
          float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * TN]);
          av[0] = a0.x; av[1] = a0.y; av[2] = a0.z; av[3] = a0.w;
          av[4] = a1.x; av[5] = a1.y; av[6] = a1.z; av[7] = a1.w;
          bv[0] = b0.x; bv[1] = b0.y; bv[2] = b0.z; bv[3] = b0.w;
        } else {
#pragma unroll
          for (int i = 0; i < TM; ++i) av[i] = As[buf][kk][ty * TM + i];
#pragma unroll
          for (int j = 0; j < TN; ++j) bv[j] = Bs[buf][kk][tx * TN + j];
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) chunk[i][j] = fma(av[i], bv[j], chunk[i][j]);
      }
      if constexpr (THREE) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) part[i][j] += chunk[i][j];
      } else {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] += chunk[i][j];
      }
      if (ch + 1 < nch) store(buf ^ 1);
      __syncthreads();
    }
    if constexpr (THREE) {
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] += part[i][j];
    }
  }
  const bool accumulate = a.mode == GM_M2L || a.mode == GM_L2L;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int row = row0 + ty * TM + i;
    if (row >= R) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int col = tx * TN + j;
      int bj = col / C, c = col % C;
      int b = ob[bj];
      if (b < 0) continue;
      T* o = a.out + ((int64_t)b * R + row) * C + c;
      T v = alph[bj] * acc[i][j];
      if (a.qscale4 && (row & 3) == 3) v *= alph[bj];
      if (accumulate)
        *o += v;
      else
        *o = v;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Leaf kernel: L->T (own downward equivalent density), M->T over the W list, S->T over the
// U list (source tiles staged by bulk async copies), one block per target leaf.
template <class T, int PR>
struct LeafArgs {
  TreeView t;
  Geo geo;
  const typename V4<T>::type* spos;  // sorted sources
  const typename V4<T>::type* sval;
  const typename V4<T>::type* tpos;  // sorted targets
  const T* unit;
  const T* dn_equiv;                 // [nbox][R][C]
  const T* up_equiv;
  const int* leaves;
  const int64_t* u_off;
  const int32_t* u_ent;
  const int64_t* w_off;
  const int32_t* w_ent;
  T* g;                              // sorted targets [nt][KT]
  unsigned* status;
  WaitLimits lim;                    // bounds of the mbarrier waits
  int stall_test;                    // test aid: first wait on a barrier nothing completes
  int n, R, near_only, kahan;
  int contact;                       // RPY: skip U-list pairs within contact (r <= b_i + b_j)
  int cap;                           // staging capacity in sources
};

constexpr int LEAF_THREADS = 128;
constexpr int LEAF_MAX_ENT = 64;

template <class T, int PR>
__device__ inline void far_eval(T xl, T yl, T zl, const typename V4<T>::type& p,
                                const typename V4<T>::type& q, T* acc) {
  // p: equivalent point (local coords), q: its density (C = 4: four channels; C = 1 G: q.xyz).
  T r0 = xl - p.x, r1 = yl - p.y, r2 = zl - p.z;
  if constexpr (PR == P_STK_L4 && sizeof(T) == 4) {
    // as below; equivalent points lie on surfaces outside the target box, so r > 0
    float rr = fmaf(r0, r0, fmaf(r1, r1, r2 * r2));
    float ir = rsqrt_ftz(rr);
    float tq = (fmaf(xl, q.x, fmaf(yl, q.y, zl * q.z)) - q.w) * (ir * ir * ir);
    acc[0] = fmaf(r0, tq, fmaf(q.x, ir, acc[0]));
    acc[1] = fmaf(r1, tq, fmaf(q.y, ir, acc[1]));
    acc[2] = fmaf(r2, tq, fmaf(q.z, ir, acc[2]));
  } else if (PR == P_LAP) {
    lap_st<T>(r0, r1, r2, q.x, acc);
  } else if (PR == P_DL || PR == P_PVEL) {   // M->T, L->T: StokesPVel from the equivalent [f, q]
    pvel_st<T>(r0, r1, r2, q.x, q.y, q.z, q.w, acc);
  } else if (deriv_out(PR)) {   // M->T, L->T: G^P + grad G^P from the equivalent [f, q]
    pvel_grad_st<T>(r0, r1, r2, q.x, q.y, q.z, q.w, acc);
  } else if (PR == P_LAPQD || PR == P_LAPQ) {   // M->T, L->T: equivalent charges, L + grad L + grad grad L
    lapqd_st<T, false>(r0, r1, r2, q.x, T(0), T(0), T(0), acc);
  } else if (PR == P_STK_L4 || PR == P_RPY_L4) {
    // 8 pi u_i = 2 [phi_i - x_j d_i phi_j + d_i phi_4] with phi = q/r (reference: leaf centre)
    T rr = r0 * r0 + r1 * r1 + r2 * r2;
    T ir = inv_r(rr);
    T ir3 = ir * ir * ir;
    T tq = (xl * q.x + yl * q.y + zl * q.z - q.w) * ir3;
    acc[0] += q.x * ir + r0 * tq;
    acc[1] += q.y * ir + r1 * tq;
    acc[2] += q.z * ir + r2 * tq;
    if (PR == P_RPY_L4) {  // 4 pi lap u_i = q_i / r^3 - 3 r_i (r.q) / r^5
      T c3 = T(3) * (r0 * q.x + r1 * q.y + r2 * q.z) * ir * ir;
      acc[3] += (q.x - r0 * c3) * ir3;
      acc[4] += (q.y - r1 * c3) * ir3;
      acc[5] += (q.z - r2 * c3) * ir3;
    }
  } else if (PR == P_STK_G || PR == P_REG_G) {   // M->T, L->T: the singular Stokeslet
    stk_st<T>(r0, r1, r2, q.x, q.y, q.z, acc);
  } else if (PR == P_RPY_G) {
    rpy_st<T>(r0, r1, r2, q.x, q.y, q.z, T(0), acc);
  }
}

// Targets per thread of the leaf kernel: in the FP32 form four for the Stokeslet (each staged
// source or equivalent point then feeds four independent pair evaluations), two for the other
// tables of at most six outputs, one otherwise.
template <class T, int PR>
struct LeafTT {
  static constexpr int V = sizeof(T) != 4 ? 1 : ((PR == P_STK_L4 || PR == P_STK_G) ? 4 : (ProbInfo<PR>::KT <= 6 ? 2 : 1));
};

// Leaf kernel, one block per target leaf.  Work split: a pass takes up to LEAF_THREADS x tt
// targets (tt = 4 when the leaf holds more than 32 and the table allows it, 2 when it holds more
// than 16); its targets are
// dealt to S slots of tt targets each, and the G = LEAF_THREADS / S threads of a slot (lane-major:
// consecutive lanes) split the sources of every interaction list among themselves; the G
// partial sums of a target are combined by warp shuffles when G divides 32, else through
// shared memory.  Far field first (L->T from the leaf's own downward equivalent density, M->T
// over the W list; equivalent points generated in shared memory), then the U list S->T with the
// sources staged by cp.async.bulk into two buffers: the copies of batch i + 1 are in flight while
// batch i is evaluated.
template <class T, int PR>
__global__ void __launch_bounds__(LEAF_THREADS) k_leaf(LeafArgs<T, PR> a) {
  using T4 = typename V4<T>::type;
  constexpr int KT = ProbInfo<PR>::KT, C = ProbInfo<PR>::C, D = ProbInfo<PR>::D, NV = ProbInfo<PR>::NV;
  constexpr int TT = LeafTT<T, PR>::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T4* sp = reinterpret_cast<T4*>(smem_raw);          // [2][cap] source / equivalent positions
  T4* sv = sp + 2 * a.cap;                            // [2][cap * NV] their values
  T* red = reinterpret_cast<T*>(sv + 2 * a.cap * NV); // [LEAF_THREADS][TT][KT]
  __shared__ uint64_t bar[2], stall_bar;
  __shared__ int ent_n[2], ent_cnt[2][LEAF_MAX_ENT], ent_sc[2][LEAF_MAX_ENT], have[2];
  __shared__ int next_e, next_s, bail;

  const int b = a.leaves[blockIdx.x];
  T cx, cy, cz, r;
  box_centre<T>(a.t, b, a.geo.L, a.geo.org, cx, cy, cz, r);
  const int t0 = a.t.tb[b], t1 = a.t.te[b];
  const int nt = t1 - t0;
  if (nt <= 0) return;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    if (a.stall_test) mbar_init(&stall_bar, 1);
    bail = 0;
  }
  __syncthreads();
  if (a.stall_test) {
    // test aid: a wait that nothing completes runs out after the wait limit; the block then
    // takes the wind-down path (no copy has been issued yet) and leaves without output
    if (tid == 0 && !mbar_wait_bounded(&stall_bar, 0, a.status, a.lim)) bail = 1;
    __syncthreads();
    if (bail) return;
  }
  const int tt = (TT == 4 && nt > 32) ? 4 : ((TT >= 2 && nt > 16) ? 2 : 1);
  const int per_pass = min(nt, LEAF_THREADS * tt);
  const int S = (per_pass + tt - 1) / tt;            // slots
  const int G = max(1, LEAF_THREADS / S);            // threads per slot
  const int slot = tid / G, grp = tid % G;
  const bool in_slot = slot < S;
  const bool shfl = G <= 32 && (32 % G) == 0;
  const int64_t u0 = a.u_off[b], u1 = a.u_off[b + 1];
  uint32_t ph[2] = {0u, 0u};

  for (int p0 = t0; p0 < t1; p0 += per_pass) {
    const int p1 = min(t1, p0 + per_pass);
    int it[TT];
    bool act[TT];
    T xl[TT], yl[TT], zl[TT], xg[TT], yg[TT], zg[TT], bi[TT];
    T acc[TT][KT], comp[TT][KT];
#pragma unroll
    for (int u = 0; u < TT; ++u) {
      it[u] = p0 + slot + u * S;
      act[u] = in_slot && u < tt && it[u] < p1;
      xl[u] = yl[u] = zl[u] = xg[u] = yg[u] = zg[u] = bi[u] = 0;
      if (act[u]) {
        T4 x = a.tpos[it[u]];
        xg[u] = x.x;
        yg[u] = x.y;
        zg[u] = x.z;
        xl[u] = x.x - cx;
        yl[u] = x.y - cy;
        zl[u] = x.z - cz;
        // the target's own radius (RPY with one shared point set)
        if ((PR == P_RPY_L4 || PR == P_RPY_G) && a.contact) bi[u] = a.sval[(int64_t)it[u] * NV].w;
      }
#pragma unroll
      for (int k = 0; k < KT; ++k) acc[u][k] = comp[u][k] = 0;
    }

    if (!a.near_only) {
      // ---- L->T and M->T: equivalent points staged (local coordinates, reference c_B)
      const int nw = (int)(a.w_off[b + 1] - a.w_off[b]);
      for (int e = -1; e < nw; ++e) {
        int sbx = b, sc = 13;
        T alpha = T(ALPHA_DE);
        const T* dens = a.dn_equiv;
        if (e >= 0) {
          int32_t ent = a.w_ent[a.w_off[b] + e];
          sbx = entry_box(ent);
          sc = entry_shift(ent);
          alpha = T(ALPHA_UE);
          dens = a.up_equiv;
        }
        int sx, sy, sz;
        shift_decode(sc, sx, sy, sz);
        T ax, ay, az, ar;
        box_centre<T>(a.t, sbx, a.geo.L, a.geo.org, ax, ay, az, ar);
        T ox = ax + (T)(sx * a.geo.L) - cx, oy = ay + (T)(sy * a.geo.L) - cy, oz = az + (T)(sz * a.geo.L) - cz;
        __syncthreads();
        for (int k = tid; k < a.n; k += blockDim.x) {
          T4 p;
          p.x = ox + alpha * ar * a.unit[3 * k];
          p.y = oy + alpha * ar * a.unit[3 * k + 1];
          p.z = oz + alpha * ar * a.unit[3 * k + 2];
          p.w = 0;
          const T* dp = dens + ((int64_t)sbx * a.R + (int64_t)k * D) * C;
          T4 q;
          if (C == 4) {
            q = *reinterpret_cast<const T4*>(dp);
            q.w = q.w + ox * q.x + oy * q.y + oz * q.z;  // re-reference to c_B
          } else if (D == 3) {
            q.x = dp[0];
            q.y = dp[1];
            q.z = dp[2];
            q.w = 0;
          } else if (D == 4) {   // StokesPVel: [f, q]
            q.x = dp[0];
            q.y = dp[1];
            q.z = dp[2];
            q.w = dp[3];
          } else {
            q.x = dp[0];
            q.y = q.z = q.w = 0;
          }
          sp[k] = p;
          sv[k] = q;
        }
        __syncthreads();
        if (act[0]) {  // partial sums per 32 equivalent points of a group, then per surface
          T fs[TT][KT];
#pragma unroll
          for (int u = 0; u < TT; ++u)
#pragma unroll
            for (int q = 0; q < KT; ++q) fs[u][q] = 0;
          for (int k0 = grp; k0 < a.n; k0 += 32 * G) {
            T fp[TT][KT];
#pragma unroll
            for (int u = 0; u < TT; ++u)
#pragma unroll
              for (int q = 0; q < KT; ++q) fp[u][q] = 0;
            const int kend = min(a.n, k0 + 32 * G);
            for (int k = k0; k < kend; k += G) {
              const T4 pk = sp[k], qk = sv[k];
#pragma unroll
              for (int u = 0; u < TT; ++u)
                if (u < tt) far_eval<T, PR>(xl[u], yl[u], zl[u], pk, qk, fp[u]);
            }
#pragma unroll
            for (int u = 0; u < TT; ++u)
#pragma unroll
              for (int q = 0; q < KT; ++q) fs[u][q] += fp[u][q];
          }
#pragma unroll
          for (int u = 0; u < TT; ++u)
#pragma unroll
            for (int q = 0; q < KT; ++q) acc[u][q] += fs[u][q];
        }
      }
    }

    // ---- S->T over the U list: batches of whole (or split) entries, two staging buffers
    // (thread 0 composes a batch: bulk copies of its sources and values completing on the
    // buffer's mbarrier)
    auto compose = [&](int bf) -> int {
      T4* dp = sp + bf * a.cap;
      T4* dv = sv + bf * a.cap * NV;
      int used = 0, ne = 0;
      uint32_t bytes = 0;
      while (next_e < u1 && ne < LEAF_MAX_ENT && used < a.cap) {
        int32_t ent = a.u_ent[next_e];
        int sbx = entry_box(ent);
        int s0 = a.t.sb[sbx] + next_s, s1 = a.t.se[sbx];
        int take = min(s1 - s0, a.cap - used);
        if (take > 0) {
          bulk_g2s(dp + used, a.spos + s0, (uint32_t)(take * sizeof(T4)), &bar[bf]);
          bulk_g2s(dv + used * NV, a.sval + (int64_t)s0 * NV, (uint32_t)(take * NV * sizeof(T4)), &bar[bf]);
          bytes += (uint32_t)(take * (1 + NV) * sizeof(T4));
          ent_cnt[bf][ne] = take;
          // the shift code (0..26), plus 32 for the target leaf's own unshifted sources (the
          // only entry that can hold a target's own point, r = 0)
          ent_sc[bf][ne] = entry_shift(ent) + ((sbx == b && entry_shift(ent) == 13) ? 32 : 0);
          ++ne;
          used += take;
        }
        if (s0 + take >= s1) {
          ++next_e;
          next_s = 0;
        } else {
          next_s += take;
        }
      }
      ent_n[bf] = ne;
      return ne > 0 ? (int)bytes : 0;
    };
    __syncthreads();   // the far field has finished reading buffer 0 (its equivalent points)
    if (tid == 0) {
      next_e = (int)u0;
      next_s = 0;
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      for (int bf = 0; bf < 2; ++bf) {
        const int bytes = compose(bf);
        have[bf] = bytes > 0;
        if (bytes) mbar_expect_tx(&bar[bf], (uint32_t)bytes);
      }
    }
    __syncthreads();
    for (int itb = 0;; ++itb) {
      const int bf = itb & 1;
      if (!have[bf]) break;
      // wait for this batch (bounded).  On expiry the block issues no further copy, skips the
      // compute and the output, waits once more (bounded) for the copies still in flight, and
      // leaves; the status word carries ST_TIMEOUT to the host.
      if (!mbar_wait_bounded(&bar[bf], ph[bf], a.status, a.lim)) bail = 1;
      __syncthreads();
      if (bail) {
        if (tid == 0) {
          mbar_wait_bounded(&bar[bf], ph[bf], a.status, a.lim);
          if (have[bf ^ 1]) mbar_wait_bounded(&bar[bf ^ 1], ph[bf ^ 1], a.status, a.lim);
        }
        __syncthreads();
        return;
      }
      ph[bf] ^= 1u;
      const T4* bp = sp + bf * a.cap;
      const T4* bv = sv + bf * a.cap * NV;
      if (act[0]) {
        int base = 0;
        for (int e = 0; e < ent_n[bf]; ++e) {
          int sx, sy, sz;
          const bool self_ent = ent_sc[bf][e] >= 32;
          shift_decode(ent_sc[bf][e] & 31, sx, sy, sz);
          const T ox = (T)(sx * a.geo.L) - cx, oy = (T)(sy * a.geo.L) - cy, oz = (T)(sz * a.geo.L) - cz;
          const int cnt = ent_cnt[bf][e];
          T pe[TT][KT];  // partial sums of this entry (plain mode)
#pragma unroll
          for (int u = 0; u < TT; ++u)
#pragma unroll
            for (int k = 0; k < KT; ++k) pe[u][k] = 0;
          bool done_fast = false;
          if constexpr ((PR == P_STK_L4 || PR == P_STK_G) && sizeof(T) == 4) {
            if (!a.kahan) {
              // Stokeslet in FP32: the image shift folded into the targets' global
              // coordinates once per entry (exact for the unshifted entries, so the self pair
              // stays at r = 0), every staged source feeding the thread's targets by FMAs
              float xe[TT], ye[TT], ze[TT];
#pragma unroll
              for (int u = 0; u < TT; ++u) {
                xe[u] = xg[u] - (float)(sx * a.geo.L);
                ye[u] = yg[u] - (float)(sy * a.geo.L);
                ze[u] = zg[u] - (float)(sz * a.geo.L);
              }
              if (TT == 4 && tt == 4) {
                if (self_ent) {
                  for (int j = grp; j < cnt; j += G) {
                    const float4 y = bp[base + j], f = bv[base + j];
#pragma unroll
                    for (int u = 0; u < TT; ++u) stk_pair_f32<true>(xe[u], ye[u], ze[u], y, f, pe[u]);
                  }
                } else {
                  for (int j = grp; j < cnt; j += G) {
                    const float4 y = bp[base + j], f = bv[base + j];
#pragma unroll
                    for (int u = 0; u < TT; ++u) stk_pair_f32<false>(xe[u], ye[u], ze[u], y, f, pe[u]);
                  }
                }
              } else if (TT >= 2 && tt == 2) {
                constexpr int U1 = TT >= 2 ? 1 : 0;
                for (int j = grp; j < cnt; j += G) {
                  const float4 y = bp[base + j], f = bv[base + j];
                  stk_pair_f32(xe[0], ye[0], ze[0], y, f, pe[0]);
                  stk_pair_f32(xe[U1], ye[U1], ze[U1], y, f, pe[U1]);
                }
              } else {
                int j = grp;
                for (; j + G < cnt; j += 2 * G) {
                  stk_pair_f32(xe[0], ye[0], ze[0], bp[base + j], bv[base + j], pe[0]);
                  stk_pair_f32(xe[0], ye[0], ze[0], bp[base + j + G], bv[base + j + G], pe[0]);
                }
                if (j < cnt) stk_pair_f32(xe[0], ye[0], ze[0], bp[base + j], bv[base + j], pe[0]);
              }
              done_fast = true;
            }
          }
          if (!done_fast) {
            for (int j = grp; j < cnt; j += G) {
              const T4 y = bp[base + j];
              const T4 v = bv[(base + j) * NV];
#pragma unroll
              for (int u = 0; u < TT; ++u) {
                if (u >= tt) continue;
                T r0 = xl[u] - (y.x + ox), r1 = yl[u] - (y.y + oy), r2 = zl[u] - (y.z + oz);
                T tmp[KT];
#pragma unroll
                for (int k = 0; k < KT; ++k) tmp[k] = 0;
                if (PR == P_LAP) {
                  lap_st<T>(r0, r1, r2, v.x, tmp);
                } else if (PR == P_LAPQD) {
                  lapqd_st<T, true>(r0, r1, r2, v.x, v.y, v.z, v.w, tmp);
                } else if (PR == P_PVEL) {
                  pvel_st<T>(r0, r1, r2, v.x, v.y, v.z, v.w, tmp);
                } else if (PR == P_PVEL_D) {
                  pvel_grad_st<T>(r0, r1, r2, v.x, v.y, v.z, v.w, tmp);
                } else if (PR == P_STK_L4 || PR == P_STK_G) {
                  stk_st<T>(r0, r1, r2, v.x, v.y, v.z, tmp);
                } else if (PR == P_REG_G) {   // S->T: the regularized kernel of the source's eps
                  reg_st<T>(r0, r1, r2, v.x, v.y, v.z, v.w, tmp);
                } else if (PR == P_RPY_L4 || PR == P_RPY_G) {
                  // contact pairs are left to the sphere-velocity pass, which adds their whole
                  // mobility (their far form is large and cancels there, beyond FP32 precision)
                  if (a.contact && in_contact<T>(xg[u], yg[u], zg[u], y.x, y.y, y.z, (T)(sx * a.geo.L),
                                                  (T)(sy * a.geo.L), (T)(sz * a.geo.L), bi[u], v.w))
                    continue;
                  rpy_st<T>(r0, r1, r2, v.x, v.y, v.z, v.w, tmp);
                } else {
                  const T4 v1 = bv[(base + j) * NV + 1], v2 = bv[(base + j) * NV + 2];
                  T Dm[9] = {v.x, v.y, v.z, v.w, v1.x, v1.y, v1.z, v1.w, v2.x};
                  if constexpr (PR == P_DL_D)
                    dl_grad_st<T>(r0, r1, r2, Dm, tmp);
                  else if constexpr (PR == P_LAPQ)
                    quad_st<T>(r0, r1, r2, Dm, tmp);
                  else
                    dl_st<T>(r0, r1, r2, Dm, tmp);
                }
                if (a.kahan) {
#pragma unroll
                  for (int k = 0; k < KT; ++k) {
                    T yk = tmp[k] - comp[u][k];
                    T tk = acc[u][k] + yk;
                    comp[u][k] = (tk - acc[u][k]) - yk;
                    acc[u][k] = tk;
                  }
                } else {
#pragma unroll
                  for (int k = 0; k < KT; ++k) pe[u][k] += tmp[k];
                }
              }
            }
          }
          if (!a.kahan) {
#pragma unroll
            for (int u = 0; u < TT; ++u)
#pragma unroll
              for (int k = 0; k < KT; ++k) acc[u][k] += pe[u][k];
          }
          base += cnt;
        }
      }
      __syncthreads();   // every read of buffer bf is done: it takes batch itb + 2
      if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        const int bytes = compose(bf);
        have[bf] = bytes > 0;
        if (bytes) mbar_expect_tx(&bar[bf], (uint32_t)bytes);
      }
    }
    // ---- combine the G partial sums of each target and write
    if (G > 1) {
      if (shfl) {
#pragma unroll
        for (int u = 0; u < TT; ++u)
#pragma unroll
          for (int k = 0; k < KT; ++k)
            for (int o = G >> 1; o > 0; o >>= 1) acc[u][k] += __shfl_xor_sync(0xffffffffu, acc[u][k], o);
      } else {
        __syncthreads();
#pragma unroll
        for (int u = 0; u < TT; ++u)
#pragma unroll
          for (int k = 0; k < KT; ++k) red[((int64_t)tid * TT + u) * KT + k] = acc[u][k];
        __syncthreads();
        if (grp == 0 && in_slot) {
          for (int q = 1; q < G; ++q)
#pragma unroll
            for (int u = 0; u < TT; ++u)
#pragma unroll
              for (int k = 0; k < KT; ++k) acc[u][k] += red[((int64_t)(tid + q) * TT + u) * KT + k];
        }
      }
    }
    if (grp == 0) {
#pragma unroll
      for (int u = 0; u < TT; ++u)
        if (act[u]) {
#pragma unroll
          for (int k = 0; k < KT; ++k) a.g[(int64_t)it[u] * KT + k] = acc[u][k] * out_scale<PR, T>(k);
        }
    }
    __syncthreads();   // the next pass reuses the staging buffers
  }
}

// Periodic Laplace: the zero-mean periodic Green's function has lap G_per = 1/V, so the sum
// depends on the trace of the second charge moment, which equivalent charges do not carry.
// Adds (sum_j q_j |y_j - c|^2 - sum_k M_k |ue_k - c|^2) / (6 V) to every target (c: root centre,
// M: the root's upward equivalent charges).
template <class T>
__global__ void k_laplace_periodic_constant(const typename V4<T>::type* __restrict__ spos,
                                            const typename V4<T>::type* __restrict__ sval, int64_t ns,
                                            const T* __restrict__ up_equiv, const T* __restrict__ unit,
                                            int n, Geo geo, T* __restrict__ g, int64_t nt) {
  __shared__ double red[32];
  __shared__ double cval;
  double c[3] = {geo.org[0] + 0.5 * geo.L, geo.org[1] + 0.5 * geo.L, geo.org[2] + 0.5 * geo.L};
  double acc = 0;
  for (int64_t j = threadIdx.x; j < ns; j += blockDim.x) {
    double d0 = (double)spos[j].x - c[0], d1 = (double)spos[j].y - c[1], d2 = (double)spos[j].z - c[2];
    acc += (double)sval[j].x * (d0 * d0 + d1 * d1 + d2 * d2);
  }
  double r0 = 0.5 * geo.L;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double u2 = 0;
    for (int d = 0; d < 3; ++d) {
      double u = ALPHA_UE * r0 * (double)unit[3 * k + d];
      u2 += u * u;
    }
    acc -= (double)up_equiv[k] * u2;  // root = box 0
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    cval = t / (6.0 * geo.L * geo.L * geo.L);
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < nt; i += blockDim.x) g[i] += (T)cval;
}

// Periodic StokesPVel table ([f, q] and double-layer sources): two source moments are not
// fixed by the far field the root's equivalent density reproduces, and each shifts the zero-mean
// periodic result by a constant (the periodic grad G_per = grad(harmonic) + r / (3 V)):
//   p += (tr M_src - tr M_eq) / (3 V),   tr M = sum f.(y - c) (an isotropic force dipole has no
//                                         free-space field);
//   u += -(d_src - d_eq) / (6 V) + (a_src - a_eq) / (3 V),  d = sum q (y - c) and the
//        potential-dipole content of the force quadrupole a = (2 v - w) / 5, v = sum f |y - c|^2,
//        w = sum (f.(y - c)) (y - c): d + a is fixed by the far field, the two pieces extend
//        periodically with different constants.
// A double-layer source D is a force dipole -sym(D) plus a source q = tr D at its point.
// Partial moments per block, [blocks][10] = tr M, d (3), v (3), w (3), in double.
template <class T, int PR>
__global__ void k_pvel_moments(const typename V4<T>::type* __restrict__ spos,
                               const typename V4<T>::type* __restrict__ sval, int64_t ns, Geo geo,
                               double* __restrict__ part) {
  constexpr int NV = ProbInfo<PR>::NV;
  __shared__ double red[10][32];
  const double c[3] = {geo.org[0] + 0.5 * geo.L, geo.org[1] + 0.5 * geo.L, geo.org[2] + 0.5 * geo.L};
  double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ns; j += (int64_t)gridDim.x * blockDim.x) {
    const double y[3] = {(double)spos[j].x - c[0], (double)spos[j].y - c[1], (double)spos[j].z - c[2]};
    const double yy = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
    if constexpr (dl_src(PR)) {
      const auto v0 = sval[j * NV], v1 = sval[j * NV + 1], v2 = sval[j * NV + 2];
      const double Dm[9] = {(double)v0.x, (double)v0.y, (double)v0.z, (double)v0.w, (double)v1.x,
                            (double)v1.y, (double)v1.z, (double)v1.w, (double)v2.x};
      double S[9], Sy[3];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) S[3 * a + b] = 0.5 * (Dm[3 * a + b] + Dm[3 * b + a]);
      const double tr = S[0] + S[4] + S[8];
      for (int a = 0; a < 3; ++a) Sy[a] = S[3 * a] * y[0] + S[3 * a + 1] * y[1] + S[3 * a + 2] * y[2];
      acc[0] -= tr;
      for (int a = 0; a < 3; ++a) {
        acc[1 + a] += tr * y[a];
        acc[4 + a] -= 2.0 * Sy[a];
        acc[7 + a] -= tr * y[a] + Sy[a];
      }
    } else {
      const auto v = sval[j * NV];
      const double f[3] = {(double)v.x, (double)v.y, (double)v.z}, q = (double)v.w;
      const double fy = f[0] * y[0] + f[1] * y[1] + f[2] * y[2];
      acc[0] += fy;
      for (int a = 0; a < 3; ++a) {
        acc[1 + a] += q * y[a];
        acc[4 + a] += f[a] * yy;
        acc[7 + a] += fy * y[a];
      }
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = 0; k < 10; ++k) {
    double x = acc[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[k][w] = x;
  }
  __syncthreads();
  if (threadIdx.x < 10) {
    double t = 0;
    for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) t += red[threadIdx.x][ww];
    part[blockIdx.x * 10 + threadIdx.x] = t;
  }
}

// One block: the partials in block order, minus the root's equivalent density's moments (real
// [f, q] per upward equivalent point, box 0), into the shifts sh = [dp, du (3)].
template <class T>
__global__ void k_pvel_shift(const double* __restrict__ part, int nblk, const T* __restrict__ up_equiv,
                             const T* __restrict__ unit, int n, Geo geo, double* __restrict__ sh) {
  __shared__ double red[10][32];
  double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  const double r0 = 0.5 * geo.L;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double y[3];
    for (int d = 0; d < 3; ++d) y[d] = ALPHA_UE * r0 * (double)unit[3 * k + d];
    const double yy = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
    const double f[3] = {(double)up_equiv[4 * k], (double)up_equiv[4 * k + 1], (double)up_equiv[4 * k + 2]};
    const double q = (double)up_equiv[4 * k + 3];
    const double fy = f[0] * y[0] + f[1] * y[1] + f[2] * y[2];
    acc[0] -= fy;
    for (int a = 0; a < 3; ++a) {
      acc[1 + a] -= q * y[a];
      acc[4 + a] -= f[a] * yy;
      acc[7 + a] -= fy * y[a];
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = 0; k < 10; ++k) {
    double x = acc[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[k][w] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m[10];
    for (int k = 0; k < 10; ++k) {
      double t = 0;
      for (int b = 0; b < nblk; ++b) t += part[b * 10 + k];
      for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) t += red[k][ww];
      m[k] = t;
    }
    const double V = geo.L * geo.L * geo.L;
    sh[0] = m[0] / (3.0 * V);
    for (int a = 0; a < 3; ++a) sh[1 + a] = -m[1 + a] / (6.0 * V) + (2.0 * m[4 + a] - m[7 + a]) / (15.0 * V);
  }
}

// Adds the shifts to [p, u] (the first four target values) of every sorted target.
template <class T, int KT>
__global__ void k_pvel_shift_apply(const double* __restrict__ sh, T* __restrict__ g, int64_t nt) {
  const T d0 = (T)sh[0], d1 = (T)sh[1], d2 = (T)sh[2], d3 = (T)sh[3];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x) {
    T* o = g + i * KT;
    o[0] += d0;
    o[1] += d1;
    o[2] += d2;
    o[3] += d3;
  }
}

// ---------------------------------------------------------------------------------------
// Host side.
#define CK(call)                                           \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(P, e_, #call); \
  } while (0)

static int grid_for(int64_t n, int threads, int maxb = 152 * 8) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > maxb) b = maxb;
  return (int)b;
}

static void add_tiles(WorkLists& W, std::vector<int>* by_cls, int NB, int range[2]) {
  range[0] = (int)W.tiles.size();
  for (int c = 0; c < 8; ++c) {
    std::vector<int>& v = by_cls[c];
    for (size_t i = 0; i < v.size(); i += NB) {
      int cnt = (int)std::min<size_t>(NB, v.size() - i);
      W.tiles.push_back(make_int4((int)W.boxlist.size(), cnt, c, 0));
      W.boxlist.insert(W.boxlist.end(), v.begin() + i, v.begin() + i + cnt);
    }
    v.clear();
  }
  range[1] = (int)W.tiles.size();
}

// Offsets of the tree's per-box fields in the page-locked download buffer.
struct WlDown {
  size_t key, xoff, vocc, tb, te, lvl, leaf, wflag, stats, meta, bytes;
  explicit WlDown(int nb) {
    key = 0;
    xoff = key + 8 * (size_t)nb;
    vocc = xoff + 8 * (size_t)(nb + 1);
    tb = vocc + 32 * (size_t)nb;
    te = tb + 4 * (size_t)nb;
    lvl = te + 4 * (size_t)nb;
    leaf = lvl + nb;
    wflag = leaf + nb;
    stats = (wflag + nb + 7) / 8 * 8;
    meta = stats + 24;
    bytes = meta + 4 * 217;
  }
};

// Enqueues the copy of the tree's per-box fields into page-locked memory (no wait): the work
// lists are laid out from them by worklists_finish, which the evaluation calls after enqueuing
// S->M, so the host work overlaps the upward pass.
int worklists_download(Plan& P, int NB, int NB_TC) {
  Tree& T = P.tree;
  cudaStream_t st = P.stream;
  const int nb = T.nbox;
  const WlDown o(nb);
  // copies of an earlier download may still be landing in the staging buffer
  if (P.wl_pending && P.wl_dl_event) CK(cudaEventSynchronize(P.wl_dl_event));
  P.wl_pending = false;
  CK(P.wl_down.reserve(o.bytes));
  HostBuf& H = P.wl_down;
  CK(cudaMemcpyAsync(H.as<void>(o.key), T.key.p, 8 * (size_t)nb, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(H.as<void>(o.xoff), T.x_off.p, 8 * (size_t)(nb + 1), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(H.as<void>(o.vocc), T.vocc.p, 32 * (size_t)nb, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(H.as<void>(o.tb), T.tb.p, 4 * (size_t)nb, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(H.as<void>(o.te), T.te.p, 4 * (size_t)nb, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(H.as<void>(o.lvl), T.level.p, nb, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(H.as<void>(o.leaf), T.leaf.p, nb, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(H.as<void>(o.wflag), T.w_flag.p, nb, cudaMemcpyDeviceToHost, st));
  // near-field pairs (status words 8-9), V entries and largest leaf (10-13), the grouped M->L
  // pair histogram (216 counts and their total)
  CK(cudaMemcpyAsync(H.as<void>(o.stats), T.status.as<unsigned>() + 8, 24, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(H.as<void>(o.meta), T.m2l_meta.p, 4 * 217, cudaMemcpyDeviceToHost, st));
  if (!P.wl_dl_event) CK(cudaEventCreateWithFlags(&P.wl_dl_event, cudaEventDisableTiming));
  CK(cudaEventRecord(P.wl_dl_event, st));
  P.wl_nb = NB;
  P.wl_nb_tc = NB_TC;
  P.wl_pending = true;
  return 0;
}

int build_worklists(Plan& P, int NB, int NB_TC) {
  int rc = worklists_download(P, NB, NB_TC);
  return rc ? rc : worklists_finish(P);
}

// Lays out the work lists of the downloaded tree on the host and uploads them (no-op unless a
// download is pending).
int worklists_finish(Plan& P) {
  if (!P.wl_pending) return 0;
  auto t0 = std::chrono::steady_clock::now();
  Tree& T = P.tree;
  cudaStream_t st = P.stream;
  const int nb = T.nbox;
  const int NB = P.wl_nb, NB_TC = P.wl_nb_tc;
  const WlDown wd(nb);
  const size_t o_key = wd.key, o_xoff = wd.xoff, o_vocc = wd.vocc, o_tb = wd.tb, o_te = wd.te, o_lvl = wd.lvl,
               o_leaf = wd.leaf, o_wflag = wd.wflag, o_stats = wd.stats, o_meta = wd.meta;
  CK(cudaEventSynchronize(P.wl_dl_event));
  P.wl_pending = false;
  HostBuf& H = P.wl_down;
  {
  const unsigned long long* hs = H.as<unsigned long long>(o_stats);
    T.near_pairs = (int64_t)hs[0];
    T.n_v = (int64_t)hs[1];
    T.max_leaf_pts = (int)hs[2];
    memcpy(T.m2l_hist, H.as<unsigned>(o_meta), sizeof(unsigned) * 217);
    T.m2l_npairs = (int64_t)T.m2l_hist[216];
  }
  const uint64_t* key = H.as<uint64_t>(o_key);
  const int64_t* xoff = H.as<int64_t>(o_xoff);
  const uint8_t* oc = H.as<uint8_t>(o_vocc);
  const int* tb = H.as<int>(o_tb);
  const int* te = H.as<int>(o_te);
  const int8_t* lvl = H.as<int8_t>(o_lvl);
  const int8_t* leaf = H.as<int8_t>(o_leaf);
  const int8_t* wflag = H.as<int8_t>(o_wflag);
  WorkLists& W = P.wl;
  W = WorkLists();
  std::vector<int> by_cls[8];
  auto cls = [&](int b) {
    uint64_t k = key[b];
    return (int)((k & 1) | ((k >> 1) & 1) << 1 | ((k >> 2) & 1) << 2);
  };
  const bool per = periodic_mask(P.bc) != 0;
  int vmin = per ? 1 : 2;
  // M->L: all boxes at levels >= vmin, by octant class (the class fixes the offset of each V
  // slot).  Tensor-core tiles take NB_TC boxes.
  for (int b = 0; b < nb; ++b)
    if (lvl[b] >= vmin) by_cls[cls(b)].push_back(b);
  // Per parent neighbour g (the 8 children of one colleague of the parent: Sec. II builds V
  // lists from such children): a tile holds boxes of one class with entries from g, sorted by
  // their 8-bit occupancy of g, and each box's result is a partial sum added to its downward
  // check in neighbour order.  Adaptive V lists are sparse and differ from box to box, so
  // tiles carrying whole V lists compute mostly empty columns; this is the default whenever
  // the partials (R x C floats per box and neighbour) fit in a quarter of the device memory.
  bool grouped = false;
  if (P.use_tc && P.tc_tiling != 1) {
    // the pairs were counted with the tree (Tree::m2l_hist); they are sorted on the device and
    // the tiles laid out here: runs of one (neighbour, class) in key order, NB_TC pairs a tile
    const int64_t npart = T.m2l_npairs;
    const double part_bytes = (double)npart * P.R * P.C * 4;
    grouped = part_bytes < (double)P.dev_mem / 4 && npart < INT32_MAX;
    if (grouped) {
      int rc = m2l_pairs_sort(P);
      if (rc) return rc;
      W.m2l[0] = (int)W.tiles.size();
      int run = 0;
      for (int gc = 0; gc < 216; ++gc) {   // key order: neighbour g = gc / 8, class gc % 8
        const int cnt = (int)T.m2l_hist[gc];
        for (int i = 0; i < cnt; i += NB_TC)
          W.tiles.push_back(make_int4(run + i, std::min(NB_TC, cnt - i), gc % 8, gc / 8 + 1));
        run += cnt;
      }
      W.m2l[1] = (int)W.tiles.size();
      W.m2l_nparts = npart;
      for (int c = 0; c < 8; ++c) by_cls[c].clear();
    }
  }
  W.m2l_grouped = grouped;
  if (!grouped) {
    // whole V lists: boxes with the same occupancy kept together (sorted by a hash of it,
    // ties in box order), so a tile's offset union stays close to each box's own V list
    std::vector<std::pair<uint64_t, int>> kv;
    for (int c = 0; c < 8; ++c) {
      kv.clear();
      for (int b : by_cls[c]) {
        unsigned long long h = 1469598103934665603ull;   // FNV-1a over the occupancy words
        const uint64_t* o = reinterpret_cast<const uint64_t*>(oc + (size_t)b * 32);
        for (int w = 0; w < 4; ++w) h = (h ^ o[w]) * 1099511628211ull;
        kv.emplace_back(h, b);
      }
      std::sort(kv.begin(), kv.end());
      for (size_t i = 0; i < kv.size(); ++i) by_cls[c][i] = kv[i].second;
    }
    add_tiles(W, by_cls, NB_TC, W.m2l);
  }
  // M->M per level: non-leaf boxes (class irrelevant: use class 0 bucket).  Multipoles are
  // read by M->L (levels >= vmin), by M->T over W lists (W entries lie at level >= 2) and, when
  // periodic, at the root; with the open boundary levels 0 and 1 are never read, so their M->M
  // is skipped.
  for (int l = 0; l < MAX_LEVELS; ++l) {
    bool needed = l >= vmin || (per && l == 0);
    if (needed)
      for (int b = T.lvl_start[l]; b < T.lvl_start[l + 1]; ++b)
        if (!leaf[b]) by_cls[0].push_back(b);
    add_tiles(W, by_cls, NB, W.m2m[l]);
  }
  // L->L per level (levels >= vmin + 1; and level 1 from the root when periodic)
  for (int l = 0; l < MAX_LEVELS; ++l) {
    if (l >= 1 && (l >= vmin + 1 || per))
      for (int b = T.lvl_start[l]; b < T.lvl_start[l + 1]; ++b) by_cls[cls(b)].push_back(b);
    add_tiles(W, by_cls, NB, W.l2l[l]);
  }
  // pseudo-inverses: up for boxes in W lists (and the root for the periodic Laplace
  // constant), down for leaves with targets
  // (the triply periodic Laplace constant and StokesPVel shifts read the root's density)
  const bool pxyz = P.bc == KAFMM_BC_PXYZ;
  for (int b = 0; b < nb; ++b)
    if (wflag[b] || (b == 0 && pxyz && (P.kernel == KAFMM_LAPLACE || P.ml_stokes == 2))) by_cls[0].push_back(b);
  add_tiles(W, by_cls, NB, W.pup);
  if (per) by_cls[0].push_back(0);
  add_tiles(W, by_cls, NB, W.root);
  for (int b = 0; b < nb; ++b)
    if (leaf[b] && te[b] > tb[b]) by_cls[0].push_back(b);
  add_tiles(W, by_cls, NB, W.pdn);
  if (P.cmp && P.use_tc) {   // compressed coordinates: S->M results of the leaves, X-list sums
    for (int b = 0; b < nb; ++b)
      if (leaf[b]) by_cls[0].push_back(b);
    add_tiles(W, by_cls, NB, W.cup);
    for (int b = 0; b < nb; ++b)
      if (xoff[b + 1] > xoff[b]) by_cls[0].push_back(b);
    add_tiles(W, by_cls, NB, W.cx);
  }
  // plain lists: leaves (with targets), boxes with X entries, leaves (S->M, last)
  W.leafbox_off = (int)W.boxlist.size();
  for (int b = 0; b < nb; ++b)
    if (leaf[b] && te[b] > tb[b]) W.boxlist.push_back(b);
  W.leaves_n = (int)W.boxlist.size() - W.leafbox_off;
  W.xbox_off = (int)W.boxlist.size();
  for (int b = 0; b < nb; ++b)
    if (xoff[b + 1] > xoff[b]) W.boxlist.push_back(b);
  W.xbox_n = (int)W.boxlist.size() - W.xbox_off;
  for (int b = 0; b < nb; ++b)
    if (leaf[b]) W.boxlist.push_back(b);
  // upload through page-locked staging: tiles and box lists; the previous upload read the
  // staging buffer, so wait for it before refilling
  const size_t u_tiles = 0, u_box = u_tiles + sizeof(int4) * W.tiles.size(),
               up_bytes = u_box + sizeof(int) * W.boxlist.size();
  if (P.wl_event) CK(cudaEventSynchronize(P.wl_event));
  CK(P.wl_up.reserve(up_bytes));
  HostBuf& U = P.wl_up;
  std::copy(W.tiles.begin(), W.tiles.end(), U.as<int4>(u_tiles));
  std::copy(W.boxlist.begin(), W.boxlist.end(), U.as<int>(u_box));
  CK(P.tiles.reserve(sizeof(int4) * (W.tiles.size() + 1)));
  CK(P.tile_meta.reserve(sizeof(int) * (W.boxlist.size() + 1)));
  CK(cudaMemcpyAsync(P.tiles.p, U.as<void>(u_tiles), sizeof(int4) * W.tiles.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(P.tile_meta.p, U.as<void>(u_box), sizeof(int) * W.boxlist.size(),
                     cudaMemcpyHostToDevice, st));
  // the staging buffers are reused by the next build, which waits for this event first
  if (!P.wl_event) CK(cudaEventCreateWithFlags(&P.wl_event, cudaEventDisableTiming));
  CK(cudaEventRecord(P.wl_event, st));
  P.host_wl_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return 0;
}

// The ML tree in compressed coordinates (mixed form, tensor cores): the upward and downward
// state of a box is its check potential projected on the leading left singular vectors of the
// check-to-equivalent matrix, which carries all the pseudo-inverse uses of it (Sec. II: the
// equivalent density is pinv x check, and every translation starts from an equivalent
// density).  S->M check potentials of the leaves (already in up_check) are compressed; M->M,
// the periodic root operator, M->L and L->L act between compressed coordinates; X-list S->L
// check potentials are compressed and added; the equivalent densities of the W-list boxes and
// of the leaves come from V S^+ applied to the coordinates (scaled by the half-width).
template <int PR>
static int run_compressed(Plan& P, S2CArgs<float, PR>& sa, WorkLists& W, const int* boxlist, int n_sleaves,
                          const int* sleaves) {
  cudaStream_t st = P.stream;
  const int nb = P.tree.nbox;
  const size_t hat_bytes = sizeof(float) * (size_t)P.rp * P.C * nb;
  CK(P.up_hat.reserve(hat_bytes));
  CK(P.dn_hat.reserve(hat_bytes));
  CK(cudaMemsetAsync(P.dn_hat.p, 0, hat_bytes, st));
  float* up_check = P.up_check.as<float>();
  float* dn_check = P.dn_check.as<float>();
  float* up_hat = P.up_hat.as<float>();
  float* dn_hat = P.dn_hat.as<float>();
  auto tcg = [&](int mode, int opset, const int* range, const float* in, float* out, int op, int write) -> int {
    const int n = range[1] - range[0];
    if (n <= 0) return 0;
    const int* bl = mode == TCM_M2L && W.m2l_grouped ? P.m2l_box.as<int>() : boxlist;
    return tc_gemm_launch(P, mode, opset, P.tiles.as<int4>() + range[0], n, bl, in, out, op, write, st);
  };
  (void)n_sleaves;
  (void)sleaves;
  int rc = tcg(TCM_APPLY, TCO_CIN, W.cup, up_check, up_hat, 0, TCW_STORE);
  for (int l = MAX_LEVELS - 1; l >= 0 && !rc; --l)
    rc = tcg(TCM_M2M, TCO_CMP, W.m2m[l], up_hat, up_hat, 0, TCW_STORE);
  if (!rc) rc = tcg(TCM_APPLY, TCO_CMP, W.root, up_hat, dn_hat, CAUX_PER, TCW_ADD);
  if (rc) return rc;
  cudaEventRecord(P.ev[4], st);
  rc = tcg(TCM_M2L, TCO_CMP, W.m2l, up_hat, dn_hat, 0, TCW_ADD);
  if (rc) return rc;
  cudaEventRecord(P.ev[5], st);
  if (W.xbox_n > 0) {   // S->L over the X lists on the check surface, then compressed and added
    CK(cudaMemsetAsync(dn_check, 0, sizeof(float) * (size_t)P.R * P.C * nb, st));
    sa.boxes = boxlist + W.xbox_off;
    sa.check = dn_check;
    sa.mode = 1;
    KL k_s2check<float, PR><<<W.xbox_n, 128, 0, st>>>(sa);
    rc = tcg(TCM_APPLY, TCO_CIN, W.cx, dn_check, dn_hat, 1, TCW_ADD);
  }
  for (int l = 0; l < MAX_LEVELS && !rc; ++l)
    rc = tcg(TCM_L2L, TCO_CMP, W.l2l[l], dn_hat, dn_hat, 0, TCW_ADD);
  if (!rc) rc = tcg(TCM_APPLY, TCO_COUT, W.pup, up_hat, P.up_equiv.as<float>(), 0, TCW_SCALE);
  if (!rc) rc = tcg(TCM_APPLY, TCO_COUT, W.pdn, dn_hat, P.dn_equiv.as<float>(), 1, TCW_SCALE);
  CK(cudaGetLastError());
  return rc;
}

template <class T, int PR>
static int run_eval(Plan& P, const void* s_in, int s_dtype, void* g_out) {
  using T4 = typename V4<T>::type;
  constexpr int KT = ProbInfo<PR>::KT, C = ProbInfo<PR>::C, D = ProbInfo<PR>::D, NV = ProbInfo<PR>::NV;
  Tree& T_ = P.tree;
  cudaStream_t st = P.stream;
  WorkLists& W = P.wl;
  int nb = T_.nbox;
  int R = P.R;
  int64_t ns = T_.n_src, nt = T_.n_trg;
  Geo geo;
  geo.L = P.L;
  for (int d = 0; d < 3; ++d) geo.org[d] = P.origin[d];
  TreeView tv = T_.view();
  tv.periodic = periodic_mask(P.bc);
  const T* unit = P.fp64() ? (const T*)P.unit64.p : (const T*)P.unit32.p;
  const T* ops = P.fp64() ? (const T*)P.ops64.p : (const T*)P.ops32.p;

  cudaEventRecord(P.ev[3], st);
  // source values -> sorted records
  CK(P.s_sorted.reserve(sizeof(T4) * NV * (ns + 1)));
  if (ns > 0) {
    if (s_dtype == KAFMM_F64)
      KL k_prep_src<double, T, PR><<<grid_for(ns, 256), 256, 0, st>>>(
          (const double*)s_in, T_.src_perm.as<uint32_t>(), ns, P.s_sorted.as<T4>());
    else
      KL k_prep_src<float, T, PR><<<grid_for(ns, 256), 256, 0, st>>>(
          (const float*)s_in, T_.src_perm.as<uint32_t>(), ns, P.s_sorted.as<T4>());
  }
  const T4* spos = T_.src_pos.as<T4>();
  const T4* tpos = T_.same ? spos : T_.trg_pos.as<T4>();
  size_t box_bytes = sizeof(T) * (size_t)R * C;
  // S->M runs over the tree's leaf list (box order); the work lists are laid out on the host
  // while it runs
  const int n_sleaves = T_.nleaf;
  const int* sleaves = T_.leaves.as<int>();
  int* boxlist = nullptr;
  if (P.near_only) {
    int rc = worklists_finish(P);
    if (rc) return rc;
    boxlist = P.tile_meta.as<int>();
  }
  if (!P.near_only) {
    CK(P.up_check.reserve(box_bytes * nb));
    CK(P.dn_check.reserve(box_bytes * nb));
    CK(P.up_equiv.reserve(box_bytes * nb));
    CK(P.dn_equiv.reserve(box_bytes * nb));
    CK(cudaMemsetAsync(P.dn_check.p, 0, box_bytes * nb, st));
    // S->M at the leaves
    S2CArgs<T, PR> sa;
    sa.t = tv;
    sa.geo = geo;
    sa.pos = spos;
    sa.val = P.s_sorted.as<T4>();
    sa.unit = unit;
    sa.x_off = T_.x_off.as<int64_t>();
    sa.x_ent = T_.x_ent.as<int32_t>();
    sa.n = P.n;
    sa.R = R;
    if (n_sleaves > 0) {
      sa.boxes = sleaves;
      sa.check = P.up_check.as<T>();
      sa.mode = 0;
      KL k_s2check<T, PR><<<n_sleaves, 128, 0, st>>>(sa);
    }
    int rcw = worklists_finish(P);
    if (rcw) return rcw;
    boxlist = P.tile_meta.as<int>();
    // The gather-GEMMs run on the tensor cores in the mixed form (four-channel and
    // single-column tables), else on the CUDA cores (k_gemm).
    constexpr bool TC_OK = sizeof(T) == 4 && (C == 4 || C == 1);
    const bool tc = TC_OK && P.use_tc;
    GemmArgs<T> ga;
    ga.qscale4 = 0;
    ga.t = tv;
    ga.geo = geo;
    ga.ops = ops;
    ga.tiles = P.tiles.as<int4>();
    ga.boxlist = boxlist;
    ga.vtab = T_.vtab.as<int32_t>();
    ga.R = R;
    dim3 blk(256);
    int rb = (R + GEMM_BM - 1) / GEMM_BM;
    // mode: TCM_*; op: operator slot (TCM_APPLY); write: TCW_*
    auto gemm = [&](int mode, const int* range, T* in, T* out, int op, int write) -> int {
      int n = range[1] - range[0];
      if (n <= 0) return 0;
      const int4* tiles = P.tiles.as<int4>() + range[0];
      // grouped M->L tiles index the sorted pair arrays
      const int* bl = mode == TCM_M2L && P.wl.m2l_grouped ? P.m2l_box.as<int>() : boxlist;
      if (tc)
        return tc_gemm_launch(P, mode, TCO_DENSE, tiles, n, bl, reinterpret_cast<const float*>(in),
                              reinterpret_cast<float*>(out), op - OP_M2M, write, st);
      ga.mode = mode == TCM_M2L ? GM_M2L : (mode == TCM_M2M ? GM_M2M : (mode == TCM_L2L ? GM_L2L : GM_APPLY));
      ga.in = in;
      ga.out = out;
      ga.op = op;
      ga.scale_r = write == TCW_SCALE;
      ga.qscale4 = write == TCW_SCALE && D == 4;
      ga.tiles = tiles;
      if (mode == TCM_M2L)
        KL k_gemm<T, C, true><<<dim3(n, rb), blk, 0, st>>>(ga);
      else
        KL k_gemm<T, C, false><<<dim3(n, rb), blk, 0, st>>>(ga);
      return 0;
    };
    int rc = 0;
    bool compressed = false;
    if constexpr (TC_OK) {
      if (tc && P.cmp) {
        rc = run_compressed<PR>(P, sa, W, boxlist, n_sleaves, sleaves);
        if (rc) return rc;
        compressed = true;
      }
    }
    if (!compressed) {
      // M->M, deepest level first
      for (int l = MAX_LEVELS - 1; l >= 0 && !rc; --l)
        rc = gemm(TCM_M2M, W.m2m[l], P.up_check.as<T>(), P.up_check.as<T>(), 0, TCW_STORE);
      if (rc) return rc;
      // periodic: far images of the root's multipole density -> root's downward check
      if (W.root[1] > W.root[0]) {
        ga.mode = GM_APPLY;
        ga.in = P.up_check.as<T>();
        ga.out = P.dn_check.as<T>();
        ga.op = OP_PER;
        ga.scale_r = 0;
        ga.qscale4 = 0;
        ga.tiles = P.tiles.as<int4>() + W.root[0];
        KL k_gemm<T, C, false><<<dim3(1, rb), blk, 0, st>>>(ga);
      }
      cudaEventRecord(P.ev[4], st);
      // M->L over the V lists (all levels)
      rc = gemm(TCM_M2L, W.m2l, P.up_check.as<T>(), P.dn_check.as<T>(), 0, TCW_ADD);
      if (rc) return rc;
      cudaEventRecord(P.ev[5], st);
      // S->L over the X lists
      if (W.xbox_n > 0) {
        sa.boxes = boxlist + W.xbox_off;
        sa.check = P.dn_check.as<T>();
        sa.mode = 1;
        KL k_s2check<T, PR><<<W.xbox_n, 128, 0, st>>>(sa);
      }
      // L->L, coarsest level first
      for (int l = 0; l < MAX_LEVELS && !rc; ++l)
        rc = gemm(TCM_L2L, W.l2l[l], P.dn_check.as<T>(), P.dn_check.as<T>(), 0, TCW_ADD);
      if (rc) return rc;
      // equivalent densities where they are evaluated at targets: r * V * ((S^+ U^T) * check),
      // the two factors applied in turn (tmp = the downward equivalent buffer of the up pass
      // is not yet used, so the up pass stages through dn_equiv and vice versa through up_equiv)
      rc = gemm(TCM_APPLY, W.pup, P.up_check.as<T>(), P.dn_equiv.as<T>(), OP_UP1, TCW_STORE);
      if (!rc) rc = gemm(TCM_APPLY, W.pup, P.dn_equiv.as<T>(), P.up_equiv.as<T>(), OP_UP2, TCW_SCALE);
      // up_check is no longer needed here
      if (!rc) rc = gemm(TCM_APPLY, W.pdn, P.dn_check.as<T>(), P.up_check.as<T>(), OP_DN1, TCW_STORE);
      if (!rc) rc = gemm(TCM_APPLY, W.pdn, P.up_check.as<T>(), P.dn_equiv.as<T>(), OP_DN2, TCW_SCALE);
      if (rc) return rc;
    }
  }
  cudaEventRecord(P.ev[6], st);
  // leaves
  CK(P.g_sorted.reserve(sizeof(T) * KT * (nt + 1)));
  if (W.leaves_n > 0) {
    LeafArgs<T, PR> la;
    la.t = tv;
    la.geo = geo;
    la.spos = spos;
    la.sval = P.s_sorted.as<T4>();
    la.tpos = tpos;
    la.unit = unit;
    la.dn_equiv = P.dn_equiv.as<T>();
    la.up_equiv = P.up_equiv.as<T>();
    la.leaves = boxlist + W.leafbox_off;
    la.u_off = T_.u_off.as<int64_t>();
    la.u_ent = T_.u_ent.as<int32_t>();
    la.w_off = T_.w_off.as<int64_t>();
    la.w_ent = T_.w_ent.as<int32_t>();
    la.g = P.g_sorted.as<T>();
    la.status = T_.status.as<unsigned>();
    la.lim = P.wait;
    la.stall_test = P.stall_test;
    la.n = P.n;
    la.R = R;
    la.near_only = P.near_only;
    la.kahan = P.kahan;
    la.contact = P.contact_split() ? 1 : 0;
    // sources per staging buffer (two buffers): 20 KB each by default (640 FP32 Stokeslet
    // sources), KAFMM_OPT_LEAF_STAGE otherwise; at least the equivalent points of a surface
    int cap = P.leaf_stage > 0 ? P.leaf_stage : (int)(20480 / ((1 + NV) * sizeof(T4)));
    if (cap < P.n) cap = P.n;
    la.cap = cap;
    size_t smem = 2 * (size_t)cap * (1 + NV) * sizeof(T4) + sizeof(T) * LEAF_THREADS * LeafTT<T, PR>::V * KT;
    CK(cudaFuncSetAttribute(k_leaf<T, PR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    KL k_leaf<T, PR><<<W.leaves_n, LEAF_THREADS, smem, st>>>(la);
  }
  CK(cudaGetLastError());
  if (PR == P_LAP && P.bc == KAFMM_BC_PXYZ && !P.near_only && nt > 0) {
    KL k_laplace_periodic_constant<T><<<1, 1024, 0, st>>>(spos, P.s_sorted.as<T4>(), ns, P.up_equiv.as<T>(), unit,
                                                       P.n, geo, P.g_sorted.as<T>(), nt);
  }
  if constexpr (pvel_table(PR)) {
    if (P.bc == KAFMM_BC_PXYZ && !P.near_only && nt > 0) {
      const int nblk = grid_for(ns, 256, 152 * 4);
      CK(P.pvel_shift.reserve(sizeof(double) * (10 * (size_t)nblk + 8)));
      double* part = P.pvel_shift.as<double>();
      double* sh = part + 10 * nblk;
      KL k_pvel_moments<T, PR><<<nblk, 256, 0, st>>>(spos, P.s_sorted.as<T4>(), ns, geo, part);
      KL k_pvel_shift<T><<<1, 256, 0, st>>>(part, ns > 0 ? nblk : 0, P.up_equiv.as<T>(), unit, P.n, geo, sh);
      KL k_pvel_shift_apply<T, KT><<<grid_for(nt, 256), 256, 0, st>>>(sh, P.g_sorted.as<T>(), nt);
    }
  }
  // back to the caller's order and dtype
  if (nt > 0) {
    const uint32_t* tperm = T_.same ? T_.src_perm.as<uint32_t>() : T_.trg_perm.as<uint32_t>();
    if constexpr (deriv_out(PR)) {
      const int kto = P.kt;
      if (s_dtype == KAFMM_F64)
        KL k_unperm_deriv<T, double><<<grid_for(nt * kto, 256), 256, 0, st>>>(P.g_sorted.as<T>(), tperm, nt,
                                                                           P.deriv_mode, (double*)g_out);
      else
        KL k_unperm_deriv<T, float><<<grid_for(nt * kto, 256), 256, 0, st>>>(P.g_sorted.as<T>(), tperm, nt,
                                                                          P.deriv_mode, (float*)g_out);
    } else if (s_dtype == KAFMM_F64)
      KL k_unperm<T, double><<<grid_for(nt * KT, 256), 256, 0, st>>>(P.g_sorted.as<T>(), tperm, nt, KT,
                                                                (double*)g_out);
    else
      KL k_unperm<T, float><<<grid_for(nt * KT, 256), 256, 0, st>>>(P.g_sorted.as<T>(), tperm, nt, KT,
                                                               (float*)g_out);
  }
  cudaEventRecord(P.ev[7], st);
  CK(cudaGetLastError());
  return 0;
}

int evaluate(Plan& P, const void* s, void* g, int dtype) {
  int pr;
  if (P.kernel == KAFMM_LAPLACE)
    pr = P_LAP;
  else if (P.kernel == KAFMM_STOKESLET)
    pr = P.C == 4 ? P_STK_L4 : P_STK_G;
  else if (P.kernel == KAFMM_RPY)
    pr = P.C == 4 ? P_RPY_L4 : P_RPY_G;
  else if (P.kernel == KAFMM_STOKES_REG)
    pr = P_REG_G;
  else if (P.kernel == KAFMM_LAPLACE_QD)
    pr = P_LAPQD;
  else if (P.kernel == KAFMM_STOKES_PVEL)
    pr = P_PVEL;
  else if (P.kernel == KAFMM_STOKES_DL)
    pr = P_DL;
  else if (P.kernel == KAFMM_LAPLACE_QUAD)
    pr = P_LAPQ;
  else if (P.kernel == KAFMM_STOKES_PVEL_GRAD || P.kernel == KAFMM_STOKES_PVEL_LAPL ||
           P.kernel == KAFMM_STOKES_PVEL_TRACTION)
    pr = P_PVEL_D;
  else
    pr = P_DL_D;
  (void)dtype;
  int sd = dtype;
#define DISPATCH(T)                                          \
  switch (pr) {                                              \
    case P_LAP: return run_eval<T, P_LAP>(P, s, sd, g);      \
    case P_STK_L4: return run_eval<T, P_STK_L4>(P, s, sd, g); \
    case P_STK_G: return run_eval<T, P_STK_G>(P, s, sd, g);  \
    case P_RPY_L4: return run_eval<T, P_RPY_L4>(P, s, sd, g); \
    case P_RPY_G: return run_eval<T, P_RPY_G>(P, s, sd, g);  \
    case P_REG_G: return run_eval<T, P_REG_G>(P, s, sd, g);  \
    case P_LAPQD: return run_eval<T, P_LAPQD>(P, s, sd, g);  \
    case P_PVEL: return run_eval<T, P_PVEL>(P, s, sd, g);    \
    case P_DL: return run_eval<T, P_DL>(P, s, sd, g);        \
    case P_PVEL_D: return run_eval<T, P_PVEL_D>(P, s, sd, g); \
    case P_LAPQ: return run_eval<T, P_LAPQ>(P, s, sd, g);    \
    default: return run_eval<T, P_DL_D>(P, s, sd, g);        \
  }
  if (P.fp64()) {
    DISPATCH(double)
  } else {
    DISPATCH(float)
  }
#undef DISPATCH
}

}  // namespace kafmm
