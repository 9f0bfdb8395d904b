// Kernel functions of the summation problems (Yan & Blackwell, Sec. II), as device code.
// r = x - y (target minus source); pairs with r^2 == 0 contribute nothing.
#pragma once
#include "common.cuh"

namespace kafmm {

// Problem = kernel + ML-tree table.
// P_PVEL_D / P_DL_D: the StokesPVel and double-layer problems with derivative target values
// (Tables tab:ktab_stkslpvelgrad, tab:ktab_stkdlpvelgrad): [p, u, grad p, grad u] at every
// target, from which the Laplacian and traction forms are taken.
// P_LAPQ: Laplace quadrupole sources (9 values) to [phi, grad phi, grad grad phi] on the Laplace
// table (LapQPGradGrad of Table tab:implement).
enum Prob { P_LAP = 0, P_STK_L4 = 1, P_STK_G = 2, P_RPY_L4 = 3, P_RPY_G = 4, P_DL = 5, P_REG_G = 6,
            P_LAPQD = 7, P_PVEL = 8, P_PVEL_D = 9, P_DL_D = 10, P_LAPQ = 11 };

// [f, q] sources, double-layer D sources, and the StokesPVel ML table shared by all four.
__host__ __device__ constexpr bool pvel_src(int pr) { return pr == P_PVEL || pr == P_PVEL_D; }
__host__ __device__ constexpr bool dl_src(int pr) { return pr == P_DL || pr == P_DL_D; }
__host__ __device__ constexpr bool pvel_table(int pr) { return pvel_src(pr) || dl_src(pr); }
__host__ __device__ constexpr bool deriv_out(int pr) { return pr == P_PVEL_D || pr == P_DL_D; }

template <int PR>
struct ProbInfo;
template <>
struct ProbInfo<P_LAP> { static constexpr int KT = 1, C = 1, D = 1, NV = 1; };
template <>
struct ProbInfo<P_STK_L4> { static constexpr int KT = 3, C = 4, D = 1, NV = 1; };
template <>
struct ProbInfo<P_STK_G> { static constexpr int KT = 3, C = 1, D = 3, NV = 1; };
template <>
struct ProbInfo<P_RPY_L4> { static constexpr int KT = 6, C = 4, D = 1, NV = 1; };
template <>
struct ProbInfo<P_RPY_G> { static constexpr int KT = 6, C = 1, D = 3, NV = 1; };
// The double layer runs on the StokesPVel table: [f, q] per equivalent point, [p, u] per check
// point (D = 4 rows per surface point).
template <>
struct ProbInfo<P_DL> { static constexpr int KT = 4, C = 1, D = 4, NV = 3; };
template <>
struct ProbInfo<P_REG_G> { static constexpr int KT = 3, C = 1, D = 3, NV = 1; };
template <>
struct ProbInfo<P_LAPQD> { static constexpr int KT = 10, C = 1, D = 1, NV = 1; };
template <>
struct ProbInfo<P_PVEL> { static constexpr int KT = 4, C = 1, D = 4, NV = 1; };
template <>
struct ProbInfo<P_PVEL_D> { static constexpr int KT = 16, C = 1, D = 4, NV = 1; };
template <>
struct ProbInfo<P_DL_D> { static constexpr int KT = 16, C = 1, D = 4, NV = 3; };
template <>
struct ProbInfo<P_LAPQ> { static constexpr int KT = 10, C = 1, D = 1, NV = 3; };

template <class T>
struct V4;
template <>
struct V4<float> { using type = float4; };
template <>
struct V4<double> { using type = double4; };

template <class T>
__device__ inline T rsqrt_(T x);
template <>
__device__ inline float rsqrt_<float>(float x) { return rsqrtf(x); }
template <>
__device__ inline double rsqrt_<double>(double x) { return rsqrt(x); }

// 1 / r for r^2 > 0, else 0.
template <class T>
__device__ inline T inv_r(T rr) { return rr > T(0) ? rsqrt_<T>(rr) : T(0); }

// ---- S->T and the check potentials of S->M / S->L -------------------------------------------
// Source values: v0 = (q | f1 f2 f3 [b]) ; DL: v0 = D00 D01 D02 D10, v1 = D11 D12 D20 D21,
// v2 = D22.  acc has KT entries.

// r^2 without contracted multiply-adds: the RPY contact test gives the same answer in the leaf
// kernel and in the sphere-velocity pass.
__device__ __forceinline__ float rr_exact(float r0, float r1, float r2) {
  return __fadd_rn(__fadd_rn(__fmul_rn(r0, r0), __fmul_rn(r1, r1)), __fmul_rn(r2, r2));
}
__device__ __forceinline__ double rr_exact(double r0, double r1, double r2) {
  return __dadd_rn(__dadd_rn(__dmul_rn(r0, r0), __dmul_rn(r1, r1)), __dmul_rn(r2, r2));
}
// Pair within contact: r^2 <= (bi + bj)^2, from global coordinates x - (y + shift).
template <class T>
__device__ __forceinline__ bool in_contact(T x0, T x1, T x2, T y0, T y1, T y2, T s0, T s1, T s2, T bi, T bj) {
  T cs = bi + bj;
  return rr_exact(x0 - (y0 + s0), x1 - (y1 + s1), x2 - (y2 + s2)) <= cs * cs;
}

// 1/sqrt(x) for normal x > 0 in one approximate instruction (inputs here are squared distances
// between distinct points in the unit cube, far above the subnormal range; zero is tested
// before the call).
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// One Stokeslet pair in FP32 accumulated into acc[0..2] (scaled by 1/(8 pi) at the end):
// acc += f / r + r (r.f) / r^3 with r = x - y; zero for r = 0.  GUARD = false where r = 0
// cannot occur (sources of another box, or of an image of the target's box: distinct points).
template <bool GUARD = true>
__device__ __forceinline__ void stk_pair_f32(float xe, float ye, float ze, const float4& y,
                                             const float4& f, float* acc) {
  float r0 = xe - y.x, r1 = ye - y.y, r2 = ze - y.z;
  float rr = fmaf(r0, r0, fmaf(r1, r1, r2 * r2));
  float ir = GUARD ? (rr > 0.f ? rsqrt_ftz(rr) : 0.f) : rsqrt_ftz(rr);
  float rf = fmaf(r0, f.x, fmaf(r1, f.y, r2 * f.z)) * (ir * ir * ir);
  acc[0] = fmaf(r0, rf, fmaf(f.x, ir, acc[0]));
  acc[1] = fmaf(r1, rf, fmaf(f.y, ir, acc[1]));
  acc[2] = fmaf(r2, rf, fmaf(f.z, ir, acc[2]));
}

// Laplace L = 1/(4 pi r)
template <class T>
__device__ inline void lap_st(T r0, T r1, T r2, T q, T* acc) {
  T ir = inv_r(r0 * r0 + r1 * r1 + r2 * r2);
  acc[0] += q * ir;  // scaled by 1/(4 pi) at the end
}

// Charges and dipoles to potential, gradient and Hessian (Sec. II.A, Table
// tab:ktab_lapqdpgradgrad), all scaled by 1/(4 pi) at the end; r = x - y:
//   phi = q/r + (d.r)/r^3,  d_i phi = -q r_i/r^3 + d_i/r^3 - 3 (d.r) r_i/r^5,
//   d_i d_j phi = q (3 r_i r_j - delta_ij r^2)/r^5 - 3 (d_i r_j + d_j r_i + (d.r) delta_ij)/r^5
//                 + 15 (d.r) r_i r_j / r^7;   Hessian order xx xy xz yy yz zz.
template <class T, bool DIPOLE>
__device__ inline void lapqd_st(T r0, T r1, T r2, T q, T d0, T d1, T d2, T* acc) {
  T ir = inv_r(r0 * r0 + r1 * r1 + r2 * r2);
  T ir2 = ir * ir, ir3 = ir2 * ir, ir5 = ir3 * ir2;
  const T r[3] = {r0, r1, r2};
  const T d[3] = {d0, d1, d2};
  T dr = DIPOLE ? (d0 * r0 + d1 * r1 + d2 * r2) : T(0);
  T a3 = T(3) * ir5 * q;                      // charge Hessian: a3 r_i r_j - q ir3 delta_ij
  T c5 = DIPOLE ? T(15) * dr * ir5 * ir2 : T(0);
  T m3 = DIPOLE ? T(3) * ir5 : T(0);
  acc[0] += q * ir + dr * ir3;
#pragma unroll
  for (int i = 0; i < 3; ++i) acc[1 + i] += -q * r[i] * ir3 + (DIPOLE ? d[i] * ir3 - T(3) * dr * r[i] * ir5 : T(0));
  int c = 4;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      T h = a3 * r[i] * r[j] + (DIPOLE ? c5 * r[i] * r[j] - m3 * (d[i] * r[j] + d[j] * r[i]) : T(0));
      if (i == j) h -= q * ir3 + (DIPOLE ? m3 * dr : T(0));
      acc[c++] += h;
    }
}

// Stokeslet u = (f / r + r (r.f) / r^3): scaled by 1/(8 pi) at the end
template <class T>
__device__ inline void stk_st(T r0, T r1, T r2, T f0, T f1, T f2, T* acc) {
  T ir = inv_r(r0 * r0 + r1 * r1 + r2 * r2);
  T ir3 = ir * ir * ir;
  T rf = (r0 * f0 + r1 * f1 + r2 * f2) * ir3;
  acc[0] += f0 * ir + r0 * rf;
  acc[1] += f1 * ir + r1 * rf;
  acc[2] += f2 * ir + r2 * rf;
}

// Regularized Stokeslet (Sec. II.B, force f spread over the blob of width eps):
//   8 pi u = [(r^2 + 2 eps^2) f + r (r.f)] / (r^2 + eps^2)^{3/2}; the pair at r = 0 is skipped.
template <class T>
__device__ inline void reg_st(T r0, T r1, T r2, T f0, T f1, T f2, T eps, T* acc) {
  T rr = r0 * r0 + r1 * r1 + r2 * r2;
  if (rr == T(0)) return;
  T ee = eps * eps;
  T id = rsqrt_<T>(rr + ee);
  T id3 = id * id * id;
  T h1 = (rr + T(2) * ee) * id3;
  T rf = (r0 * f0 + r1 * f1 + r2 * f2) * id3;
  acc[0] += h1 * f0 + r0 * rf;
  acc[1] += h1 * f1 + r1 * rf;
  acc[2] += h1 * f2 + r2 * rf;
}

// RPY: u = G f + b^2/6 lap G f, lap u = lap G f with lap G = (I/r^3 - 3 r r^T / r^5)/(4 pi).
// acc[0..2] scaled by 1/(8 pi), acc[3..5] by 1/(4 pi) at the end:
//   8 pi u   = f/r + r (r.f)/r^3 + b^2/3 (f/r^3 - 3 r (r.f)/r^5)
//   4 pi lap = f/r^3 - 3 r (r.f)/r^5
template <class T>
__device__ inline void rpy_st(T r0, T r1, T r2, T f0, T f1, T f2, T b, T* acc) {
  T ir = inv_r(r0 * r0 + r1 * r1 + r2 * r2);
  T ir2 = ir * ir, ir3 = ir2 * ir;
  T rf = r0 * f0 + r1 * f1 + r2 * f2;
  T c3 = T(3) * rf * ir2;  // 3 (r.f)/r^2
  T l0 = (f0 - r0 * c3) * ir3, l1 = (f1 - r1 * c3) * ir3, l2 = (f2 - r2 * c3) * ir3;
  T bb = b * b * T(1.0 / 3.0);
  T g = rf * ir3;
  acc[0] += f0 * ir + r0 * g + bb * l0;
  acc[1] += f1 * ir + r1 * g + bb * l1;
  acc[2] += f2 * ir + r2 * g + bb * l2;
  acc[3] += l0;
  acc[4] += l1;
  acc[5] += l2;
}

// StokesPVel (Eqs. stkslp, stkslvel) from an equivalent point's [f, q]:
//   4 pi p = (r.f) / r^3 (acc[0]),  8 pi u = f / r + r (r.f) / r^3 - r q / r^3 (acc[1..3]).
template <class T>
__device__ inline void pvel_st(T r0, T r1, T r2, T f0, T f1, T f2, T q, T* acc) {
  T ir = inv_r(r0 * r0 + r1 * r1 + r2 * r2);
  T ir3 = ir * ir * ir;
  T rf = (r0 * f0 + r1 * f1 + r2 * f2) * ir3;
  T g = rf - q * ir3;
  acc[0] += rf;
  acc[1] += f0 * ir + r0 * g;
  acc[2] += f1 * ir + r1 * g;
  acc[3] += f2 * ir + r2 * g;
}

// Stokes double layer: 4 pi p = -3 (r.D.r)/r^5 + tr D / r^3 ; 8 pi u = -3 r (r.D.r) / r^5.
// acc[0] scaled by 1/(4 pi), acc[1..3] by 1/(8 pi) at the end.
template <class T>
__device__ inline void dl_st(T r0, T r1, T r2, const T* Dm, T* acc) {
  T ir = inv_r(r0 * r0 + r1 * r1 + r2 * r2);
  T ir2 = ir * ir, ir3 = ir2 * ir, ir5 = ir3 * ir2;
  T rDr = r0 * (Dm[0] * r0 + Dm[1] * r1 + Dm[2] * r2) + r1 * (Dm[3] * r0 + Dm[4] * r1 + Dm[5] * r2) +
          r2 * (Dm[6] * r0 + Dm[7] * r1 + Dm[8] * r2);
  T tr = Dm[0] + Dm[4] + Dm[8];
  acc[0] += -T(3) * rDr * ir5 + tr * ir3;
  T c = -T(3) * rDr * ir5;
  acc[1] += c * r0;
  acc[2] += c * r1;
  acc[3] += c * r2;
}

// StokesPVel with its derivatives (Eqs. stkslp, stkslvel differentiated in x) from [f, q]:
// [p, u, grad p, grad u] with grad u = d u_i / d x_j at 7 + 3 i + j; acc[0] and acc[4..6] are
// scaled by 1/(4 pi), the rest by 1/(8 pi) at the end:
//   4 pi d_j p   = f_j / r^3 - 3 (r.f) r_j / r^5,
//   8 pi d_j u_i = [delta_ij (r.f - q) + r_i f_j - f_i r_j] / r^3 + 3 r_i r_j (q - r.f) / r^5.
template <class T>
__device__ inline void pvel_grad_st(T r0, T r1, T r2, T f0, T f1, T f2, T q, T* acc) {
  T ir = inv_r(r0 * r0 + r1 * r1 + r2 * r2);
  T ir2 = ir * ir, ir3 = ir2 * ir, ir5 = ir3 * ir2;
  const T r[3] = {r0, r1, r2}, f[3] = {f0, f1, f2};
  T rf = r0 * f0 + r1 * f1 + r2 * f2;
  T g = (rf - q) * ir3;
  T c = T(3) * rf * ir5;
  T e = T(3) * (q - rf) * ir5;
  acc[0] += rf * ir3;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    acc[1 + i] += f[i] * ir + r[i] * g;
    acc[4 + i] += f[i] * ir3 - c * r[i];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      acc[7 + 3 * i + j] += (r[i] * f[j] - f[i] * r[j]) * ir3 + r[i] * r[j] * e + (i == j ? g : T(0));
}

// Double layer with its derivatives (Eqs. stkdlp, stkdlvel differentiated in x), same layout
// and scaling; rDr = r.D.r, a_j = (D r)_j + (D^T r)_j, t = tr D:
//   4 pi d_j p   = -3 a_j / r^5 + 15 rDr r_j / r^7 - 3 t r_j / r^5,
//   8 pi d_j u_i = -3 [delta_ij rDr / r^5 + r_i a_j / r^5 - 5 r_i r_j rDr / r^7].
template <class T>
__device__ inline void dl_grad_st(T r0, T r1, T r2, const T* Dm, T* acc) {
  T ir = inv_r(r0 * r0 + r1 * r1 + r2 * r2);
  T ir2 = ir * ir, ir3 = ir2 * ir, ir5 = ir3 * ir2, ir7 = ir5 * ir2;
  const T r[3] = {r0, r1, r2};
  T dr[3], a[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) dr[j] = Dm[3 * j] * r0 + Dm[3 * j + 1] * r1 + Dm[3 * j + 2] * r2;
#pragma unroll
  for (int j = 0; j < 3; ++j) a[j] = dr[j] + Dm[j] * r0 + Dm[3 + j] * r1 + Dm[6 + j] * r2;
  T rDr = r0 * dr[0] + r1 * dr[1] + r2 * dr[2];
  T t = Dm[0] + Dm[4] + Dm[8];
  T c5 = rDr * ir5, c7 = T(5) * rDr * ir7;
  acc[0] += -T(3) * c5 + t * ir3;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    acc[1 + i] += -T(3) * c5 * r[i];
    acc[4 + i] += -T(3) * a[i] * ir5 + T(3) * (c7 - t * ir5) * r[i];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      acc[7 + 3 * i + j] += -T(3) * ((i == j ? c5 : T(0)) + r[i] * a[j] * ir5 - r[i] * r[j] * c7);
}

// Laplace quadrupole Q (Q_jk at 3j + k) to potential, gradient and Hessian: phi = Q_jk d_j d_k L
// (L = 1/(4 pi r), derivatives in x), scaled by 1/(4 pi) at the end.  With S = sym(Q),
// s = S r, rQr = r.Q.r, t = tr Q:
//   4 pi phi         = 3 rQr / r^5 - t / r^3,
//   4 pi d_i phi     = -15 r_i rQr / r^7 + 3 (2 s_i + t r_i) / r^5,
//   4 pi d_i d_l phi = 105 r_i r_l rQr / r^9 - 15 (delta_il rQr + 2 r_l s_i + 2 r_i s_l + t r_i r_l) / r^7
//                      + 3 (delta_il t + 2 S_il) / r^5;   Hessian order xx xy xz yy yz zz.
template <class T>
__device__ inline void quad_st(T r0, T r1, T r2, const T* Q, T* acc) {
  T ir = inv_r(r0 * r0 + r1 * r1 + r2 * r2);
  T ir2 = ir * ir, ir3 = ir2 * ir, ir5 = ir3 * ir2, ir7 = ir5 * ir2, ir9 = ir7 * ir2;
  const T r[3] = {r0, r1, r2};
  T S[9], sv[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) S[3 * a + b] = T(0.5) * (Q[3 * a + b] + Q[3 * b + a]);
#pragma unroll
  for (int a = 0; a < 3; ++a) sv[a] = S[3 * a] * r0 + S[3 * a + 1] * r1 + S[3 * a + 2] * r2;
  const T rQr = r0 * sv[0] + r1 * sv[1] + r2 * sv[2];
  const T t = Q[0] + Q[4] + Q[8];
  acc[0] += T(3) * rQr * ir5 - t * ir3;
#pragma unroll
  for (int i = 0; i < 3; ++i) acc[1 + i] += -T(15) * r[i] * rQr * ir7 + T(3) * (T(2) * sv[i] + t * r[i]) * ir5;
  int c = 4;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int l = i; l < 3; ++l) {
      T h = T(105) * r[i] * r[l] * rQr * ir9 -
            T(15) * (T(2) * r[l] * sv[i] + T(2) * r[i] * sv[l] + t * r[i] * r[l]) * ir7 + T(6) * S[3 * i + l] * ir5;
      if (i == l) h += -T(15) * rQr * ir7 + T(3) * t * ir5;
      acc[c++] += h;
    }
}

// Final scale factors of the accumulators.
template <int PR, class T>
__device__ inline T out_scale(int k) {
  const T f4 = T(1.0 / (4.0 * PI)), f8 = T(1.0 / (8.0 * PI));
  if (PR == P_LAP || PR == P_LAPQD || PR == P_LAPQ) return f4;
  if (PR == P_STK_L4 || PR == P_STK_G || PR == P_REG_G) return f8;
  if (PR == P_RPY_L4 || PR == P_RPY_G) return k < 3 ? f8 : f4;
  if (deriv_out(PR)) return (k == 0 || (k >= 4 && k < 7)) ? f4 : f8;   // [p, u, grad p, grad u]
  return k == 0 ? f4 : f8;  // DL, StokesPVel: [p, u]
}

}  // namespace kafmm
