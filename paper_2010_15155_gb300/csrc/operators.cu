// FP64 translation operators, built on the device at plan time.
//
// KIFMM matches potentials on check surfaces with equivalent densities (Sec. II); the
// check-to-equivalent map is the pseudo-inverse of a kernel matrix (Sec. II: an SVD
// pseudo-inverse as in PVFMM).  The ML-tree kernels (Laplace 1/(4 pi r), Stokeslet G) are
// homogeneous of degree -1, so with every box described in units of its own half-width the
// operators do not depend on the level.  The evaluator keeps the check potentials of each box
// and folds the pseudo-inverse into the translation operators:
//   M->L(o)  = K(dc <- ue at offset o) * UC2UE
//   M->M(c)  = K(uc parent <- ue child c) * UC2UE
//   L->L(c)  = 2 K(dc child c <- de parent) * DC2DE
// each formed through the SVD factors, (K V)(S^+ U^T), so the large entries of the
// pseudo-inverse never meet the rounding of the product.
// (geometry in units of the half-width of the child / of the box), which equals the paper's
// sequence "equivalent density = pinv * check, then translate" up to rounding.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "plan.cuh"

namespace kafmm {

std::vector<double> unit_surface(int m) {
  std::vector<double> pts;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j)
      for (int k = 0; k < m; ++k) {
        int lo = std::min(i, std::min(j, k)), hi = std::max(i, std::max(j, k));
        if (lo == 0 || hi == m - 1) {
          pts.push_back(-1.0 + 2.0 * i / (m - 1));
          pts.push_back(-1.0 + 2.0 * j / (m - 1));
          pts.push_back(-1.0 + 2.0 * k / (m - 1));
        }
      }
  return pts;
}

// K[i][j] (R x R): target points ct + at * s_i, source points cs + as * s_j.
// ML kernels: stokes = 0 Laplace (1 x 1 per point pair), 1 Stokeslet G (3 x 3), 2 StokesPVel
// G^P (4 x 4: rows p, u; columns f, q; Eqs. stkslp, stkslvel).
__global__ void k_fill_kernel_matrix(const double* __restrict__ unit, int n, int stokes, double ctx,
                                     double cty, double ctz, double at, double csx, double csy,
                                     double csz, double as, double* __restrict__ K) {
  int R = stokes == 2 ? 4 * n : (stokes ? 3 * n : n);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    double r0 = (ctx + at * unit[3 * i]) - (csx + as * unit[3 * j]);
    double r1 = (cty + at * unit[3 * i + 1]) - (csy + as * unit[3 * j + 1]);
    double r2 = (ctz + at * unit[3 * i + 2]) - (csz + as * unit[3 * j + 2]);
    double rr = r0 * r0 + r1 * r1 + r2 * r2;
    double rn = sqrt(rr);
    if (!stokes) {
      K[(int64_t)i * R + j] = 1.0 / (4.0 * PI * rn);
    } else if (stokes == 2) {
      double r[3] = {r0, r1, r2};
      double inv = 1.0 / (8.0 * PI * rn), inv3 = inv / rr;
      for (int b = 0; b < 3; ++b) K[(int64_t)(4 * i) * R + 4 * j + b] = 2.0 * r[b] * inv3;
      K[(int64_t)(4 * i) * R + 4 * j + 3] = 0.0;
      for (int a2 = 0; a2 < 3; ++a2) {
        for (int b = 0; b < 3; ++b)
          K[(int64_t)(4 * i + 1 + a2) * R + 4 * j + b] = (a2 == b ? inv : 0.0) + r[a2] * r[b] * inv3;
        K[(int64_t)(4 * i + 1 + a2) * R + 4 * j + 3] = -r[a2] * inv3;
      }
    } else {
      double r[3] = {r0, r1, r2};
      double inv = 1.0 / (8.0 * PI * rn), inv3 = inv / rr;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
          K[(int64_t)(3 * i + a) * R + 3 * j + b] = (a == b ? inv : 0.0) + r[a] * r[b] * inv3;
    }
  }
}

// Batch of M->L kernel matrices, one per blockIdx.z: K_z = K(dc of the box at the origin <- ue of
// the box whose centre is 2 offs[z] away), the layout of k_fill_kernel_matrix, K_z at K + z sK.
__global__ void k_fill_m2l_batch(const double* __restrict__ unit, int n, int stokes, double at, double as,
                                 const int* __restrict__ offs, double* __restrict__ K, int64_t sK) {
  const int z = blockIdx.z;
  const double csx = 2.0 * offs[3 * z], csy = 2.0 * offs[3 * z + 1], csz = 2.0 * offs[3 * z + 2];
  double* Kz = K + z * sK;
  int R = stokes == 2 ? 4 * n : (stokes ? 3 * n : n);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    double r0 = (at * unit[3 * i]) - (csx + as * unit[3 * j]);
    double r1 = (at * unit[3 * i + 1]) - (csy + as * unit[3 * j + 1]);
    double r2 = (at * unit[3 * i + 2]) - (csz + as * unit[3 * j + 2]);
    double rr = r0 * r0 + r1 * r1 + r2 * r2;
    double rn = sqrt(rr);
    if (!stokes) {
      Kz[(int64_t)i * R + j] = 1.0 / (4.0 * PI * rn);
    } else if (stokes == 2) {
      double r[3] = {r0, r1, r2};
      double inv = 1.0 / (8.0 * PI * rn), inv3 = inv / rr;
      for (int b = 0; b < 3; ++b) Kz[(int64_t)(4 * i) * R + 4 * j + b] = 2.0 * r[b] * inv3;
      Kz[(int64_t)(4 * i) * R + 4 * j + 3] = 0.0;
      for (int a2 = 0; a2 < 3; ++a2) {
        for (int b = 0; b < 3; ++b)
          Kz[(int64_t)(4 * i + 1 + a2) * R + 4 * j + b] = (a2 == b ? inv : 0.0) + r[a2] * r[b] * inv3;
        Kz[(int64_t)(4 * i + 1 + a2) * R + 4 * j + 3] = -r[a2] * inv3;
      }
    } else {
      double r[3] = {r0, r1, r2};
      double inv = 1.0 / (8.0 * PI * rn), inv3 = inv / rr;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
          Kz[(int64_t)(3 * i + a) * R + 3 * j + b] = (a == b ? inv : 0.0) + r[a] * r[b] * inv3;
    }
  }
}

// Multiplies every 4th row (rows = 1, starting at first) or column (rows = 0) of the R x R
// matrix K by f: the StokesPVel p rows or q columns.
__global__ void k_scale_every4(double* __restrict__ K, int R, int rows, int first, double f) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)R * R;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / R), j = (int)(e % R);
    if (((rows ? i : j) & 3) == first) K[e] *= f;
  }
}

// Transpose: out[j][i] = in[i][j].
__global__ void k_transpose(const double* __restrict__ in, int n, double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    out[(int64_t)j * n + i] = in[e];
  }
}

__global__ void k_identity(double* V, int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x)
    V[e] = (e / n == e % n) ? 1.0 : 0.0;
}

// Grid-wide barrier of a cooperative launch (every block resident): sense by generation
// counter, the wait bounded by %globaltimer.  Returns false (ST_TIMEOUT in *status) when the
// other blocks did not arrive within limit_ns.
__device__ bool grid_barrier(unsigned* count, unsigned* gen, unsigned nblocks, unsigned* status,
                             unsigned long long limit_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned g = *(volatile unsigned*)gen;
    __threadfence();
    if (atomicAdd(count, 1u) + 1u == nblocks) {
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
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// One-sided (Hestenes) Jacobi SVD of the rows of At (= columns of A), whole decomposition in one
// cooperative launch: per sweep the n - 1 rounds of the round-robin schedule, each round's n/2
// disjoint pairs spread over the blocks, a grid barrier after every round.  A sweep that rotates
// no pair (|a_i . a_j| <= tol |a_i| |a_j| for all pairs) ends the iteration.  st (device ints):
// [0..2] rotated flag of sweep s at s % 3, [3..5] largest relative off-orthogonality of sweep s
// (float bits), [6] sweeps done, [7] barrier count, [8] barrier generation.
__global__ void __launch_bounds__(256) k_jacobi_svd(double* __restrict__ At, double* __restrict__ Vt, int n,
                                                    double tol, int max_sweeps, unsigned* st,
                                                    unsigned* status, unsigned long long limit_ns) {
  __shared__ double red[3][8];
  __shared__ double cs[2];
  const unsigned nb = gridDim.x;
  auto player = [&](int pos, int round) { return pos == 0 ? 0 : ((pos - 1 + round) % (n - 1)) + 1; };
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    unsigned* rotated = st + sweep % 3;
    unsigned* worst = st + 3 + sweep % 3;
    if (blockIdx.x == 0 && threadIdx.x == 0) {   // nobody touches the next sweep's slots now
      st[(sweep + 1) % 3] = 0u;
      st[3 + (sweep + 1) % 3] = 0u;
    }
    for (int round = 0; round < n - 1; ++round) {
      for (int pr = blockIdx.x; pr < n / 2; pr += nb) {
        const int i = player(pr, round), j = player(n - 1 - pr, round);
        double* ai = At + (int64_t)i * n;
        double* aj = At + (int64_t)j * n;
        double a = 0, b = 0, g = 0;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
          double x = ai[k], y = aj[k];
          a += x * x;
          b += y * y;
          g += x * y;
        }
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_down_sync(0xffffffffu, a, o);
          b += __shfl_down_sync(0xffffffffu, b, o);
          g += __shfl_down_sync(0xffffffffu, g, o);
        }
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) {
          red[0][w] = a;
          red[1][w] = b;
          red[2][w] = g;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          a = b = g = 0;
          for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            a += red[0][k];
            b += red[1][k];
            g += red[2][k];
          }
          double c = 1.0, s = 0.0;
          if (a > 0 && b > 0) atomicMax(worst, __float_as_uint((float)(fabs(g) / sqrt(a * b))));
          if (fabs(g) > tol * sqrt(a * b) && a > 0 && b > 0) {
            double zeta = (b - a) / (2.0 * g);
            double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            c = 1.0 / sqrt(1.0 + t * t);
            s = c * t;
            *(volatile unsigned*)rotated = 1u;
          }
          cs[0] = c;
          cs[1] = s;
        }
        __syncthreads();
        const double c = cs[0], s = cs[1];
        if (s != 0.0) {
          double* vi = Vt + (int64_t)i * n;
          double* vj = Vt + (int64_t)j * n;
          for (int k = threadIdx.x; k < n; k += blockDim.x) {
            double x = ai[k], y = aj[k];
            ai[k] = c * x - s * y;
            aj[k] = s * x + c * y;
            x = vi[k];
            y = vj[k];
            vi[k] = c * x - s * y;
            vj[k] = s * x + c * y;
          }
        }
        __syncthreads();
      }
      if (!grid_barrier(st + 7, st + 8, nb, status, limit_ns)) return;
    }
    const bool again = *(volatile unsigned*)rotated != 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) st[6] = (unsigned)(sweep + 1);
    if (!again) return;
  }
}

__global__ void k_row_norms(const double* At, int n, double* w) {
  int k = blockIdx.x;
  double s = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += At[(int64_t)k * n + i] * At[(int64_t)k * n + i];
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    w[k] = t;  // sigma_k^2
  }
}

// w[k] <- 1 / sigma_k^2 for sigma_k >= rcond * sigma_max, else 0.
__global__ void k_pinv_weights(double* w, int n, double rcond) {
  __shared__ double smax;
  if (threadIdx.x == 0) {
    double m = 0;
    for (int k = 0; k < n; ++k) m = fmax(m, w[k]);
    smax = m;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double s2 = w[k];
    w[k] = (s2 > 0 && sqrt(s2) >= rcond * sqrt(smax)) ? 1.0 / s2 : 0.0;
  }
}

// C = alpha * op(A) * diag(w) * B with op(A) = A^T when ta (A stored [k][i]) else A ([i][k]).
// Plain 32x32-tiled FP64 GEMM; n x n x n.
// Batched over blockIdx.z: A_z = A + z sA, C_z = Cm + (cidx ? cidx[z] : z) sC (B shared).
__global__ void k_gemm64(const double* __restrict__ A, int ta, const double* __restrict__ w,
                         const double* __restrict__ B, double alpha, int n, double* __restrict__ Cm,
                         int64_t sA = 0, int64_t sC = 0, const int* __restrict__ cidx = nullptr) {
  A += blockIdx.z * sA;
  Cm += (cidx ? cidx[blockIdx.z] : (int)blockIdx.z) * sC;
  __shared__ double As[32][33], Bs[32][33];
  int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  double acc[4] = {0, 0, 0, 0};
  for (int k0 = 0; k0 < n; k0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      int i = i0 + r, k = k0 + tx;
      double av = 0;
      if (ta) {
        int kk = k0 + r, ii = i0 + tx;  // As[r=k][tx=i]
        av = (kk < n && ii < n) ? A[(int64_t)kk * n + ii] * (w ? w[kk] : 1.0) : 0.0;
        As[tx][r] = av;
      } else {
        av = (i < n && k < n) ? A[(int64_t)i * n + k] * (w ? w[k] : 1.0) : 0.0;
        As[r][tx] = av;
      }
      int kb = k0 + r, jb = j0 + tx;
      Bs[r][tx] = (kb < n && jb < n) ? B[(int64_t)kb * n + jb] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      double b = Bs[k][tx];
      for (int q = 0; q < 4; ++q) acc[q] += As[ty + 8 * q][k] * b;
    }
    __syncthreads();
  }
  for (int q = 0; q < 4; ++q) {
    int i = i0 + ty + 8 * q, j = j0 + tx;
    if (i < n && j < n) Cm[(int64_t)i * n + j] = alpha * acc[q];
  }
}

__global__ void k_scale_rows(const double* in, const double* w, int n, double* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = in[e] * w[e / n];
}

// Periodic far-image operator at unit scale (root half-width 1, period 2):
//   T[i][j] = G_per(dc_i - ue_j) - sum_{max|n| <= 1} K(dc_i - ue_j - 2n)
// with G_per the Ewald sum with the k = 0 mode removed (Laplace; Stokeslet by Hasimoto's split,
// weight (1 + k^2/4xi^2) e^{-k^2/4xi^2}).  xi = 2 (xi * period = 4), real images |n| <= 2,
// Fourier modes |m| <= 8 (converged to FP64 rounding).  Where dc_i and ue_j coincide, the n = 0
// real-space term is replaced by its regular limit and the n = 0 near image is left out.
// StokesPVel (stokes = 2, 4 x 4 blocks [p, u] <- [f, q]): u <- f is Hasimoto's Stokeslet; the
// pressure of a force and the flow of a source are gradients of the Laplace function,
// p = -f . grad G and u = (q / 2) grad G, taken periodically from grad G_per (real-space terms
// differentiated, Fourier terms -k e^{-k^2/4xi^2} sin(k.r) / (k^2 V)); p <- q is zero.
__global__ void k_periodic_operator(const double* __restrict__ unit, int n, int stokes, double adc,
                                    double aue, double* __restrict__ T) {
  const double Lp = 2.0, xi = 2.0, V = Lp * Lp * Lp;
  const double sp = 2.0 * xi / sqrt(PI);
  int R = stokes == 2 ? 4 * n : (stokes ? 3 * n : n);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    // products rounded separately (no FMA contraction), so coincident points give r = 0 exactly
    double r[3];
    for (int q = 0; q < 3; ++q) r[q] = __dmul_rn(adc, unit[3 * i + q]) - __dmul_rn(aue, unit[3 * j + q]);
    double m[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    double gl[3] = {0, 0, 0};   // grad G_per (StokesPVel)
    double lap = stokes ? 0.0 : -1.0 / (4.0 * xi * xi * V);
    for (int a = -2; a <= 2; ++a)
      for (int b = -2; b <= 2; ++b)
        for (int c = -2; c <= 2; ++c) {
          double d[3] = {r[0] + a * Lp, r[1] + b * Lp, r[2] + c * Lp};
          double rr = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
          double rn = sqrt(rr);
          // near images (max|n| <= 1) are removed again: there the real-space term minus the
          // free-space kernel is taken in the form -erf(xi r)/r, free of cancellation
          bool near = abs(a) <= 1 && abs(b) <= 1 && abs(c) <= 1;
          double ex = exp(-xi * xi * rr);
          double h = near ? -erf(xi * rn) : erfc(xi * rn);  // the erfc factor, minus 1 if near
          if (!stokes) {
            lap += rn == 0.0 ? -xi / (2.0 * PI * sqrt(PI)) : h / (4.0 * PI * rn);
          } else if (rn == 0.0) {
            for (int q = 0; q < 3; ++q) m[4 * q] += -2.0 * sp / (8.0 * PI);
          } else {
            double A = (h / rn - sp * ex) / (8.0 * PI), B = (h / rn + sp * ex) / (8.0 * PI) / rr;
            for (int p = 0; p < 3; ++p)
              for (int q = 0; q < 3; ++q) m[3 * p + q] += (p == q ? A : 0.0) + B * d[p] * d[q];
            if (stokes == 2) {   // d/dr (h(r) / r) = -sp e^{-xi^2 r^2} / r - h / r^2
              double gr = -(sp * ex * rn + h) / (4.0 * PI * rr * rn);
              for (int q = 0; q < 3; ++q) gl[q] += gr * d[q];
            }
          }
        }
    for (int a = -8; a <= 8; ++a)
      for (int b = -8; b <= 8; ++b)
        for (int c = -8; c <= 8; ++c) {
          if (a == 0 && b == 0 && c == 0) continue;
          double kv[3] = {2.0 * PI * a / Lp, 2.0 * PI * b / Lp, 2.0 * PI * c / Lp};
          double k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
          double cs = cos(kv[0] * r[0] + kv[1] * r[1] + kv[2] * r[2]);
          double g = exp(-k2 / (4.0 * xi * xi)) / (k2 * V) * cs;
          if (!stokes) {
            lap += g;
          } else {
            if (stokes == 2) {
              double sn = -exp(-k2 / (4.0 * xi * xi)) / (k2 * V) * sin(kv[0] * r[0] + kv[1] * r[1] + kv[2] * r[2]);
              for (int q = 0; q < 3; ++q) gl[q] += sn * kv[q];
            }
            g *= 1.0 + k2 / (4.0 * xi * xi);
            for (int p = 0; p < 3; ++p)
              for (int q = 0; q < 3; ++q) m[3 * p + q] += g * ((p == q ? 1.0 : 0.0) - kv[p] * kv[q] / k2);
          }
        }
    if (!stokes) {
      T[(int64_t)i * R + j] = lap;
    } else if (stokes == 2) {
      for (int q = 0; q < 3; ++q) T[(int64_t)(4 * i) * R + 4 * j + q] = -gl[q];
      T[(int64_t)(4 * i) * R + 4 * j + 3] = 0.0;
      for (int p = 0; p < 3; ++p) {
        for (int q = 0; q < 3; ++q) T[(int64_t)(4 * i + 1 + p) * R + 4 * j + q] = m[3 * p + q];
        T[(int64_t)(4 * i + 1 + p) * R + 4 * j + 3] = 0.5 * gl[p];
      }
    } else {
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) T[(int64_t)(3 * i + p) * R + 3 * j + q] = m[3 * p + q];
    }
  }
}

// Singly / doubly periodic far-image operator at unit scale (root half-width 1, period 2):
//   T[i][j] = lim_{N -> inf} sum_{2 <= max|n| <= N} K(dc_i - ue_j - 2 n)
// over the images n = (a, 0, 0) (axes 1, PX) or (a, b, 0) (axes 2, PXY), in square shells
// max|n| = s.  One thread per (dc point, ue point) pair accumulates the Laplace value
// (stokes = 0) or the 3 x 3 Stokeslet block (stokes = 1) and writes the partial sums at
// N = n0 2^k, k < nlev, to part[k][R][R]; k_lattice_extrapolate takes N -> infinity.
__global__ void k_lattice_partials(const double* __restrict__ unit, int n, int stokes, double adc, double aue,
                                   int axes, int n0, int nlev, double* __restrict__ part) {
  const int D = stokes ? 3 : 1;
  const int64_t R = (int64_t)D * n, RR = R * R;
  const int nmax = n0 << (nlev - 1);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    double r[3];
    for (int q = 0; q < 3; ++q) r[q] = adc * unit[3 * i + q] - aue * unit[3 * j + q];
    double m[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    auto add = [&](int a, int b) {
      const double d0 = r[0] - 2.0 * a, d1 = r[1] - 2.0 * b, d2 = r[2];
      const double ri = rsqrt(d0 * d0 + d1 * d1 + d2 * d2);
      if (!stokes) {
        m[0] += ri;
        return;
      }
      const double r3 = ri * ri * ri;
      const double d[3] = {d0, d1, d2};
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) m[3 * p + q] += (p == q ? ri : 0.0) + d[p] * d[q] * r3;
    };
    int lev = 0;
    for (int s = 2; s <= nmax; ++s) {
      if (axes == 1) {
        add(-s, 0);
        add(s, 0);
      } else {   // the ring max(|a|, |b|) = s: four sides of 2 s images, each corner once
        for (int t = -s; t < s; ++t) {
          add(t, -s);
          add(s, t);
          add(-t, s);
          add(-s, -t);
        }
      }
      if (s == (n0 << lev)) {
        const double c = stokes ? 1.0 / (8.0 * PI) : 1.0 / (4.0 * PI);
        for (int p = 0; p < D; ++p)
          for (int q = 0; q < D; ++q) part[lev * RR + (int64_t)(D * i + p) * R + D * j + q] = c * m[D * p + q];
        ++lev;
      }
    }
  }
}

// N -> infinity from the partial sums at N = n0 2^k: the tails are power series in 1/N (sums
// of smooth functions over the lattice cells outside a square, by the midpoint rule), removed
// one power per level by repeated Richardson extrapolation.
__global__ void k_lattice_extrapolate(const double* __restrict__ part, int nlev, int64_t count,
                                      double* __restrict__ T) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    double t[12];
    for (int k = 0; k < nlev; ++k) t[k] = part[k * count + e];
    for (int j = 1; j < nlev; ++j) {
      const double f = (double)(1 << j);
      for (int k = 0; k + j < nlev; ++k) t[k] = (f * t[k + 1] - t[k]) / (f - 1.0);
    }
    T[e] = t[0];
  }
}

// Projection onto neutral densities: per row of T (R x R, D components per point) and source
// component c, subtract the mean over the n equivalent points.  The image sums of a net charge
// or force diverge with N (a constant matrix per component pair); a neutral density is left
// unchanged.  One block of 256 threads per row.
__global__ void k_project_neutral(double* __restrict__ T, int n, int D) {
  const int64_t R = (int64_t)D * n;
  double* row = T + blockIdx.x * R;
  __shared__ double part[3][256];
  double acc[3] = {0, 0, 0};
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    for (int c = 0; c < D; ++c) acc[c] += row[D * j + c];
  for (int c = 0; c < 3; ++c) part[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int c = 0; c < 3; ++c) part[c][threadIdx.x] += part[c][threadIdx.x + w];
    __syncthreads();
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    for (int c = 0; c < D; ++c) row[D * j + c] -= part[c][0] / n;
}

__global__ void k_round32(const double* in, int64_t n, float* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (float)in[e];
}

// Split into tf32 hi + lo (stored as fp32), columns padded with zeros: operator op has rows x
// cols entries at in[(op * rows + i) * ld + j]; out[(op * 2 + h)][i][colpad].
__global__ void k_split_tf32(const double* in, int rows, int cols, int ld, int colpad, int64_t nops,
                             float* out) {
  int64_t total = nops * rows * (int64_t)colpad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t op = e / ((int64_t)rows * colpad);
    int64_t rem = e % ((int64_t)rows * colpad);
    int i = (int)(rem / colpad), j = (int)(rem % colpad);
    float v = j < cols ? (float)in[(op * rows + i) * ld + j] : 0.f;
    uint32_t hb, lb;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(v));
    float hi = __uint_as_float(hb);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lb) : "f"(v - hi));
    out[((op * 2 + 0) * rows + i) * colpad + j] = hi;
    out[((op * 2 + 1) * rows + i) * colpad + j] = __uint_as_float(lb);
  }
}

// Split into bf16 hi + lo, the same layout as k_split_tf32.
__global__ void k_split_bf16(const double* in, int rows, int cols, int ld, int colpad, int64_t nops,
                             __nv_bfloat16* out) {
  int64_t total = nops * rows * (int64_t)colpad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t op = e / ((int64_t)rows * colpad);
    int64_t rem = e % ((int64_t)rows * colpad);
    int i = (int)(rem / colpad), j = (int)(rem % colpad);
    float v = j < cols ? (float)in[(op * rows + i) * ld + j] : 0.f;
    __nv_bfloat16 hi = __float2bfloat16_rn(v);
    __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    out[((op * 2 + 0) * rows + i) * colpad + j] = hi;
    out[((op * 2 + 1) * rows + i) * colpad + j] = lo;
  }
}

// General FP64 GEMM, C[M][N] (row stride ldc) = alpha op(A) op(B), op(A)[i][k] = A[i lda + k]
// (ta = 0) or A[k lda + i] (ta = 1), op(B)[k][j] = B[k ldb + j] (tb = 0) or B[j ldb + k].
// 32 x 32 tiles; plan time only.
// Batched over blockIdx.z: A, B and Cm advance by sA, sB and sC per batch index.
__global__ void k_gemm64g(const double* __restrict__ A, int lda, int ta, const double* __restrict__ B,
                          int ldb, int tb, double* __restrict__ Cm, int ldc, int M, int N, int K,
                          double alpha, int64_t sA = 0, int64_t sB = 0, int64_t sC = 0) {
  A += blockIdx.z * sA;
  B += blockIdx.z * sB;
  Cm += blockIdx.z * sC;
  __shared__ double As[32][33], Bs[32][33];
  int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  double acc[4] = {0, 0, 0, 0};
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      // As[i][k], Bs[k][j]
      int i = i0 + r, k = k0 + tx;
      As[r][tx] = (i < M && k < K) ? (ta ? A[(int64_t)k * lda + i] : A[(int64_t)i * lda + k]) : 0.0;
      int kb = k0 + r, j = j0 + tx;
      Bs[r][tx] = (kb < K && j < N) ? (tb ? B[(int64_t)j * ldb + kb] : B[(int64_t)kb * ldb + j]) : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      double b = Bs[k][tx];
      for (int q = 0; q < 4; ++q) acc[q] += As[ty + 8 * q][k] * b;
    }
    __syncthreads();
  }
  for (int q = 0; q < 4; ++q) {
    int i = i0 + ty + 8 * q, j = j0 + tx;
    if (i < M && j < N) Cm[(int64_t)i * ldc + j] = alpha * acc[q];
  }
}

// dst[i][0..n) = scale[i] * src[idx[i]][0..n) for i < nsel, zero rows for nsel <= i < rows.
__global__ void k_select_rows(const double* __restrict__ src, int n, const int* __restrict__ idx,
                              const double* __restrict__ scale, int nsel, int rows,
                              double* __restrict__ dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)rows * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    dst[e] = i < nsel ? scale[i] * src[(int64_t)idx[i] * n + j] : 0.0;
  }
}

// dst[j][0..cols) (row stride cols) = scale[i] * src[j][idx[i]] in column i < nsel, zero columns
// for nsel <= i < cols; src is n x n.
__global__ void k_select_cols(const double* __restrict__ src, int n, const int* __restrict__ idx,
                              const double* __restrict__ scale, int nsel, int cols,
                              double* __restrict__ dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    int j = (int)(e / cols), i = (int)(e % cols);
    dst[e] = i < nsel ? scale[i] * src[(int64_t)j * n + idx[i]] : 0.0;
  }
}

#define CK(call)                                           \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(P, e_, #call); \
  } while (0)

// Factored pinv of K (R x R) via one-sided Jacobi SVD: K = W V^T with orthogonal columns
// W = U S.  out1 = S^+ U^T = diag(w) W^T (w_k = 1/sigma_k^2 above the cutoff), out2 = V.
static int pinv64(Plan& P, const double* K, double* out1, double* out2, double* At, double* Vt,
                  double* w, int* flag, std::vector<double>* w_host = nullptr) {
  int R = P.R;
  cudaStream_t st = P.stream;
  int g = 512;
  KL k_transpose<<<g, 256, 0, st>>>(K, R, At);
  KL k_identity<<<g, 256, 0, st>>>(Vt, R);
  // stop when a sweep rotates no pair: |a_i . a_j| <= tol |a_i| |a_j| with tol = 4 R eps, the
  // level FP64 rounding of a length-R dot product can resolve
  double tol = 4.0 * R * 2.220446049250313e-16;
  int max_sweeps = 80;
  unsigned* jst = reinterpret_cast<unsigned*>(flag);   // 9 words, see k_jacobi_svd
  unsigned* status = jst + 12;
  CK(cudaMemsetAsync(jst, 0, 16 * sizeof(unsigned), st));
  // one cooperative launch: as many blocks as can be resident at once, at most one per pair
  int dev = 0, nsm = 0, per_sm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_svd, 256, 0));
  int blocks = std::max(1, std::min(R / 2, std::max(1, per_sm) * nsm));
  // one round between barriers takes microseconds: the wait limit, at least the 2 s default
  unsigned long long limit = std::max(P.wait.hard_ns, 2000000000ull);
  void* args[] = {&At, &Vt, &R, &tol, &max_sweeps, &jst, &status, &limit};
  ++g_launches;
  CK(cudaLaunchCooperativeKernel((const void*)k_jacobi_svd, dim3(blocks), dim3(256), args, 0, st));
  unsigned h[16];
  CK(cudaMemcpyAsync(h, jst, sizeof(h), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h[12] & ST_TIMEOUT) return fail(P, KAFMM_ERR_TIMEOUT, "Jacobi SVD: a grid barrier timed out");
  const int sweeps = (int)h[6];
  float last = 0.f;
  memcpy(&last, &h[3 + (sweeps + 2) % 3], sizeof(float));   // the last sweep's slot
  if (sweeps >= max_sweeps && h[(sweeps + 2) % 3] && last > 1e-11f)
    return fail(P, KAFMM_ERR_CUDA, "Jacobi SVD did not converge (off-orthogonality %.3g)", last);
  KL k_row_norms<<<R, 256, 0, st>>>(At, R, w);
  KL k_pinv_weights<<<1, 256, 0, st>>>(w, R, P.fp64() ? PINV_RCOND_FP64 : PINV_RCOND_FP32);
  // rows of At are the columns of W = K V; pinv = V diag(w) W^T
  KL k_scale_rows<<<512, 256, 0, st>>>(At, w, R, out1);
  KL k_transpose<<<512, 256, 0, st>>>(Vt, R, out2);
  CK(cudaGetLastError());
  if (w_host) {   // the weights 1 / sigma_k^2 of the kept singular values (0: dropped)
    w_host->resize(R);
    CK(cudaMemcpyAsync(w_host->data(), w, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  return 0;
}

// The operators of the compressed coordinates (see Plan::cmp) from the dense FP64 operators O
// and the kept singular values (w = 1 / sigma^2, 0 where dropped) of the two pseudo-inverses.
// Row k of the factor S^+ U^T is u_k^T / sigma_k and column k of V is v_k, so the projection
// rows are u_k^T = sigma_k (S^+ U^T)_k and the decompression columns v_k / sigma_k.
static int build_compressed(Plan& P, const double* O, const std::vector<double>& w_up,
                            const std::vector<double>& w_dn) {
  cudaStream_t st = P.stream;
  const int R = P.R;
  const size_t RR = (size_t)R * R;
  std::vector<int> idx[2];
  std::vector<double> sig[2], isig[2];
  for (int h = 0; h < 2; ++h) {
    const std::vector<double>& w = h == 0 ? w_up : w_dn;
    for (int k = 0; k < R; ++k)
      if (w[k] > 0) {
        idx[h].push_back(k);
        sig[h].push_back(1.0 / std::sqrt(w[k]));
        isig[h].push_back(std::sqrt(w[k]));
      }
  }
  // compress option 2: when rounding the larger rank down to a multiple of 64 keeps at least
  // 90 % of it, keep only that many leading singular vectors (largest sigma) on both sides, so no
  // row or k-value of the tensor-core tiles is padding
  if (P.compress_opt == 2) {
    const int rmax = (int)std::max(idx[0].size(), idx[1].size());
    const int rdown = rmax / 64 * 64;
    if (rdown >= 64 && 10 * rdown >= 9 * rmax)
      for (int h = 0; h < 2; ++h) {
        std::vector<int> ord(idx[h].size());
        for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
        std::sort(ord.begin(), ord.end(), [&](int a, int b) { return sig[h][a] > sig[h][b]; });
        ord.resize(std::min<size_t>(ord.size(), (size_t)rdown));
        std::vector<int> i2;
        std::vector<double> s2, is2;
        for (int o : ord) {
          i2.push_back(idx[h][o]);
          s2.push_back(sig[h][o]);
          is2.push_back(isig[h][o]);
        }
        idx[h] = i2;
        sig[h] = s2;
        isig[h] = is2;
      }
  }
  const int ru = (int)idx[0].size(), rd = (int)idx[1].size();
  const int rp = std::max(64, (std::max(ru, rd) + 63) / 64 * 64);
  if (rp >= P.Rpad) return 0;   // nothing to gain: keep the dense coordinates
  const size_t rr = (size_t)rp * rp, rR = (size_t)rp * R;
  DevBuf d_idx, d_sc, cin, cout, cops, X, Xb;
  CK(d_idx.reserve(sizeof(int) * 2 * R));
  CK(d_sc.reserve(sizeof(double) * 4 * R));
  CK(cin.reserve(sizeof(double) * 2 * rR));     // U_u^T, U_d^T  [rp][R] each
  CK(cout.reserve(sizeof(double) * 2 * rR));    // V_u S_u^+, V_d S_d^+  [R][rp] each
  CK(cops.reserve(sizeof(double) * rr * (N_M2L + N_CAUX)));
  CK(X.reserve(sizeof(double) * rR));
  int* di = d_idx.as<int>();
  double* ds = d_sc.as<double>();
  for (int h = 0; h < 2; ++h) {
    const int r = h == 0 ? ru : rd;
    CK(cudaMemcpyAsync(di + h * R, idx[h].data(), sizeof(int) * r, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ds + (2 * h) * R, sig[h].data(), sizeof(double) * r, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ds + (2 * h + 1) * R, isig[h].data(), sizeof(double) * r, cudaMemcpyHostToDevice, st));
    const double* f1 = O + RR * (h == 0 ? OP_UP1 : OP_DN1);
    const double* f2 = O + RR * (h == 0 ? OP_UP2 : OP_DN2);
    KL k_select_rows<<<1024, 256, 0, st>>>(f1, R, di + h * R, ds + (2 * h) * R, r, rp, cin.as<double>() + h * rR);
    KL k_select_cols<<<1024, 256, 0, st>>>(f2, R, di + h * R, ds + (2 * h + 1) * R, r, rp,
                                           cout.as<double>() + h * rR);
  }
  const double* PuT = cin.as<double>();
  const double* PdT = PuT + rR;
  // dst (rp x rp) = A^T T B with A^T, B^T given as [rp][R] projection rows
  auto sandwich = [&](const double* T, const double* AT, const double* BT, double* dst) {
    KL k_gemm64g<<<dim3((rp + 31) / 32, (R + 31) / 32), 256, 0, st>>>(T, R, 0, BT, R, 1, X.as<double>(), rp,
                                                                      R, rp, R, 1.0);
    KL k_gemm64g<<<dim3((rp + 31) / 32, (rp + 31) / 32), 256, 0, st>>>(AT, R, 0, X.as<double>(), rp, 0,
                                                                       dst, rp, rp, rp, R, 1.0);
  };
  double* C = cops.as<double>();
  {   // the M->L operators in batches (the near offsets are zero and stay zero): X_z = T_z Pu,
      // C_z = Pd^T X_z, one pair of launches per batch
    const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(N_M2L, (int64_t)(1.0e9 / (8.0 * R * rp))));
    CK(Xb.reserve(sizeof(double) * (size_t)chunk * R * rp));
    for (int o0 = 0; o0 < N_M2L; o0 += chunk) {
      const int nbt = std::min(chunk, N_M2L - o0);
      KL k_gemm64g<<<dim3((rp + 31) / 32, (R + 31) / 32, nbt), 256, 0, st>>>(
          O + RR * (OP_M2L + o0), R, 0, PuT, R, 1, Xb.as<double>(), rp, R, rp, R, 1.0, RR, 0, (int64_t)R * rp);
      KL k_gemm64g<<<dim3((rp + 31) / 32, (rp + 31) / 32, nbt), 256, 0, st>>>(
          PdT, R, 0, Xb.as<double>(), rp, 0, C + rr * o0, rp, rp, rp, R, 1.0, 0, (int64_t)R * rp, rr);
    }
  }
  double* CA = C + rr * N_M2L;
  for (int c = 0; c < 8; ++c) {
    sandwich(O + RR * (OP_M2M + c), PuT, PuT, CA + rr * c);
    sandwich(O + RR * (OP_L2L + c), PdT, PdT, CA + rr * (8 + c));
  }
  sandwich(O + RR * OP_PER, PdT, PuT, CA + rr * CAUX_PER);
  CK(cudaGetLastError());
  // split format: the plan's when chosen; the automatic choice takes BF16x3 up to 512
  // compressed rows for p >= 10 and up to 256 rows for p = 8, 9, else TF32x3.  Measured: 512
  // Stokeslet problems at p = 8 (four-channel table, 192 rows) 6.2e-6 worst problem against the
  // FP64 form with BF16x3 (3.4e-6 TF32x3) at 0.58x the M->L time; the periodic G table at p = 8
  // (512 rows) 1.4e-5 against the FP32 form with BF16x3; the G table at p = 12 (640 rows) 2.6e-5
  // against the Ewald sum on 2^22 periodic points with BF16x3, TF32x3 below 1e-5; below p = 8
  // the ranks are small and TF32x3 costs little
  P.tc_split_cm = P.tc_split;
  if (P.tc_split_opt == KAFMM_TC_AUTO) {
    const bool bf16 = (P.p >= 10 && rp <= 512) || (P.p >= 8 && rp <= 256);
    P.tc_split_cm = bf16 ? SPLIT_BF16 : SPLIT_TF32;
  }
  if (P.tc_split_cm == SPLIT_TF32) {
    CK(P.opstc_cm2l.reserve(sizeof(float) * 2 * rr * N_M2L));
    KL k_split_tf32<<<2048, 256, 0, st>>>(C, rp, rp, rp, rp, N_M2L, P.opstc_cm2l.as<float>());
  } else {
    CK(P.opstc_cm2l.reserve(sizeof(__nv_bfloat16) * 2 * rr * N_M2L));
    KL k_split_bf16<<<2048, 256, 0, st>>>(C, rp, rp, rp, rp, N_M2L, P.opstc_cm2l.as<__nv_bfloat16>());
  }
  CK(P.opstc_caux.reserve(sizeof(float) * 2 * rr * N_CAUX));
  KL k_split_tf32<<<2048, 256, 0, st>>>(CA, rp, rp, rp, rp, N_CAUX, P.opstc_caux.as<float>());
  CK(P.opstc_cin.reserve(sizeof(float) * 2 * 2 * (size_t)rp * P.Rpad));
  KL k_split_tf32<<<2048, 256, 0, st>>>(cin.as<double>(), rp, R, R, P.Rpad, 2, P.opstc_cin.as<float>());
  CK(P.opstc_cout.reserve(sizeof(float) * 2 * 2 * rR));
  KL k_split_tf32<<<2048, 256, 0, st>>>(cout.as<double>(), R, rp, rp, rp, 2, P.opstc_cout.as<float>());
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));   // the temporaries are released on return
  P.rp = rp;
  P.r_up = ru;
  P.r_dn = rd;
  P.cmp = true;
  return 0;
}

int build_operators(Plan& P) {
  P.cmp = false;
  cudaStream_t st = P.stream;
  int n = P.n, R = P.R;
  std::vector<double> us = unit_surface(P.p);
  CK(P.unit64.reserve(sizeof(double) * us.size()));
  CK(P.unit32.reserve(sizeof(float) * us.size()));
  CK(cudaMemcpyAsync(P.unit64.p, us.data(), sizeof(double) * us.size(), cudaMemcpyHostToDevice, st));
  std::vector<float> uf(us.begin(), us.end());
  CK(cudaMemcpyAsync(P.unit32.p, uf.data(), sizeof(float) * uf.size(), cudaMemcpyHostToDevice, st));

  size_t RR = (size_t)R * R;
  DevBuf ops, scratch;
  CK(ops.reserve(sizeof(double) * RR * N_OPS));
  CK(scratch.reserve(sizeof(double) * (RR * 4 + R + 64)));   // the tail holds 16 status words
  double* O = ops.as<double>();
  double* K = scratch.as<double>();
  double* At = K + RR;
  double* Vt = At + RR;
  double* Tm = Vt + RR;
  double* w = Tm + RR;
  int* flag = (int*)(w + R + 8);
  const double* unit = P.unit64.as<double>();
  int g = 1024;
  int stokes = P.ml_stokes;
  // pseudo-inverses at half-width 1 (factored)
  KL k_fill_kernel_matrix<<<g, 256, 0, st>>>(unit, n, stokes, 0, 0, 0, ALPHA_UC, 0, 0, 0, ALPHA_UE, K);
  std::vector<double> w_up, w_dn;
  int rc = pinv64(P, K, O + RR * OP_UP1, O + RR * OP_UP2, At, Vt, w, flag, &w_up);
  if (rc) return rc;
  KL k_fill_kernel_matrix<<<g, 256, 0, st>>>(unit, n, stokes, 0, 0, 0, ALPHA_DC, 0, 0, 0, ALPHA_DE, K);
  rc = pinv64(P, K, O + RR * OP_DN1, O + RR * OP_DN2, At, Vt, w, flag, &w_dn);
  if (rc) return rc;
  dim3 gg((R + 31) / 32, (R + 31) / 32);
  // Op = alpha * (K * V) * (S^+ U^T): the product through the factors
  auto compose = [&](int f1, int f2, double alpha, double* dst) {
    KL k_gemm64<<<gg, 256, 0, st>>>(K, 0, nullptr, O + RR * f2, 1.0, R, Tm);
    KL k_gemm64<<<gg, 256, 0, st>>>(Tm, 0, nullptr, O + RR * f1, alpha, R, dst);
  };
  // M->L: centres 2 o apart (box side 2); the 27 near offsets are zero; the other 316 in
  // batches (kernel matrices of a batch filled by one launch, composed by two batched GEMMs)
  {
    std::vector<int> offs, dsti;
    for (int oz = -3; oz <= 3; ++oz)
      for (int oy = -3; oy <= 3; ++oy)
        for (int ox = -3; ox <= 3; ++ox) {
          const int idx = m2l_index(ox, oy, oz);
          if (abs(ox) <= 1 && abs(oy) <= 1 && abs(oz) <= 1) {
            CK(cudaMemsetAsync(O + RR * (OP_M2L + idx), 0, sizeof(double) * RR, st));
            continue;
          }
          offs.push_back(ox);
          offs.push_back(oy);
          offs.push_back(oz);
          dsti.push_back(OP_M2L + idx);
        }
    const int nall = (int)dsti.size();
    const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(nall, (int64_t)(1.0e9 / (16.0 * RR))));
    DevBuf kb, tb, tab;
    CK(kb.reserve(sizeof(double) * (size_t)chunk * RR));
    CK(tb.reserve(sizeof(double) * (size_t)chunk * RR));
    CK(tab.reserve(sizeof(int) * 4 * (size_t)nall));
    int* d_offs = tab.as<int>();
    int* d_dst = d_offs + 3 * nall;
    CK(cudaMemcpyAsync(d_offs, offs.data(), sizeof(int) * 3 * nall, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_dst, dsti.data(), sizeof(int) * nall, cudaMemcpyHostToDevice, st));
    for (int c0 = 0; c0 < nall; c0 += chunk) {
      const int nbt = std::min(chunk, nall - c0);
      KL k_fill_m2l_batch<<<dim3(g, 1, nbt), 256, 0, st>>>(unit, n, stokes, ALPHA_DC, ALPHA_UE, d_offs + 3 * c0,
                                                           kb.as<double>(), RR);
      // Op = (K V) (S^+ U^T), the compose() of one operator for every z of the batch
      dim3 gb(gg.x, gg.y, nbt);
      KL k_gemm64<<<gb, 256, 0, st>>>(kb.as<double>(), 0, nullptr, O + RR * OP_UP2, 1.0, R, tb.as<double>(), RR, RR,
                                    nullptr);
      KL k_gemm64<<<gb, 256, 0, st>>>(tb.as<double>(), 0, nullptr, O + RR * OP_UP1, 1.0, R, O, RR, RR, d_dst + c0);
    }
    CK(cudaStreamSynchronize(st));   // the batch buffers are released on leaving this scope
  }
  // M->M / L->L: child half-width 1, parent half-width 2, child centre at +-1 per axis
  for (int c = 0; c < 8; ++c) {
    double cx = (c & 1) ? 1.0 : -1.0, cy = (c & 2) ? 1.0 : -1.0, cz = (c & 4) ? 1.0 : -1.0;
    KL k_fill_kernel_matrix<<<g, 256, 0, st>>>(unit, n, stokes, 0, 0, 0, 2.0 * ALPHA_UC, cx, cy, cz,
                                            ALPHA_UE, K);
    // StokesPVel, check values stored as [h p, u]: the parent's p rows carry h = 2 (the
    // child's h = 1 cancels in its pseudo-inverse)
    if (stokes == 2) KL k_scale_every4<<<g, 256, 0, st>>>(K, R, 1, 0, 2.0);
    compose(OP_UP1, OP_UP2, 1.0, O + RR * (OP_M2M + c));
    KL k_fill_kernel_matrix<<<g, 256, 0, st>>>(unit, n, stokes, cx, cy, cz, ALPHA_DC, 0, 0, 0,
                                            2.0 * ALPHA_DE, K);
    // StokesPVel: the parent's equivalent q is its scaled q times h = 2
    if (stokes == 2) KL k_scale_every4<<<g, 256, 0, st>>>(K, R, 0, 3, 2.0);
    compose(OP_DN1, OP_DN2, 2.0, O + RR * (OP_L2L + c));
  }
  if (P.bc == KAFMM_BC_PXYZ) {  // root far images, composed with the upward pseudo-inverse
    KL k_periodic_operator<<<1024, 128, 0, st>>>(unit, n, stokes, ALPHA_DC, ALPHA_UE, K);
    compose(OP_UP1, OP_UP2, 1.0, O + RR * OP_PER);
  } else if (P.bc == KAFMM_BC_PX || P.bc == KAFMM_BC_PXY) {
    // images along a line: N = 16 ... 2048 (4097 images, extrapolated to rounding); over a
    // plane: N = 4 ... 128 (66049 images, about 1e-9)
    const int axes = P.bc == KAFMM_BC_PX ? 1 : 2;
    const int n0 = axes == 1 ? 16 : 4, nlev = axes == 1 ? 8 : 6;
    DevBuf part;
    CK(part.reserve(sizeof(double) * RR * nlev));
    KL k_lattice_partials<<<(int)(((int64_t)n * n + 127) / 128), 128, 0, st>>>(unit, n, stokes, ALPHA_DC,
                                                                               ALPHA_UE, axes, n0, nlev,
                                                                               part.as<double>());
    KL k_lattice_extrapolate<<<2048, 256, 0, st>>>(part.as<double>(), nlev, (int64_t)RR, K);
    KL k_project_neutral<<<R, 256, 0, st>>>(K, n, stokes ? 3 : 1);
    compose(OP_UP1, OP_UP2, 1.0, O + RR * OP_PER);
    CK(cudaStreamSynchronize(st));   // the partial sums are released on leaving this scope
  } else {
    CK(cudaMemsetAsync(O + RR * OP_PER, 0, sizeof(double) * RR, st));
  }
  CK(cudaGetLastError());
  if (P.fp64()) {
    CK(P.ops64.reserve(sizeof(double) * RR * N_OPS));
    CK(cudaMemcpyAsync(P.ops64.p, O, sizeof(double) * RR * N_OPS, cudaMemcpyDeviceToDevice, st));
  } else {
    CK(P.ops32.reserve(sizeof(float) * RR * N_OPS));
    KL k_round32<<<2048, 256, 0, st>>>(O, (int64_t)RR * N_OPS, P.ops32.as<float>());
    extern bool tc_table(const Plan& P);
    if (P.prec == KAFMM_PREC_MIXED && tc_table(P)) {
      P.Rpad = (R + 63) / 64 * 64;
      P.tmap_ready = false;
      if (P.tc_split == SPLIT_TF32) {
        CK(P.opstc.reserve(sizeof(float) * 2 * (size_t)R * P.Rpad * N_M2L));
        KL k_split_tf32<<<2048, 256, 0, st>>>(O + RR * OP_M2L, R, R, R, P.Rpad, N_M2L, P.opstc.as<float>());
      } else {
        CK(P.opstc.reserve(sizeof(__nv_bfloat16) * 2 * (size_t)R * P.Rpad * N_M2L));
        KL k_split_bf16<<<2048, 256, 0, st>>>(O + RR * OP_M2L, R, R, R, P.Rpad, N_M2L,
                                              P.opstc.as<__nv_bfloat16>());
      }
      // M->M, L->L and the pseudo-inverse factors: TF32 split (about FP32 accuracy)
      CK(P.opstc_aux.reserve(sizeof(float) * 2 * (size_t)R * P.Rpad * N_AUX));
      KL k_split_tf32<<<2048, 256, 0, st>>>(O + RR * OP_M2M, R, R, R, P.Rpad, N_AUX, P.opstc_aux.as<float>());
      P.cmp = false;
      if (P.compress_opt) {
        rc = build_compressed(P, O, w_up, w_dn);
        if (rc) return rc;
      }
    }
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  P.ops_ready = true;
  return 0;
}

}  // namespace kafmm
