/*
 * CPU ORACLE -- test infrastructure only.  Plain FP64 direct sums of the kernel functions of
 * Yan & Blackwell, "Kernel Aggregated Fast Multipole Method" (arXiv:2010.15155).
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load this code;
 * the CUDA evaluator never does.
 *
 * Every routine ACCUMULATES into g (g += sum over sources), loops over all target/source
 * pairs in the plainest order (targets outer, sources inner) and skips pairs with r^2 == 0
 * (the self pair when sources and targets are the same set; any other coincident pair
 * contributes nothing).  r = x - y (target minus source), viscosity mu = 1.
 * Row-major layouts: x[nt][3], y[ns][3], s[ns][k_s], g[nt][k_t].
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846

/* Threads of the OpenMP loops below (n > 0), for timing the sums on one core and on all of
 * them; returns the previous maximum. */
int orc_set_threads(int n) {
#ifdef _OPENMP
  int prev = omp_get_max_threads();
  if (n > 0) omp_set_num_threads(n);
  return prev;
#else
  (void)n;
  return 1;
#endif
}

/* Laplace single layer, Sec. II.A: L = 1/(4 pi r).  s: [q], g: [phi]. */
void orc_laplace(const double* x, int64_t nt, const double* y, int64_t ns,
                 const double* s, double* g) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t a = 0; a < nt; ++a) {
    double acc = 0.0;
    for (int64_t b = 0; b < ns; ++b) {
      double r0 = x[3 * a] - y[3 * b], r1 = x[3 * a + 1] - y[3 * b + 1],
             r2 = x[3 * a + 2] - y[3 * b + 2];
      double rr = r0 * r0 + r1 * r1 + r2 * r2;
      if (rr == 0.0) continue;
      acc += s[b] / (4.0 * PI * sqrt(rr));
    }
    g[a] += acc;
  }
}

/* Laplace charges -> [phi, grad phi (3), grad grad phi (6: xx xy xz yy yz zz)], the
 * combined kernel L + grad L + grad grad L of Table tab:ktab_lapqdpgradgrad.
 * d/dx_i (1/r) = -r_i/r^3 ; d2/dx_i dx_j (1/r) = (3 r_i r_j - delta_ij r^2)/r^5.  g: 10 cols. */
void orc_laplace_pgradgrad(const double* x, int64_t nt, const double* y, int64_t ns,
                           const double* s, double* g) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t a = 0; a < nt; ++a) {
    double acc[10] = {0};
    for (int64_t b = 0; b < ns; ++b) {
      double r[3] = {x[3 * a] - y[3 * b], x[3 * a + 1] - y[3 * b + 1],
                     x[3 * a + 2] - y[3 * b + 2]};
      double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      if (rr == 0.0) continue;
      double rn = sqrt(rr), q = s[b] / (4.0 * PI);
      double r3 = rr * rn, r5 = r3 * rr;
      acc[0] += q / rn;
      for (int i = 0; i < 3; ++i) acc[1 + i] += -q * r[i] / r3;
      int c = 4;
      for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
          double h = 3.0 * r[i] * r[j] / r5 - (i == j ? 1.0 / r3 : 0.0);
          acc[c++] += q * h;
        }
    }
    for (int k = 0; k < 10; ++k) g[10 * a + k] += acc[k];
  }
}

/* Laplace dipole potential, Sec. II.A: phi = L^D_j d_j with L^D_j = -dL/dx_j = r_j/(4 pi r^3).
 * s: [d1 d2 d3], g: [phi]. */
void orc_laplace_dipole(const double* x, int64_t nt, const double* y, int64_t ns,
                        const double* s, double* g) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t a = 0; a < nt; ++a) {
    double acc = 0.0;
    for (int64_t b = 0; b < ns; ++b) {
      double r0 = x[3 * a] - y[3 * b], r1 = x[3 * a + 1] - y[3 * b + 1],
             r2 = x[3 * a + 2] - y[3 * b + 2];
      double rr = r0 * r0 + r1 * r1 + r2 * r2;
      if (rr == 0.0) continue;
      double rn = sqrt(rr);
      acc += (r0 * s[3 * b] + r1 * s[3 * b + 1] + r2 * s[3 * b + 2]) / (4.0 * PI * rr * rn);
    }
    g[a] += acc;
  }
}

/* Charges and dipoles to potential, gradient and Hessian, Sec. II.A (Table
 * tab:ktab_lapqdpgradgrad): phi = L q + L^D_j d_j with L^D_j = -dL/dx_j, so with r = x - y
 *   4 pi phi         = q / r + (d.r) / r^3,
 *   4 pi d_i phi     = -q r_i / r^3 + d_i / r^3 - 3 (d.r) r_i / r^5,
 *   4 pi d_i d_j phi = q (3 r_i r_j - delta_ij r^2) / r^5
 *                      - 3 (d_i r_j + d_j r_i + (d.r) delta_ij) / r^5 + 15 (d.r) r_i r_j / r^7.
 * s: [q d1 d2 d3] (4), g: [phi, grad (3), Hessian xx xy xz yy yz zz (6)] (10). */
void orc_laplace_qd(const double* x, int64_t nt, const double* y, int64_t ns,
                    const double* s, double* g) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t a = 0; a < nt; ++a) {
    double acc[10] = {0};
    for (int64_t b = 0; b < ns; ++b) {
      double r[3] = {x[3 * a] - y[3 * b], x[3 * a + 1] - y[3 * b + 1],
                     x[3 * a + 2] - y[3 * b + 2]};
      double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      if (rr == 0.0) continue;
      const double* v = s + 4 * b;
      double q = v[0], d[3] = {v[1], v[2], v[3]};
      double rn = sqrt(rr), r3 = rr * rn, r5 = r3 * rr, r7 = r5 * rr;
      double dr = d[0] * r[0] + d[1] * r[1] + d[2] * r[2];
      acc[0] += (q / rn + dr / r3) / (4.0 * PI);
      for (int i = 0; i < 3; ++i)
        acc[1 + i] += (-q * r[i] / r3 + d[i] / r3 - 3.0 * dr * r[i] / r5) / (4.0 * PI);
      int c = 4;
      for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
          double dij = i == j ? 1.0 : 0.0;
          double h = q * (3.0 * r[i] * r[j] - dij * rr) / r5 -
                     3.0 * (d[i] * r[j] + d[j] * r[i] + dr * dij) / r5 + 15.0 * dr * r[i] * r[j] / r7;
          acc[c++] += h / (4.0 * PI);
        }
    }
    for (int k = 0; k < 10; ++k) g[10 * a + k] += acc[k];
  }
}

/* Laplace quadrupoles to potential, gradient and Hessian (LapQPGradGrad of Table
 * tab:implement; the phi^Q sum of Table tab:rpywall): phi = Q_jk d_j d_k L, L = 1/(4 pi r),
 * derivatives in x, r = x - y.  With the derivatives of 1/r
 *   D2_jk   = (3 r_j r_k - delta_jk r^2) / r^5,
 *   D3_ijk  = -15 r_i r_j r_k / r^7 + 3 (delta_ij r_k + delta_ik r_j + delta_jk r_i) / r^5,
 *   D4_ijkl = 105 r_i r_j r_k r_l / r^9 - 15 (delta_ij r_k r_l + delta_ik r_j r_l + delta_il r_j r_k
 *             + delta_jk r_i r_l + delta_jl r_i r_k + delta_kl r_i r_j) / r^7
 *             + 3 (delta_ij delta_kl + delta_ik delta_jl + delta_il delta_jk) / r^5,
 * 4 pi phi = Q_jk D2_jk, 4 pi d_i phi = Q_jk D3_ijk, 4 pi d_i d_l phi = Q_jk D4_iljk.
 * s: Q row-major (Q_jk at 3j+k, 9), g: [phi, grad (3), Hessian xx xy xz yy yz zz (6)] (10). */
void orc_laplace_quad(const double* x, int64_t nt, const double* y, int64_t ns,
                      const double* s, double* g) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t a = 0; a < nt; ++a) {
    double acc[10] = {0};
    for (int64_t b = 0; b < ns; ++b) {
      double r[3] = {x[3 * a] - y[3 * b], x[3 * a + 1] - y[3 * b + 1],
                     x[3 * a + 2] - y[3 * b + 2]};
      double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      if (rr == 0.0) continue;
      const double* Q = s + 9 * b;
      double rn = sqrt(rr), r5 = rr * rr * rn, r7 = r5 * rr, r9 = r7 * rr;
      double phi = 0.0, gr[3] = {0, 0, 0}, H[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
          double q = Q[3 * j + k];
          if (q == 0.0) continue;
          double djk = j == k ? 1.0 : 0.0;
          phi += q * (3.0 * r[j] * r[k] - djk * rr) / r5;
          for (int i = 0; i < 3; ++i) {
            double dij = i == j ? 1.0 : 0.0, dik = i == k ? 1.0 : 0.0;
            gr[i] += q * (-15.0 * r[i] * r[j] * r[k] / r7 + 3.0 * (dij * r[k] + dik * r[j] + djk * r[i]) / r5);
            for (int l = 0; l < 3; ++l) {
              double dil = i == l ? 1.0 : 0.0, djl = j == l ? 1.0 : 0.0, dkl = k == l ? 1.0 : 0.0;
              H[i][l] += q * (105.0 * r[i] * r[j] * r[k] * r[l] / r9 -
                              15.0 * (dij * r[k] * r[l] + dik * r[j] * r[l] + dil * r[j] * r[k] +
                                      djk * r[i] * r[l] + djl * r[i] * r[k] + dkl * r[i] * r[j]) / r7 +
                              3.0 * (dij * dkl + dik * djl + dil * djk) / r5);
            }
          }
        }
      acc[0] += phi / (4.0 * PI);
      for (int i = 0; i < 3; ++i) acc[1 + i] += gr[i] / (4.0 * PI);
      int c = 4;
      for (int i = 0; i < 3; ++i)
        for (int l = i; l < 3; ++l) acc[c++] += H[i][l] / (4.0 * PI);
    }
    for (int k = 0; k < 10; ++k) g[10 * a + k] += acc[k];
  }
}

/* Stokeslet, Sec. II.B: G_ij = (delta_ij / r + r_i r_j / r^3) / (8 pi).  s: f (3), g: u (3). */
void orc_stokeslet(const double* x, int64_t nt, const double* y, int64_t ns,
                   const double* s, double* g) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t a = 0; a < nt; ++a) {
    double u[3] = {0, 0, 0};
    for (int64_t b = 0; b < ns; ++b) {
      double r[3] = {x[3 * a] - y[3 * b], x[3 * a + 1] - y[3 * b + 1],
                     x[3 * a + 2] - y[3 * b + 2]};
      double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      if (rr == 0.0) continue;
      double rn = sqrt(rr);
      const double* f = s + 3 * b;
      double rf = r[0] * f[0] + r[1] * f[1] + r[2] * f[2];
      for (int i = 0; i < 3; ++i)
        u[i] += (f[i] / rn + r[i] * rf / (rr * rn)) / (8.0 * PI);
    }
    for (int i = 0; i < 3; ++i) g[3 * a + i] += u[i];
  }
}

/* StokesPVel, Sec. II.C (Eqs. stkslp, stkslvel): [p, u] = G^P [f, q],
 *   p = r.f / (4 pi r^3),  u_i = (delta_ij / r + r_i r_j / r^3) f_j / (8 pi) - r_i q / (8 pi r^3),
 * q twice the fluid removed (a sink for q > 0).  s: [f1 f2 f3 q] (4), g: [p, u] (4). */
void orc_stokes_pvel(const double* x, int64_t nt, const double* y, int64_t ns,
                     const double* s, double* g) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t a = 0; a < nt; ++a) {
    double acc[4] = {0, 0, 0, 0};
    for (int64_t b = 0; b < ns; ++b) {
      double r[3] = {x[3 * a] - y[3 * b], x[3 * a + 1] - y[3 * b + 1],
                     x[3 * a + 2] - y[3 * b + 2]};
      double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      if (rr == 0.0) continue;
      const double* v = s + 4 * b;
      double rn = sqrt(rr), r3 = rr * rn;
      double rf = r[0] * v[0] + r[1] * v[1] + r[2] * v[2];
      acc[0] += rf / (4.0 * PI * r3);
      for (int i = 0; i < 3; ++i)
        acc[1 + i] += (v[i] / rn + r[i] * rf / r3 - r[i] * v[3] / r3) / (8.0 * PI);
    }
    for (int k = 0; k < 4; ++k) g[4 * a + k] += acc[k];
  }
}

/* Regularized Stokeslet, Sec. II.B (Table tab:ktab_reg): the flow of the force f spread by
 * the blob psi(r) = 15 eps^4 / (8 pi (r^2 + eps^2)^{7/2}) around the source,
 *   G^eps_ij = [ (r^2 + 2 eps^2) delta_ij + r_i r_j ] / (8 pi (r^2 + eps^2)^{3/2}),
 * eps per source.  s: [f1 f2 f3 eps] (4), g: u (3).  eps = 0 gives the Stokeslet. */
void orc_stokeslet_reg(const double* x, int64_t nt, const double* y, int64_t ns,
                       const double* s, double* g) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t a = 0; a < nt; ++a) {
    double u[3] = {0, 0, 0};
    for (int64_t b = 0; b < ns; ++b) {
      double r[3] = {x[3 * a] - y[3 * b], x[3 * a + 1] - y[3 * b + 1],
                     x[3 * a + 2] - y[3 * b + 2]};
      double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      if (rr == 0.0) continue;
      const double* f = s + 4 * b;
      double ee = f[3] * f[3];
      double d = rr + ee, d3 = d * sqrt(d);
      double rf = r[0] * f[0] + r[1] * f[1] + r[2] * f[2];
      for (int i = 0; i < 3; ++i) u[i] += ((rr + 2.0 * ee) * f[i] + r[i] * rf) / (8.0 * PI * d3);
    }
    for (int i = 0; i < 3; ++i) g[3 * a + i] += u[i];
  }
}

/* RPY flow field and its Laplacian, Eqs. RPYflow/RPYkernel and Table tab:ktab_rpy:
 *   u = G f + (b^2/6) lap(G) f,   lap(u) = lap(G) f   (lap lap G = 0),
 *   lap(G)_ij = (delta_ij / r^3 - 3 r_i r_j / r^5) / (4 pi).
 * s: [f1 f2 f3 b] (4), g: [u (3), lap u (3)] (6).  With b = 0 this is G + lap G. */
void orc_rpy(const double* x, int64_t nt, const double* y, int64_t ns,
             const double* s, double* g) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t a = 0; a < nt; ++a) {
    double u[3] = {0, 0, 0}, lu[3] = {0, 0, 0};
    for (int64_t b = 0; b < ns; ++b) {
      double r[3] = {x[3 * a] - y[3 * b], x[3 * a + 1] - y[3 * b + 1],
                     x[3 * a + 2] - y[3 * b + 2]};
      double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      if (rr == 0.0) continue;
      double rn = sqrt(rr), r3 = rr * rn, r5 = r3 * rr;
      const double* f = s + 4 * b;
      double bb = f[3] * f[3];
      double rf = r[0] * f[0] + r[1] * f[1] + r[2] * f[2];
      for (int i = 0; i < 3; ++i) {
        double gf = (f[i] / rn + r[i] * rf / r3) / (8.0 * PI);
        double lgf = (f[i] / r3 - 3.0 * r[i] * rf / r5) / (4.0 * PI);
        u[i] += gf + bb / 6.0 * lgf;
        lu[i] += lgf;
      }
    }
    for (int i = 0; i < 3; ++i) {
      g[6 * a + i] += u[i];
      g[6 * a + 3 + i] += lu[i];
    }
  }
}

/* Stokes double layer, Eqs. stkdlp / stkdlvel:
 *   p   = (1/4pi) (-3 r_j r_k / r^5 + delta_jk / r^3) D_jk,
 *   u_i = -(3/8pi) r_i r_j r_k D_jk / r^5.
 * s: D flattened row-major (D_jk at 3j+k, 9), g: [p, u1, u2, u3] (4). */
void orc_stokes_dl(const double* x, int64_t nt, const double* y, int64_t ns,
                   const double* s, double* g) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t a = 0; a < nt; ++a) {
    double acc[4] = {0, 0, 0, 0};
    for (int64_t b = 0; b < ns; ++b) {
      double r[3] = {x[3 * a] - y[3 * b], x[3 * a + 1] - y[3 * b + 1],
                     x[3 * a + 2] - y[3 * b + 2]};
      double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      if (rr == 0.0) continue;
      double rn = sqrt(rr), r3 = rr * rn, r5 = r3 * rr;
      const double* D = s + 9 * b;
      double rDr = 0.0, tr = D[0] + D[4] + D[8];
      for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) rDr += r[j] * D[3 * j + k] * r[k];
      acc[0] += (-3.0 * rDr / r5 + tr / r3) / (4.0 * PI);
      for (int i = 0; i < 3; ++i) acc[1 + i] += -3.0 / (8.0 * PI) * r[i] * rDr / r5;
    }
    for (int k = 0; k < 4; ++k) g[4 * a + k] += acc[k];
  }
}

/* ---------------------------------------------------------------------------------------
 * Derivatives of the StokesPVel and double-layer fields at the targets (the T column of
 * Tables tab:ktab_stkslpvelgrad and tab:ktab_stkdlpvelgrad; target values of PVelGrad,
 * PVelLaplacian and Traction in Table tab:implement).  Layouts of the target values:
 *   grad:      [p, u_1..3, d p / d x_1..3, d u_i / d x_j at 7 + 3 i + j]          (16)
 *   laplacian: [p, u_1..3, lap u_1..3]                                             (7)
 *   traction:  sigma_ij = -p delta_ij + d u_i / d x_j + d u_j / d x_i at 3 i + j   (9)
 * (Eq. stressdef with mu = 1). */

/* One StokesPVel pair (Eqs. stkslp, stkslvel differentiated in x), r = x - y, v = [f, q]:
 *   4 pi d_j p   = f_j / r^3 - 3 (r.f) r_j / r^5,
 *   8 pi d_j u_i = [delta_ij (r.f) + r_i f_j - f_i r_j - q delta_ij] / r^3
 *                  + 3 r_i r_j (q - r.f) / r^5. */
static void pvel_pair_grad(const double r[3], const double* v, double* o) {
  double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  double rn = sqrt(rr), r3 = rr * rn, r5 = r3 * rr;
  double rf = r[0] * v[0] + r[1] * v[1] + r[2] * v[2], q = v[3];
  o[0] = rf / (4.0 * PI * r3);
  for (int i = 0; i < 3; ++i) o[1 + i] = (v[i] / rn + r[i] * rf / r3 - r[i] * q / r3) / (8.0 * PI);
  for (int j = 0; j < 3; ++j) o[4 + j] = (v[j] / r3 - 3.0 * rf * r[j] / r5) / (4.0 * PI);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double dij = i == j ? 1.0 : 0.0;
      o[7 + 3 * i + j] = ((dij * rf + r[i] * v[j] - v[i] * r[j] - q * dij) / r3 +
                          3.0 * r[i] * r[j] * (q - rf) / r5) / (8.0 * PI);
    }
}

/* One double-layer pair (Eqs. stkdlp, stkdlvel differentiated in x), D_jk at 3 j + k, with
 * rDr = r_j D_jk r_k, a_j = d(rDr)/d r_j = D_jk r_k + r_k D_kj, t = tr D:
 *   4 pi d_j p   = -3 a_j / r^5 + 15 rDr r_j / r^7 - 3 t r_j / r^5,
 *   8 pi d_j u_i = -3 [delta_ij rDr / r^5 + r_i a_j / r^5 - 5 r_i r_j rDr / r^7]. */
static void dl_pair_grad(const double r[3], const double* D, double* o) {
  double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  double rn = sqrt(rr), r3 = rr * rn, r5 = r3 * rr, r7 = r5 * rr;
  double rDr = 0.0, t = D[0] + D[4] + D[8], a[3];
  for (int j = 0; j < 3; ++j) {
    a[j] = 0.0;
    for (int k = 0; k < 3; ++k) {
      rDr += r[j] * D[3 * j + k] * r[k];
      a[j] += D[3 * j + k] * r[k] + r[k] * D[3 * k + j];
    }
  }
  o[0] = (-3.0 * rDr / r5 + t / r3) / (4.0 * PI);
  for (int i = 0; i < 3; ++i) o[1 + i] = -3.0 / (8.0 * PI) * r[i] * rDr / r5;
  for (int j = 0; j < 3; ++j) o[4 + j] = (-3.0 * a[j] / r5 + 15.0 * rDr * r[j] / r7 - 3.0 * t * r[j] / r5) / (4.0 * PI);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      o[7 + 3 * i + j] = -3.0 / (8.0 * PI) *
                         ((i == j ? rDr / r5 : 0.0) + r[i] * a[j] / r5 - 5.0 * r[i] * r[j] * rDr / r7);
}

/* Laplacian of the velocity, worked out from the velocities themselves (not from the pressure):
 * StokesPVel: the source term -q r / r^3 is a gradient of 1/r (harmonic away from the source),
 * and lap (f / r + r (r.f) / r^3) = 2 f / r^3 - 6 r (r.f) / r^5, so
 *   8 pi lap u_i = 2 f_i / r^3 - 6 r_i (r.f) / r^5;
 * double layer: lap (r_i rDr / r^5) = 2 a_i / r^5 + 2 t r_i / r^5 - 10 r_i rDr / r^7, so
 *   8 pi lap u_i = -3 [2 a_i / r^5 + 2 t r_i / r^5 - 10 r_i rDr / r^7]. */
static void pvel_pair_lapl(const double r[3], const double* v, double* o) {
  double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  double rn = sqrt(rr), r3 = rr * rn, r5 = r3 * rr;
  double rf = r[0] * v[0] + r[1] * v[1] + r[2] * v[2], q = v[3];
  o[0] = rf / (4.0 * PI * r3);
  for (int i = 0; i < 3; ++i) {
    o[1 + i] = (v[i] / rn + r[i] * rf / r3 - r[i] * q / r3) / (8.0 * PI);
    o[4 + i] = (2.0 * v[i] / r3 - 6.0 * r[i] * rf / r5) / (8.0 * PI);
  }
}

static void dl_pair_lapl(const double r[3], const double* D, double* o) {
  double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  double rn = sqrt(rr), r3 = rr * rn, r5 = r3 * rr, r7 = r5 * rr;
  double rDr = 0.0, t = D[0] + D[4] + D[8], a[3];
  for (int j = 0; j < 3; ++j) {
    a[j] = 0.0;
    for (int k = 0; k < 3; ++k) {
      rDr += r[j] * D[3 * j + k] * r[k];
      a[j] += D[3 * j + k] * r[k] + r[k] * D[3 * k + j];
    }
  }
  o[0] = (-3.0 * rDr / r5 + t / r3) / (4.0 * PI);
  for (int i = 0; i < 3; ++i) {
    o[1 + i] = -3.0 / (8.0 * PI) * r[i] * rDr / r5;
    o[4 + i] = -3.0 / (8.0 * PI) * (2.0 * a[i] / r5 + 2.0 * t * r[i] / r5 - 10.0 * r[i] * rDr / r7);
  }
}

/* Shared loop of the derivative kernels: mode 0 grad (16), 1 laplacian (7), 2 traction (9);
 * dl selects the double-layer sources (9 per source) over [f, q] (4). */
static void deriv_sum(int dl, int mode, const double* x, int64_t nt, const double* y, int64_t ns,
                      const double* s, double* g) {
  const int ks = dl ? 9 : 4, kt = mode == 0 ? 16 : (mode == 1 ? 7 : 9);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t a = 0; a < nt; ++a) {
    double acc[16] = {0};
    for (int64_t b = 0; b < ns; ++b) {
      double r[3] = {x[3 * a] - y[3 * b], x[3 * a + 1] - y[3 * b + 1], x[3 * a + 2] - y[3 * b + 2]};
      if (r[0] * r[0] + r[1] * r[1] + r[2] * r[2] == 0.0) continue;
      double o[16];
      const double* v = s + ks * b;
      if (mode == 1) {
        if (dl) dl_pair_lapl(r, v, o);
        else pvel_pair_lapl(r, v, o);
        for (int k = 0; k < 7; ++k) acc[k] += o[k];
      } else {
        if (dl) dl_pair_grad(r, v, o);
        else pvel_pair_grad(r, v, o);
        if (mode == 0) {
          for (int k = 0; k < 16; ++k) acc[k] += o[k];
        } else {
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
              acc[3 * i + j] += (i == j ? -o[0] : 0.0) + o[7 + 3 * i + j] + o[7 + 3 * j + i];
        }
      }
    }
    for (int k = 0; k < kt; ++k) g[kt * a + k] += acc[k];
  }
}

void orc_stokes_pvel_grad(const double* x, int64_t nt, const double* y, int64_t ns, const double* s, double* g) {
  deriv_sum(0, 0, x, nt, y, ns, s, g);
}
void orc_stokes_pvel_lapl(const double* x, int64_t nt, const double* y, int64_t ns, const double* s, double* g) {
  deriv_sum(0, 1, x, nt, y, ns, s, g);
}
void orc_stokes_pvel_traction(const double* x, int64_t nt, const double* y, int64_t ns, const double* s,
                              double* g) {
  deriv_sum(0, 2, x, nt, y, ns, s, g);
}
void orc_stokes_dl_grad(const double* x, int64_t nt, const double* y, int64_t ns, const double* s, double* g) {
  deriv_sum(1, 0, x, nt, y, ns, s, g);
}
void orc_stokes_dl_lapl(const double* x, int64_t nt, const double* y, int64_t ns, const double* s, double* g) {
  deriv_sum(1, 1, x, nt, y, ns, s, g);
}
void orc_stokes_dl_traction(const double* x, int64_t nt, const double* y, int64_t ns, const double* s,
                            double* g) {
  deriv_sum(1, 2, x, nt, y, ns, s, g);
}

/* Pair mobility of two spheres (radii ai at the target, aj at the source), r = x - y.
 * Far form (r > ai + aj): the assembled RPY tensor of Eqs. RPYkernel/RPYtrgvel,
 *   M = G + (ai^2 + aj^2)/6 lap G.
 * Overlapping spheres (r <= ai + aj), which the paper defers to a post-processing pass
 * (Sec. II.B, citing Zuk et al. 2014) -- the unequal-radius regularisation:
 *   |ai-aj| < r <= ai+aj : M = [A I + B rhat rhat] / (6 pi ai aj),
 *        A = (16 r^3 (ai+aj) - ((ai-aj)^2 + 3 r^2)^2) / (32 r^3),
 *        B = 3 ((ai-aj)^2 - r^2)^2 / (32 r^3);
 *   r <= |ai-aj|         : M = I / (6 pi max(ai, aj)).
 * Writes the 3x3 tensor (row-major) into m.  r == 0 with ai == aj gives I/(6 pi a). */
static void rpy_pair_tensor(const double r[3], double ai, double aj, double m[9]) {
  double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  double rn = sqrt(rr);
  double d = fabs(ai - aj), s = ai + aj;
  double A, B;
  if (rn > s) {
    double c = (ai * ai + aj * aj);
    A = (1.0 + c / (3.0 * rr)) / (8.0 * PI * rn);
    B = (1.0 - c / rr) / (8.0 * PI * rn);
  } else if (rn > d) {
    double r3 = rr * rn, t = d * d + 3.0 * rr, e = d * d - rr;
    A = (16.0 * r3 * s - t * t) / (32.0 * r3) / (6.0 * PI * ai * aj);
    B = 3.0 * e * e / (32.0 * r3) / (6.0 * PI * ai * aj);
  } else {
    A = 1.0 / (6.0 * PI * (ai > aj ? ai : aj));
    B = 0.0;
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double rh = rn > 0.0 ? r[i] * r[j] / rr : 0.0;
      m[3 * i + j] = (i == j ? A : 0.0) + B * rh;
    }
}

/* 3x3 pair mobility for a single pair (exposed for the pins). */
void orc_rpy_pair(const double* r, double ai, double aj, double* m) { rpy_pair_tensor(r, ai, aj, m); }

/* Sphere velocities with the overlap regularisation, brute force over all pairs:
 *   U_a = sum_{b != a} M(x_a - y_b; a_a, b_b) f_b
 * with M the far form outside contact and the overlap form inside.  Pairs with r == 0 and
 * the same index are skipped (self mobility is not part of the kernel sum).
 * x: [nt][3], at: [nt] target radii, y: [ns][3], s: [ns][4] = (f, b), g: [nt][3].
 * same_set != 0 means targets and sources are the same list (index identity = self). */
void orc_rpy_velocity(const double* x, const double* at, int64_t nt, const double* y,
                      int64_t ns, const double* s, int same_set, double* g) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t a = 0; a < nt; ++a) {
    double u[3] = {0, 0, 0}, m[9];
    for (int64_t b = 0; b < ns; ++b) {
      if (same_set && a == b) continue;
      double r[3] = {x[3 * a] - y[3 * b], x[3 * a + 1] - y[3 * b + 1],
                     x[3 * a + 2] - y[3 * b + 2]};
      double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      if (rr == 0.0 && !(s[4 * b + 3] > 0.0 && at[a] > 0.0)) continue;
      rpy_pair_tensor(r, at[a], s[4 * b + 3], m);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) u[i] += m[3 * i + j] * s[4 * b + j];
    }
    for (int i = 0; i < 3; ++i) g[3 * a + i] += u[i];
  }
}

/* Overlap correction only: for pairs within contact (0 < r <= ai + aj, or r == 0 between
 * different indices) add (M_overlap - M_far) f, where M_far is the far form the kernel sum
 * already used (taken as 0 when r == 0, because the kernel sum skips coincident pairs).
 * Used by the plain KAFMM after the tree traversal, Sec. II.B. */
void orc_rpy_overlap_correction(const double* x, const double* at, int64_t nt,
                                const double* y, int64_t ns, const double* s, int same_set,
                                double* g) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t a = 0; a < nt; ++a) {
    double u[3] = {0, 0, 0}, m[9];
    for (int64_t b = 0; b < ns; ++b) {
      if (same_set && a == b) continue;
      double r[3] = {x[3 * a] - y[3 * b], x[3 * a + 1] - y[3 * b + 1],
                     x[3 * a + 2] - y[3 * b + 2]};
      double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      double ai = at[a], aj = s[4 * b + 3];
      if (sqrt(rr) > ai + aj) continue;
      rpy_pair_tensor(r, ai, aj, m);
      if (rr > 0.0) {
        double rn = sqrt(rr), c = ai * ai + aj * aj;
        double A = (1.0 + c / (3.0 * rr)) / (8.0 * PI * rn);
        double B = (1.0 - c / rr) / (8.0 * PI * rn);
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) m[3 * i + j] -= (i == j ? A : 0.0) + B * r[i] * r[j] / rr;
      }
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) u[i] += m[3 * i + j] * s[4 * b + j];
    }
    for (int i = 0; i < 3; ++i) g[3 * a + i] += u[i];
  }
}

/* ---------------------------------------------------------------------------------------
 * Triply periodic sums by Ewald summation (periodic cube of side L), the k = 0 Fourier mode
 * removed -- the zero-mean field of a neutral (sum q = 0) or force-free (sum f = 0) system.
 * Used for the periodic boundary condition of Sec. III.B (the paper's periodisation builds on
 * a precomputed far-image operator; this is its plain definition).
 *
 * Laplace 1/(4 pi r):  G_per(r) = sum_n erfc(xi |r+nL|)/(4 pi |r+nL|) - 1/(4 xi^2 V)
 *                                 + (1/V) sum_{k != 0} exp(-k^2/4xi^2)/k^2 cos(k.r)
 * Stokeslet (Hasimoto split, weight (1 + k^2/4xi^2) exp(-k^2/4xi^2)):
 *   real part  (1/8pi)[ I (erfc(xi r)/r - 2xi/sqrt(pi) e^{-xi^2 r^2})
 *                       + rr/r^2 (erfc(xi r)/r + 2xi/sqrt(pi) e^{-xi^2 r^2}) ]
 *   Fourier    (1/V) sum_{k != 0} (I - kk/k^2)/k^2 (1 + k^2/4xi^2) e^{-k^2/4xi^2} cos(k.r)
 * k = 2 pi m / L, real images n in [-nreal, nreal]^3, m in [-nfour, nfour]^3.  At r = 0 the
 * n = 0 real-space term is replaced by its regular limit (the point's own images only).
 * Differences r must lie in (-L, L)^3 (points inside one cell).
 * ------------------------------------------------------------------------------------- */
static void ewald_lap_block(const double r[3], double L, double xi, int nreal, int nfour,
                           double* out) {
  double V = L * L * L, acc = -1.0 / (4.0 * xi * xi * V);
  for (int i = -nreal; i <= nreal; ++i)
    for (int j = -nreal; j <= nreal; ++j)
      for (int k = -nreal; k <= nreal; ++k) {
        double d[3] = {r[0] + i * L, r[1] + j * L, r[2] + k * L};
        double rn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (rn == 0.0)
          acc += -xi / (2.0 * PI * sqrt(PI));  /* lim (erfc(xi r) - 1)/(4 pi r) */
        else
          acc += erfc(xi * rn) / (4.0 * PI * rn);
      }
  for (int a = -nfour; a <= nfour; ++a)
    for (int b = -nfour; b <= nfour; ++b)
      for (int c = -nfour; c <= nfour; ++c) {
        if (a == 0 && b == 0 && c == 0) continue;
        double kv[3] = {2.0 * PI * a / L, 2.0 * PI * b / L, 2.0 * PI * c / L};
        double k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
        acc += exp(-k2 / (4.0 * xi * xi)) / k2 * cos(kv[0] * r[0] + kv[1] * r[1] + kv[2] * r[2]) / V;
      }
  *out = acc;
}

static void ewald_stk_block(const double r[3], double L, double xi, int nreal, int nfour,
                            double m[9]) {
  double V = L * L * L;
  for (int q = 0; q < 9; ++q) m[q] = 0.0;
  double sp = 2.0 * xi / sqrt(PI);
  for (int i = -nreal; i <= nreal; ++i)
    for (int j = -nreal; j <= nreal; ++j)
      for (int k = -nreal; k <= nreal; ++k) {
        double d[3] = {r[0] + i * L, r[1] + j * L, r[2] + k * L};
        double rr = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double rn = sqrt(rr);
        if (rn == 0.0) {  /* lim (g_R - G) at r = 0: (1/8pi)(-4 xi/sqrt(pi)) I */
          for (int q = 0; q < 3; ++q) m[4 * q] += -2.0 * sp / (8.0 * PI);
          continue;
        }
        double e = exp(-xi * xi * rr), ec = erfc(xi * rn);
        double A = (ec / rn - sp * e) / (8.0 * PI), B = (ec / rn + sp * e) / (8.0 * PI) / rr;
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) m[3 * p + q] += (p == q ? A : 0.0) + B * d[p] * d[q];
      }
  for (int a = -nfour; a <= nfour; ++a)
    for (int b = -nfour; b <= nfour; ++b)
      for (int c = -nfour; c <= nfour; ++c) {
        if (a == 0 && b == 0 && c == 0) continue;
        double kv[3] = {2.0 * PI * a / L, 2.0 * PI * b / L, 2.0 * PI * c / L};
        double k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
        double w = (1.0 + k2 / (4.0 * xi * xi)) * exp(-k2 / (4.0 * xi * xi)) / k2 / V *
                   cos(kv[0] * r[0] + kv[1] * r[1] + kv[2] * r[2]);
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) m[3 * p + q] += w * ((p == q ? 1.0 : 0.0) - kv[p] * kv[q] / k2);
      }
}

/* Gradient of the periodic Laplace Green's function above, d G_per / d r_i: the real-space
 * terms differentiated, d/dr (erfc(xi r)/r) = -erfc(xi r)/r^2 - (2 xi/sqrt(pi)) e^{-xi^2 r^2}/r,
 * and the Fourier terms, -(1/V) sum_{k != 0} e^{-k^2/4xi^2}/k^2 k_i sin(k.r).  At r = 0 the
 * n = 0 real-space term (the point's own regular part, even in r) contributes nothing. */
static void ewald_lapgrad_block(const double r[3], double L, double xi, int nreal, int nfour,
                                double out[3]) {
  double V = L * L * L, sp = 2.0 * xi / sqrt(PI);
  out[0] = out[1] = out[2] = 0.0;
  for (int i = -nreal; i <= nreal; ++i)
    for (int j = -nreal; j <= nreal; ++j)
      for (int k = -nreal; k <= nreal; ++k) {
        double d[3] = {r[0] + i * L, r[1] + j * L, r[2] + k * L};
        double rr = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (rr == 0.0) continue;
        double rn = sqrt(rr);
        double dr = (-erfc(xi * rn) / rr - sp * exp(-xi * xi * rr) / rn) / (4.0 * PI);
        for (int q = 0; q < 3; ++q) out[q] += dr * d[q] / rn;
      }
  for (int a = -nfour; a <= nfour; ++a)
    for (int b = -nfour; b <= nfour; ++b)
      for (int c = -nfour; c <= nfour; ++c) {
        if (a == 0 && b == 0 && c == 0) continue;
        double kv[3] = {2.0 * PI * a / L, 2.0 * PI * b / L, 2.0 * PI * c / L};
        double k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
        double w = -exp(-k2 / (4.0 * xi * xi)) / k2 / V * sin(kv[0] * r[0] + kv[1] * r[1] + kv[2] * r[2]);
        for (int q = 0; q < 3; ++q) out[q] += w * kv[q];
      }
}

/* Periodic StokesPVel block [p, u] <- [f, q] (4 x 4, row-major), Eqs. stkslp, stkslvel with
 * every image: u <- f is Hasimoto's periodic Stokeslet; the pressure of a force and the flow of
 * a source are gradients of the Laplace Green's function, p = -f . grad(1/(4 pi r)) and
 * u = (q/2) grad(1/(4 pi r)), so periodically -f . grad G_per and (q/2) grad G_per (the zero
 * mean pressure of Hasimoto's solution, whose uniform backflow balances the net force, and a
 * uniform sink balancing the net source); p <- q is zero. */
static void ewald_pvel_block(const double r[3], double L, double xi, int nreal, int nfour, double m[16]) {
  double s9[9], gl[3];
  ewald_stk_block(r, L, xi, nreal, nfour, s9);
  ewald_lapgrad_block(r, L, xi, nreal, nfour, gl);
  for (int b = 0; b < 3; ++b) m[b] = -gl[b];
  m[3] = 0.0;
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) m[4 * (1 + a) + b] = s9[3 * a + b];
    m[4 * (1 + a) + 3] = 0.5 * gl[a];
  }
}

/* Rows/columns per point of the periodic kernels: 0 Laplace (1), 1 Stokeslet (3), 2 StokesPVel (4). */
static int ewald_dim(int kernel) { return kernel == 0 ? 1 : (kernel == 1 ? 3 : 4); }

static void ewald_block(int kernel, const double r[3], double L, double xi, int nreal, int nfour, double* m) {
  if (kernel == 0)
    ewald_lap_block(r, L, xi, nreal, nfour, m);
  else if (kernel == 1)
    ewald_stk_block(r, L, xi, nreal, nfour, m);
  else
    ewald_pvel_block(r, L, xi, nreal, nfour, m);
}

/* g += sum_b K_per(x_a - y_b) s_b; kernel 0 = Laplace (k_s = k_t = 1), 1 = Stokeslet (3),
 * 2 = StokesPVel ([f, q] -> [p, u], 4). */
void orc_ewald_sum(int kernel, const double* x, int64_t nt, const double* y, int64_t ns,
                   const double* s, double L, double xi, int nreal, int nfour, double* g) {
  const int kt = ewald_dim(kernel);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t a = 0; a < nt; ++a) {
    double acc[4] = {0, 0, 0, 0}, m[16];
    for (int64_t b = 0; b < ns; ++b) {
      double r[3] = {x[3 * a] - y[3 * b], x[3 * a + 1] - y[3 * b + 1], x[3 * a + 2] - y[3 * b + 2]};
      ewald_block(kernel, r, L, xi, nreal, nfour, m);
      for (int p = 0; p < kt; ++p)
        for (int q = 0; q < kt; ++q) acc[p] += m[kt * p + q] * s[kt * b + q];
    }
    for (int p = 0; p < kt; ++p) g[kt * a + p] += acc[p];
  }
}

/* Kernel matrix of the periodic Green's function: out[(a, p), (b, q)], row-major
 * [nt * kt][ns * kt]. */
void orc_ewald_matrix(int kernel, const double* x, int64_t nt, const double* y, int64_t ns, double L,
                      double xi, int nreal, int nfour, double* out) {
  const int kt = ewald_dim(kernel);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t a = 0; a < nt; ++a) {
    double m[16];
    for (int64_t b = 0; b < ns; ++b) {
      double r[3] = {x[3 * a] - y[3 * b], x[3 * a + 1] - y[3 * b + 1], x[3 * a + 2] - y[3 * b + 2]};
      ewald_block(kernel, r, L, xi, nreal, nfour, m);
      for (int p = 0; p < kt; ++p)
        for (int q = 0; q < kt; ++q) out[(kt * a + p) * (kt * ns) + kt * b + q] = m[kt * p + q];
    }
  }
}

/* Real-space part of the Ewald sum with the minimum-image convention: for every pair the image
 * difference d (each component of r moved into [-L/2, L/2]) contributes its erfc term when
 * |d| < rc <= L/2; every other image lies at least L/2 away, beyond the cutoff.  d = 0 (the
 * target is the source) takes the regular limit of the n = 0 term, as in the blocks above.
 * g += sum over such pairs; kernel 0 = Laplace (no constant term here), 1 = Stokeslet. */
void orc_ewald_real_mi(int kernel, const double* x, int64_t nt, const double* y, int64_t ns,
                       const double* s, double L, double xi, double rc, double* g) {
  const double sp = 2.0 * xi / sqrt(PI), rc2 = rc * rc;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t a = 0; a < nt; ++a) {
    double acc[3] = {0, 0, 0};
    for (int64_t b = 0; b < ns; ++b) {
      double d[3];
      for (int q = 0; q < 3; ++q) {   /* points in one cell: differences in (-L, L) */
        double r = x[3 * a + q] - y[3 * b + q];
        d[q] = r > 0.5 * L ? r - L : (r < -0.5 * L ? r + L : r);
      }
      double rr = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (rr >= rc2) continue;
      if (kernel == 0) {
        acc[0] += s[b] * (rr == 0.0 ? -xi / (2.0 * PI * sqrt(PI)) : erfc(xi * sqrt(rr)) / (4.0 * PI * sqrt(rr)));
      } else if (rr == 0.0) {
        for (int p = 0; p < 3; ++p) acc[p] += -2.0 * sp / (8.0 * PI) * s[3 * b + p];
      } else {
        double rn = sqrt(rr), e = exp(-xi * xi * rr), ec = erfc(xi * rn);
        double A = (ec / rn - sp * e) / (8.0 * PI), B = (ec / rn + sp * e) / (8.0 * PI) / rr;
        double df = d[0] * s[3 * b] + d[1] * s[3 * b + 1] + d[2] * s[3 * b + 2];
        for (int p = 0; p < 3; ++p) acc[p] += A * s[3 * b + p] + B * d[p] * df;
      }
    }
    int kt = kernel == 0 ? 1 : 3;
    for (int p = 0; p < kt; ++p) g[kt * a + p] += acc[p];
  }
}

/* ---------------------------------------------------------------------------------------
 * Stokeslet above a no-slip wall (the plane x_3 = zw), Blake's image system: for a source at
 * y with height h = y_3 - zw and its image y^I = (y_1, y_2, zw - h), r = x - y, R = x - y^I,
 *   8 pi u_i = [S_ij(r) - S_ij(R)] f_j + 2 h sum_k (M f)_k d/dR_k D_i(R),
 *   S_ij(r) = delta_ij / r + r_i r_j / r^3,  M = diag(1, 1, -1),
 *   D_i(R) = h R_i / R^3 - delta_i3 / R - R_i R_3 / R^3.
 * The field vanishes on the wall and equals the free-space Stokeslet plus a regular field near
 * the source.  Sources and targets must lie above the wall; at r = 0 (a target on its source)
 * the free-space term is skipped and the image terms are kept.
 * ------------------------------------------------------------------------------------- */
void orc_stokeslet_wall(const double* x, int64_t nt, const double* y, int64_t ns, const double* f,
                        double zw, double* g) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t a = 0; a < nt; ++a) {
    double acc[3] = {0, 0, 0};
    for (int64_t b = 0; b < ns; ++b) {
      const double h = y[3 * b + 2] - zw;
      double r[3], R[3];
      for (int q = 0; q < 3; ++q) r[q] = x[3 * a + q] - y[3 * b + q];
      R[0] = r[0];
      R[1] = r[1];
      R[2] = x[3 * a + 2] - (zw - h);
      const double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      const double rn = sqrt(rr), Rn = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
      const double* fb = f + 3 * b;
      const double Mf[3] = {fb[0], fb[1], -fb[2]};
      double rf = 0, Rf = 0;
      for (int q = 0; q < 3; ++q) {
        rf += r[q] * fb[q];
        Rf += R[q] * fb[q];
      }
      for (int i = 0; i < 3; ++i) {
        /* r = 0 (the target is the source): the free-space part is skipped, the image part kept */
        double u = (rr > 0.0 ? fb[i] / rn + r[i] * rf / (rn * rn * rn) : 0.0) - fb[i] / Rn -
                   R[i] * Rf / (Rn * Rn * Rn);
        double d = 0;
        for (int k = 0; k < 3; ++k) {
          const double dik = i == k ? 1.0 : 0.0, di3 = i == 2 ? 1.0 : 0.0, d3k = k == 2 ? 1.0 : 0.0;
          const double R3 = Rn * Rn * Rn, R5 = R3 * Rn * Rn;
          d += Mf[k] * (h * (dik / R3 - 3.0 * R[i] * R[k] / R5) + di3 * R[k] / R3 -
                        (dik * R[2] + R[i] * d3k) / R3 + 3.0 * R[i] * R[2] * R[k] / R5);
        }
        acc[i] += u + 2.0 * h * d;
      }
    }
    for (int i = 0; i < 3; ++i) g[3 * a + i] += acc[i] / (8.0 * PI);
  }
}

/* ---------------------------------------------------------------------------------------
 * Singly and doubly periodic image sums (Sec. III.B, boundaries PX and PXY): the kernel
 * matrix summed over the images n L of a 1D lattice (axes = 1: n = (a, 0, 0)) or a 2D
 * lattice (axes = 2: n = (a, b, 0)), taken in square shells max|n| = s for s from nmin up,
 * with the partial sums S_N over nmin <= max|n| <= N written out for N = n0 2^k, k < nlev
 * (the caller extrapolates N -> infinity).  kernel 0: Laplace 1/(4 pi r), 1 x 1 blocks;
 * kernel 1: Stokeslet (delta_ij / r + r_i r_j / r^3) / (8 pi), 3 x 3 blocks; kernel 2:
 * StokesPVel [p, u] <- [f, q] (as orc_stokes_pvel), 4 x 4 blocks.
 * out[k][kt nt][kt ns] (row: target a, output component i; column: source b, component j).
 * Pairs at zero distance are skipped.
 * ------------------------------------------------------------------------------------- */
static void lattice_pair(int kernel, const double r[3], double* m) {
  const double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  if (rr == 0.0) return;
  const double rn = sqrt(rr);
  if (kernel == 0) {
    m[0] += 1.0 / (4.0 * PI * rn);
    return;
  }
  const double r3 = rr * rn;
  if (kernel == 2) {   /* StokesPVel block: rows [p, u], columns [f, q] (Eqs. stkslp, stkslvel) */
    for (int j = 0; j < 3; ++j) m[j] += r[j] / (4.0 * PI * r3);
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j)
        m[4 * (1 + i) + j] += ((i == j ? 1.0 / rn : 0.0) + r[i] * r[j] / r3) / (8.0 * PI);
      m[4 * (1 + i) + 3] += -r[i] / (8.0 * PI * r3);
    }
    return;
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) m[3 * i + j] += ((i == j ? 1.0 / rn : 0.0) + r[i] * r[j] / r3) / (8.0 * PI);
}

void orc_lattice_matrix(int kernel, int axes, const double* x, int64_t nt, const double* y,
                        int64_t ns, double L, int nmin, int n0, int nlev, double* out) {
  const int kt = kernel == 0 ? 1 : (kernel == 1 ? 3 : 4);
  const int64_t rows = kt * nt, cols = kt * ns;
  const int nmax = n0 << (nlev - 1);
#pragma omp parallel for collapse(2) schedule(dynamic, 8)
  for (int64_t a = 0; a < nt; ++a)
    for (int64_t b = 0; b < ns; ++b) {
      double m[16] = {0};
      int lev = 0;
      for (int s = nmin; s <= nmax; ++s) {
        /* the images of shell s: (+-s, 0) for the 1D lattice; the square ring max(|i|,|j|) = s
         * for the 2D lattice (rows j = +-s, then columns i = +-s between them) */
        int cnt = axes == 1 ? 2 : 8 * s;
        for (int e = 0; e < cnt; ++e) {
          int i, j;
          if (axes == 1) {
            i = e == 0 ? -s : s;
            j = 0;
          } else if (e < 2 * (2 * s + 1)) {
            i = -s + e % (2 * s + 1);
            j = e < 2 * s + 1 ? -s : s;
          } else {
            int e2 = e - 2 * (2 * s + 1);
            i = e2 % 2 == 0 ? -s : s;
            j = -s + 1 + e2 / 2;
          }
          double r[3] = {x[3 * a] - y[3 * b] - i * L, x[3 * a + 1] - y[3 * b + 1] - j * L,
                         x[3 * a + 2] - y[3 * b + 2]};
          lattice_pair(kernel, r, m);
        }
        if (s == (n0 << lev)) {
          for (int p = 0; p < kt; ++p)
            for (int q = 0; q < kt; ++q)
              out[(int64_t)lev * rows * cols + (kt * a + p) * cols + kt * b + q] = m[kt * p + q];
          ++lev;
        }
      }
    }
}
