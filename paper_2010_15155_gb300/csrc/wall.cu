// Stokeslet above a no-slip wall (Sec. III.C, Table tab:rpywall at b = 0): one Stokeslet sum
// and two Laplace charge + dipole sums over the sources and their mirror images, assembled at
// the targets as
//     u = u^S + grad phi^SDZ + x_3 grad phi^SD - [0, 0, phi^SD]      (x_3: height above the wall)
// with, for a source force f at height h:
//     u^S:  f_12 = (f_1, f_2, 0) at y,  -f_12 at the image y^I            (Stokeslet)
//     SD:   charge -f_3 / 2 at y;  charge f_3 / 2 and dipole h (-f_1, -f_2, f_3) at y^I
//     SDZ:  charge h f_3 / 2 at y;  charge -h f_3 / 2 at y^I
// (the charges of SD read as -f_3 / 2 and +f_3 / 2: with them the assembly is Blake's image
// system).  The RPY kernel (radius b) replaces the Stokeslet sum by an RPY sum of (f_12, b) at y
// and (-f_12, b) at y^I, adds the dipole (b^2/6) (0, 0, f_3) at y and at y^I to SDZ, and a
// fourth sum of Laplace quadrupoles (b^2/3) [[f_3, 0, 0], [0, f_3, 0], [f_1, f_2, 0]] at y^I
// (the table prints it under "source at y"; at y^I the assembly equals the RPY operator
// (1 + b^2/6 lap_y) applied to Blake's solution):
//     u     = u^S + grad phi^SDZ + x_3 grad (phi^SD + phi^Q) - [0, 0, phi^SD + phi^Q]
//     lap u = lap u^S + 2 d_3 grad (phi^SD + phi^Q).
// The wall is the plane z = origin_z + L / 2 and every point lies above it, so the images fall
// in the lower half of the same cube and one octree per sum holds sources, images and targets.
// The sums are child plans (open boundary): a Stokeslet or RPY plan, a Laplace charge + dipole
// plan evaluated twice, and (RPY) a Laplace quadrupole plan.
#include "plan.cuh"

namespace kafmm {

namespace {

template <class T>
__global__ void k_wall_check(const T* __restrict__ p, int64_t n, double zw, unsigned* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!((double)p[3 * i + 2] >= zw)) atomicOr(status, (unsigned)ST_DOMAIN);
}

// yy = [y; y^I], y^I = (y_1, y_2, 2 zw - y_3).
template <class T>
__global__ void k_wall_points(const T* __restrict__ y, int64_t ns, double zw, T* __restrict__ yy) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x) {
    const T a = y[3 * i], b = y[3 * i + 1], c = y[3 * i + 2];
    yy[3 * i] = a;
    yy[3 * i + 1] = b;
    yy[3 * i + 2] = c;
    yy[3 * (ns + i)] = a;
    yy[3 * (ns + i) + 1] = b;
    yy[3 * (ns + i) + 2] = (T)(2.0 * zw - (double)c);
  }
}

// Source values of the three sums over [y; y^I] (layouts of the Stokeslet [3] and of the
// Laplace charge + dipole [q, d_1, d_2, d_3] problems).
template <class T>
__global__ void k_wall_sources(const T* __restrict__ y, const T* __restrict__ f, int64_t ns, double zw,
                               T* __restrict__ s_stk, T* __restrict__ s_sd, T* __restrict__ s_sdz) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x) {
    const T f1 = f[3 * i], f2 = f[3 * i + 1], f3 = f[3 * i + 2];
    const T h = (T)((double)y[3 * i + 2] - zw);
    const int64_t j = ns + i;
    s_stk[3 * i] = f1;
    s_stk[3 * i + 1] = f2;
    s_stk[3 * i + 2] = 0;
    s_stk[3 * j] = -f1;
    s_stk[3 * j + 1] = -f2;
    s_stk[3 * j + 2] = 0;
    s_sd[4 * i] = T(-0.5) * f3;
    s_sd[4 * i + 1] = s_sd[4 * i + 2] = s_sd[4 * i + 3] = 0;
    s_sd[4 * j] = T(0.5) * f3;
    s_sd[4 * j + 1] = -h * f1;
    s_sd[4 * j + 2] = -h * f2;
    s_sd[4 * j + 3] = h * f3;
    s_sdz[4 * i] = T(0.5) * h * f3;
    s_sdz[4 * i + 1] = s_sdz[4 * i + 2] = s_sdz[4 * i + 3] = 0;
    s_sdz[4 * j] = T(-0.5) * h * f3;
    s_sdz[4 * j + 1] = s_sdz[4 * j + 2] = s_sdz[4 * j + 3] = 0;
  }
}

// RPY wall: sources of the four sums over [y; y^I] from [f, b] (RPY [f_12, b], SD and SDZ
// [q, d], quadrupoles Q_jk at 3j + k).
template <class T>
__global__ void k_wall_sources_rpy(const T* __restrict__ y, const T* __restrict__ s, int64_t ns, double zw,
                                   T* __restrict__ s_rpy, T* __restrict__ s_sd, T* __restrict__ s_sdz,
                                   T* __restrict__ s_q) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x) {
    const T f1 = s[4 * i], f2 = s[4 * i + 1], f3 = s[4 * i + 2], b = s[4 * i + 3];
    const T h = (T)((double)y[3 * i + 2] - zw);
    const T bb = b * b;
    const int64_t j = ns + i;
    s_rpy[4 * i] = f1;
    s_rpy[4 * i + 1] = f2;
    s_rpy[4 * i + 2] = 0;
    s_rpy[4 * i + 3] = b;
    s_rpy[4 * j] = -f1;
    s_rpy[4 * j + 1] = -f2;
    s_rpy[4 * j + 2] = 0;
    s_rpy[4 * j + 3] = b;
    s_sd[4 * i] = T(-0.5) * f3;
    s_sd[4 * i + 1] = s_sd[4 * i + 2] = s_sd[4 * i + 3] = 0;
    s_sd[4 * j] = T(0.5) * f3;
    s_sd[4 * j + 1] = -h * f1;
    s_sd[4 * j + 2] = -h * f2;
    s_sd[4 * j + 3] = h * f3;
    s_sdz[4 * i] = T(0.5) * h * f3;
    s_sdz[4 * i + 1] = s_sdz[4 * i + 2] = 0;
    s_sdz[4 * i + 3] = bb * T(1.0 / 6.0) * f3;
    s_sdz[4 * j] = T(-0.5) * h * f3;
    s_sdz[4 * j + 1] = s_sdz[4 * j + 2] = 0;
    s_sdz[4 * j + 3] = bb * T(1.0 / 6.0) * f3;
    const T c = bb * T(1.0 / 3.0);
#pragma unroll
    for (int k = 0; k < 9; ++k) s_q[9 * i + k] = 0;
    s_q[9 * j] = c * f3;
    s_q[9 * j + 1] = 0;
    s_q[9 * j + 2] = 0;
    s_q[9 * j + 3] = 0;
    s_q[9 * j + 4] = c * f3;
    s_q[9 * j + 5] = 0;
    s_q[9 * j + 6] = c * f1;
    s_q[9 * j + 7] = c * f2;
    s_q[9 * j + 8] = 0;
  }
}

// RPY wall: [u, lap u] from [u^S, lap u^S] (6) and the Laplace sums (10 each: [phi, grad,
// Hessian xx xy xz yy yz zz]).
template <class T>
__global__ void k_wall_assemble_rpy(const T* __restrict__ x, int64_t nt, double zw, const T* __restrict__ us,
                                    const T* __restrict__ sd, const T* __restrict__ sdz, const T* __restrict__ q,
                                    T* __restrict__ g) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x) {
    const T x3 = (T)((double)x[3 * i + 2] - zw);
    const T* a = sd + 10 * i;
    const T* c = sdz + 10 * i;
    const T* e = q + 10 * i;
    const T* u = us + 6 * i;
    g[6 * i] = u[0] + c[1] + x3 * (a[1] + e[1]);
    g[6 * i + 1] = u[1] + c[2] + x3 * (a[2] + e[2]);
    g[6 * i + 2] = u[2] + c[3] + x3 * (a[3] + e[3]) - (a[0] + e[0]);
    g[6 * i + 3] = u[3] + T(2) * (a[6] + e[6]);
    g[6 * i + 4] = u[4] + T(2) * (a[8] + e[8]);
    g[6 * i + 5] = u[5] + T(2) * (a[9] + e[9]);
  }
}

// g = u^S + grad phi^SDZ + x_3 grad phi^SD - [0, 0, phi^SD]; the Laplace outputs are
// [phi, grad phi, Hessian] (10 per target).
template <class T>
__global__ void k_wall_assemble(const T* __restrict__ x, int64_t nt, double zw, const T* __restrict__ us,
                                const T* __restrict__ sd, const T* __restrict__ sdz, T* __restrict__ g) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x) {
    const T x3 = (T)((double)x[3 * i + 2] - zw);
    const T* a = sd + 10 * i;
    const T* c = sdz + 10 * i;
    g[3 * i] = us[3 * i] + c[1] + x3 * a[1];
    g[3 * i + 1] = us[3 * i + 1] + c[2] + x3 * a[2];
    g[3 * i + 2] = us[3 * i + 2] + c[3] + x3 * a[3] - a[0];
  }
}

int grid_of(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 8));
}

#define CK(call)                                           \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(P, e_, #call); \
  } while (0)

// Forwards a child plan's failure to the parent (code and message).
int child_fail(Plan& P, kafmm_plan_t c, int rc, const char* what) {
  return fail(P, rc, "%s: %s", what, kafmm_last_error(c));
}

}  // namespace

double wall_z(const Plan& P) { return P.origin[2] + 0.5 * P.L; }

// Points of a wall plan: checks that every point lies above the wall, keeps device copies of
// the targets and of [sources; images], and builds the children's trees.  y and x are device
// arrays of the call's dtype.
int wall_set_points(Plan& P, const void* y, int64_t ns, const void* x, int64_t nt, int dtype) {
  cudaStream_t st = P.stream;
  const size_t es = dtype == KAFMM_F64 ? 8 : 4;
  const double zw = wall_z(P);
  CK(P.wall_buf[0].reserve(es * 3 * (2 * ns + 1)));   // [y; y^I]
  CK(P.wall_buf[1].reserve(es * 3 * (nt + 1)));       // targets
  CK(P.tree.status.reserve(64));
  CK(cudaMemsetAsync(P.tree.status.p, 0, 4, st));
  unsigned* status = P.tree.status.as<unsigned>();
  if (dtype == KAFMM_F64) {
    if (ns) KL k_wall_check<double><<<grid_of(ns), 256, 0, st>>>((const double*)y, ns, zw, status);
    if (nt) KL k_wall_check<double><<<grid_of(nt), 256, 0, st>>>((const double*)x, nt, zw, status);
    if (ns) KL k_wall_points<double><<<grid_of(ns), 256, 0, st>>>((const double*)y, ns, zw, P.wall_buf[0].as<double>());
  } else {
    if (ns) KL k_wall_check<float><<<grid_of(ns), 256, 0, st>>>((const float*)y, ns, zw, status);
    if (nt) KL k_wall_check<float><<<grid_of(nt), 256, 0, st>>>((const float*)x, nt, zw, status);
    if (ns) KL k_wall_points<float><<<grid_of(ns), 256, 0, st>>>((const float*)y, ns, zw, P.wall_buf[0].as<float>());
  }
  if (nt) CK(cudaMemcpyAsync(P.wall_buf[1].p, x, es * 3 * nt, cudaMemcpyDeviceToDevice, st));
  unsigned h = 0;
  CK(cudaMemcpyAsync(&h, status, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h & ST_DOMAIN)
    return fail(P, KAFMM_ERR_DOMAIN, "a point lies below the wall z = %.17g (or is not finite)", zw);
  for (int c = 0; c < WALL_CHILDREN; ++c) {
    if (!P.wall_child[c]) continue;
    int rc = kafmm_set_points(P.wall_child[c], P.wall_buf[0].p, 2 * ns, P.wall_buf[1].p, nt, dtype);
    if (rc) return child_fail(P, P.wall_child[c], rc, c == 0 ? "Stokeslet / RPY sum" : "Laplace sums");
  }
  P.tree.n_src = ns;
  P.tree.n_trg = nt;
  P.tree.dtype_pts = dtype;
  return 0;
}

// RPY wall: the four sums and the assembly.
static int wall_eval_rpy(Plan& P, const void* s, void* g, int dtype) {
  cudaStream_t st = P.stream;
  const int64_t ns = P.tree.n_src, nt = P.tree.n_trg;
  const size_t es = dtype == KAFMM_F64 ? 8 : 4;
  const double zw = wall_z(P);
  CK(P.wall_buf[2].reserve(es * 4 * (2 * ns + 1)));   // RPY [f_12, b]
  CK(P.wall_buf[3].reserve(es * 4 * (2 * ns + 1)));   // SD charges + dipoles
  CK(P.wall_buf[4].reserve(es * 4 * (2 * ns + 1)));   // SDZ charges + dipoles
  CK(P.wall_buf[8].reserve(es * 9 * (2 * ns + 1)));   // quadrupoles
  CK(P.wall_buf[5].reserve(es * 6 * (nt + 1)));       // [u^S, lap u^S]
  CK(P.wall_buf[6].reserve(es * 10 * (nt + 1)));      // phi^SD, grad, Hessian
  CK(P.wall_buf[7].reserve(es * 10 * (nt + 1)));      // phi^SDZ, grad, Hessian
  CK(P.wall_buf[9].reserve(es * 10 * (nt + 1)));      // phi^Q, grad, Hessian
  if (ns) {
    if (dtype == KAFMM_F64)
      KL k_wall_sources_rpy<double><<<grid_of(ns), 256, 0, st>>>(
          P.wall_buf[0].as<double>(), (const double*)s, ns, zw, P.wall_buf[2].as<double>(), P.wall_buf[3].as<double>(),
          P.wall_buf[4].as<double>(), P.wall_buf[8].as<double>());
    else
      KL k_wall_sources_rpy<float><<<grid_of(ns), 256, 0, st>>>(
          P.wall_buf[0].as<float>(), (const float*)s, ns, zw, P.wall_buf[2].as<float>(), P.wall_buf[3].as<float>(),
          P.wall_buf[4].as<float>(), P.wall_buf[8].as<float>());
  }
  int rc = kafmm_eval(P.wall_child[0], P.wall_buf[2].p, P.wall_buf[5].p, dtype);
  if (rc) return child_fail(P, P.wall_child[0], rc, "RPY sum");
  rc = kafmm_eval(P.wall_child[1], P.wall_buf[3].p, P.wall_buf[6].p, dtype);
  if (rc) return child_fail(P, P.wall_child[1], rc, "Laplace sum SD");
  rc = kafmm_eval(P.wall_child[1], P.wall_buf[4].p, P.wall_buf[7].p, dtype);
  if (rc) return child_fail(P, P.wall_child[1], rc, "Laplace sum SDZ");
  rc = kafmm_eval(P.wall_child[2], P.wall_buf[8].p, P.wall_buf[9].p, dtype);
  if (rc) return child_fail(P, P.wall_child[2], rc, "Laplace quadrupole sum");
  if (nt) {
    if (dtype == KAFMM_F64)
      KL k_wall_assemble_rpy<double><<<grid_of(nt), 256, 0, st>>>(
          P.wall_buf[1].as<double>(), nt, zw, P.wall_buf[5].as<double>(), P.wall_buf[6].as<double>(),
          P.wall_buf[7].as<double>(), P.wall_buf[9].as<double>(), (double*)g);
    else
      KL k_wall_assemble_rpy<float><<<grid_of(nt), 256, 0, st>>>(
          P.wall_buf[1].as<float>(), nt, zw, P.wall_buf[5].as<float>(), P.wall_buf[6].as<float>(),
          P.wall_buf[7].as<float>(), P.wall_buf[9].as<float>(), (float*)g);
  }
  CK(cudaGetLastError());
  return 0;
}

// kafmm_eval of a wall plan: s and g device arrays of the call's dtype.
int wall_eval(Plan& P, const void* s, void* g, int dtype) {
  if (P.kernel == KAFMM_RPY) return wall_eval_rpy(P, s, g, dtype);
  cudaStream_t st = P.stream;
  const int64_t ns = P.tree.n_src, nt = P.tree.n_trg;
  const size_t es = dtype == KAFMM_F64 ? 8 : 4;
  const double zw = wall_z(P);
  CK(P.wall_buf[2].reserve(es * 3 * (2 * ns + 1)));   // Stokeslet forces
  CK(P.wall_buf[3].reserve(es * 4 * (2 * ns + 1)));   // SD charges + dipoles
  CK(P.wall_buf[4].reserve(es * 4 * (2 * ns + 1)));   // SDZ charges
  CK(P.wall_buf[5].reserve(es * 3 * (nt + 1)));       // u^S
  CK(P.wall_buf[6].reserve(es * 10 * (nt + 1)));      // phi^SD, grad, Hessian
  CK(P.wall_buf[7].reserve(es * 10 * (nt + 1)));      // phi^SDZ, grad, Hessian
  if (ns) {
    if (dtype == KAFMM_F64)
      KL k_wall_sources<double><<<grid_of(ns), 256, 0, st>>>(P.wall_buf[0].as<double>(), (const double*)s, ns, zw,
                                                          P.wall_buf[2].as<double>(), P.wall_buf[3].as<double>(),
                                                          P.wall_buf[4].as<double>());
    else
      KL k_wall_sources<float><<<grid_of(ns), 256, 0, st>>>(P.wall_buf[0].as<float>(), (const float*)s, ns, zw,
                                                         P.wall_buf[2].as<float>(), P.wall_buf[3].as<float>(),
                                                         P.wall_buf[4].as<float>());
  }
  int rc = kafmm_eval(P.wall_child[0], P.wall_buf[2].p, P.wall_buf[5].p, dtype);
  if (rc) return child_fail(P, P.wall_child[0], rc, "Stokeslet sum");
  rc = kafmm_eval(P.wall_child[1], P.wall_buf[3].p, P.wall_buf[6].p, dtype);
  if (rc) return child_fail(P, P.wall_child[1], rc, "Laplace sum SD");
  rc = kafmm_eval(P.wall_child[1], P.wall_buf[4].p, P.wall_buf[7].p, dtype);
  if (rc) return child_fail(P, P.wall_child[1], rc, "Laplace sum SDZ");
  if (nt) {
    if (dtype == KAFMM_F64)
      KL k_wall_assemble<double><<<grid_of(nt), 256, 0, st>>>(P.wall_buf[1].as<double>(), nt, zw,
                                                           P.wall_buf[5].as<double>(), P.wall_buf[6].as<double>(),
                                                           P.wall_buf[7].as<double>(), (double*)g);
    else
      KL k_wall_assemble<float><<<grid_of(nt), 256, 0, st>>>(P.wall_buf[1].as<float>(), nt, zw,
                                                          P.wall_buf[5].as<float>(), P.wall_buf[6].as<float>(),
                                                          P.wall_buf[7].as<float>(), (float*)g);
  }
  CK(cudaGetLastError());
  return 0;
}

}  // namespace kafmm
