// C ABI of the evaluator (declared in include/kafmm.h).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdarg>
#include <cstring>

#include "plan.cuh"

namespace kafmm {

thread_local long long g_launches = 0;

static std::atomic<long long> g_device_allocs{0};
void count_device_allocation() { g_device_allocs.fetch_add(1, std::memory_order_relaxed); }
long long device_allocations() { return g_device_allocs.load(std::memory_order_relaxed); }

int fail(Plan& P, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  P.err = buf;
  return code;
}

int cuda_fail(Plan& P, cudaError_t e, const char* where) {
  P.err = std::string("CUDA error '") + cudaGetErrorString(e) + "' at " + where;
  cudaGetLastError();  // clear a non-sticky error
  return e == cudaErrorMemoryAllocation ? KAFMM_ERR_NOMEM : KAFMM_ERR_CUDA;
}

// Problem dimensions from kernel, boundary condition and ML variant.
static void configure(Plan& P) {
  int v = P.variant;
  if (periodic_mask(P.bc)) v = KAFMM_ML_G;
  P.ml_stokes = 0;
  P.C = 1;
  P.D = 1;
  switch (P.kernel) {
    case KAFMM_LAPLACE:
      P.ks = 1;
      P.kt = 1;
      break;
    case KAFMM_STOKESLET:
    case KAFMM_RPY:
      P.ks = P.kernel == KAFMM_STOKESLET ? 3 : 4;
      P.kt = P.kernel == KAFMM_STOKESLET ? 3 : 6;
      if (v == KAFMM_ML_L4) {
        P.C = 4;
      } else {
        P.ml_stokes = 1;
        P.D = 3;
      }
      break;
    case KAFMM_LAPLACE_QD:  // [q, d] -> [phi, grad, grad grad] on the Laplace table
      P.ks = 4;
      P.kt = 10;
      break;
    case KAFMM_LAPLACE_QUAD:  // Q -> [phi, grad, grad grad] on the Laplace table
      P.ks = 9;
      P.kt = 10;
      break;
    case KAFMM_STOKES_PVEL:  // [f, q] -> [p, u], G^P for every interaction (Sec. II.C)
      P.ks = 4;
      P.kt = 4;
      P.ml_stokes = 2;
      P.D = 4;
      break;
    case KAFMM_STOKES_REG:  // [f, eps] -> u on the G table (Table tab:ktab_reg)
      P.ks = 4;
      P.kt = 3;
      P.ml_stokes = 1;
      P.D = 3;
      break;
    case KAFMM_STOKES_PVEL_GRAD:       // [f, q] or D -> derivative target values on the
    case KAFMM_STOKES_PVEL_LAPL:       // StokesPVel table (Tables tab:ktab_stkslpvelgrad,
    case KAFMM_STOKES_PVEL_TRACTION:   // tab:ktab_stkdlpvelgrad)
    case KAFMM_STOKES_DL_GRAD:
    case KAFMM_STOKES_DL_LAPL:
    case KAFMM_STOKES_DL_TRACTION: {
      const int k = P.kernel;
      const bool dl = k == KAFMM_STOKES_DL_GRAD || k == KAFMM_STOKES_DL_LAPL || k == KAFMM_STOKES_DL_TRACTION;
      P.deriv_mode = (k == KAFMM_STOKES_PVEL_GRAD || k == KAFMM_STOKES_DL_GRAD)
                         ? 0
                         : ((k == KAFMM_STOKES_PVEL_LAPL || k == KAFMM_STOKES_DL_LAPL) ? 1 : 2);
      P.ks = dl ? 9 : 4;
      P.kt = P.deriv_mode == 0 ? 16 : (P.deriv_mode == 1 ? 7 : 9);
      P.ml_stokes = 2;
      P.D = 4;
      break;
    }
    default:  // double layer D -> [p, u] on the StokesPVel table (Table tab:ktab_stkdlpvelgrad)
      P.ks = 9;
      P.kt = 4;
      P.ml_stokes = 2;
      P.D = 4;
      break;
  }
  P.n = 6 * (P.p - 1) * (P.p - 1) + 2;
  P.R = P.n * P.D;
  P.tc_split = P.tc_split_opt == KAFMM_TC_AUTO ? (P.p >= 10 ? SPLIT_BF16 : SPLIT_TF32)
                                               : (P.tc_split_opt == KAFMM_TC_BF16X3 ? SPLIT_BF16 : SPLIT_TF32);
  P.ops_ready = false;
  P.use_tc = false;
}

static bool is_host_ptr(const void* p) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeUnregistered || a.type == cudaMemoryTypeHost;
}

static int ensure_ops(Plan& P) {
  if (P.ops_ready) return 0;
  int rc = build_operators(P);
  if (rc) return rc;
  extern bool tc_supported(Plan & P);
  P.use_tc = tc_supported(P);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    total_b = 0;
  }
  P.dev_mem = total_b;
  return 0;
}

}  // namespace kafmm

using namespace kafmm;

static thread_local std::string g_err;

#define PLAN_CHECK(pl)                                         \
  if (!(pl)) {                                                 \
    g_err = "null plan";                                       \
    return KAFMM_ERR_ARG;                                      \
  }                                                            \
  Plan& P = *reinterpret_cast<Plan*>(pl);

// Wall plans: queries of the tree, the operators, the autotuner and the RPY calls do not apply.
#define NOT_FOR_WALL(name)                                                             \
  if (P.wall_child[0]) return fail(P, KAFMM_ERR_ARG, name " is not available for a wall plan");

#define CKP(call)                                          \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(P, e_, #call); \
  } while (0)

extern "C" int kafmm_plan(kafmm_kernel kernel, kafmm_bc bc, int p, int q, kafmm_plan_t* out) {
  if (!out) {
    g_err = "kafmm_plan: out is NULL";
    return KAFMM_ERR_ARG;
  }
  *out = nullptr;
  // singly / doubly periodic: the kernels on the Laplace or Stokeslet M->L table
  const bool px_ok = kernel == KAFMM_LAPLACE || kernel == KAFMM_LAPLACE_QD || kernel == KAFMM_LAPLACE_QUAD ||
                     kernel == KAFMM_STOKESLET || kernel == KAFMM_RPY || kernel == KAFMM_STOKES_REG;
  if ((int)kernel < 0 || (int)kernel > 13 ||
      ((kernel == KAFMM_LAPLACE_QD || kernel == KAFMM_LAPLACE_QUAD) && bc == KAFMM_BC_PXYZ) ||
      ((int)bc < KAFMM_BC_OPEN || (int)bc > KAFMM_BC_WALL_PXY) ||
      ((bc == KAFMM_BC_PX || bc == KAFMM_BC_PXY) && !px_ok) ||
      (bc >= KAFMM_BC_WALL && kernel != KAFMM_STOKESLET && kernel != KAFMM_RPY) || p < 2 || p > 16 || q < 1 ||
      q > 4096) {
    g_err = "kafmm_plan: invalid kernel, boundary condition, order (2..16) or leaf size (1..4096)";
    return KAFMM_ERR_ARG;
  }
  Plan* P = new Plan();
  P->kernel = kernel;
  P->bc = bc;
  P->p = p;
  P->q = q;
  configure(*P);
  for (int i = 0; i < 8; ++i) {
    if (cudaEventCreate(&P->ev[i]) != cudaSuccess) {
      g_err = "kafmm_plan: cudaEventCreate failed (no usable CUDA device?)";
      cudaGetLastError();
      delete P;
      return KAFMM_ERR_CUDA;
    }
  }
  if (bc >= KAFMM_BC_WALL) {   // the sums of the image system: Stokeslet or RPY, Laplace charges +
                               // dipoles, and (RPY) Laplace quadrupoles
    const bool rpy = kernel == KAFMM_RPY;
    const kafmm_kernel kk[3] = {rpy ? KAFMM_RPY : KAFMM_STOKESLET, KAFMM_LAPLACE_QD, KAFMM_LAPLACE_QUAD};
    for (int c = 0; c < (rpy ? 3 : 2); ++c) {
      // open, or periodic along x (and y) with the wall
      const kafmm_bc cbc = bc == KAFMM_BC_WALL ? KAFMM_BC_OPEN : (bc == KAFMM_BC_WALL_PX ? KAFMM_BC_PX : KAFMM_BC_PXY);
      int rc = kafmm_plan(kk[c], cbc, p, q, &P->wall_child[c]);
      if (rc) {
        for (int d = 0; d < c; ++d) kafmm_destroy(P->wall_child[d]);
        for (int i = 0; i < 8; ++i) cudaEventDestroy(P->ev[i]);
        delete P;
        return rc;
      }
    }
  }
  *out = reinterpret_cast<kafmm_plan_t>(P);
  return 0;
}

extern "C" int kafmm_set_option(kafmm_plan_t pl, int key, int64_t value) {
  PLAN_CHECK(pl);
  for (int c = 0; c < WALL_CHILDREN; ++c)   // a wall plan's sums take the same options
    if (P.wall_child[c]) {
      int rc = kafmm_set_option(P.wall_child[c], key, value);
      if (rc) return fail(P, rc, "%s", kafmm_last_error(P.wall_child[c]));
    }
  switch (key) {
    case KAFMM_OPT_PRECISION:
      if (value < 0 || value > 2) return fail(P, KAFMM_ERR_ARG, "bad precision %lld", (long long)value);
      if (P.prec != (int)value) {
        P.prec = (int)value;
        configure(P);
        P.have_points = false;
      }
      return 0;
    case KAFMM_OPT_ML_VARIANT:
      if (value < 0 || value > 1) return fail(P, KAFMM_ERR_ARG, "bad ML variant %lld", (long long)value);
      if (P.variant != (int)value) {
        P.variant = (int)value;
        configure(P);
        P.have_points = false;
      }
      return 0;
    case KAFMM_OPT_STREAM:
      P.stream = reinterpret_cast<cudaStream_t>(value);
      return 0;
    case KAFMM_OPT_NEAR_ONLY:
      P.near_only = value ? 1 : 0;
      return 0;
    case KAFMM_OPT_KAHAN:
      P.kahan = value ? 1 : 0;
      return 0;
    case KAFMM_OPT_SYNC:
      P.sync = value ? 1 : 0;
      return 0;
    case KAFMM_OPT_TC_STAGES:
      if (value != 2 && value != 4) return fail(P, KAFMM_ERR_ARG, "tensor-core stages must be 2 or 4");
      P.tc_stages = (int)value;
      return 0;
    case KAFMM_OPT_TC_TILING:
      if (value < 0 || value > 2) return fail(P, KAFMM_ERR_ARG, "bad M->L tiling %lld", (long long)value);
      P.tc_tiling = (int)value;
      return 0;
    case KAFMM_OPT_RPY_CONTACT:
      if (value < 0 || value > 1) return fail(P, KAFMM_ERR_ARG, "bad RPY contact mode %lld", (long long)value);
      P.rpy_contact = (int)value;
      return 0;
    case KAFMM_OPT_TC_RANGES:
      if (value != 1 && value != 2 && value != 4 && value != 8)
        return fail(P, KAFMM_ERR_ARG, "tensor-core slot ranges must be 1, 2, 4 or 8");
      P.tc_ranges = (int)value;
      return 0;
    case KAFMM_OPT_WAIT_LIMIT_US:
      if (value < 1 || value > 60000000)
        return fail(P, KAFMM_ERR_ARG, "wait limit must be 1 .. 60,000,000 microseconds");
      P.wait.hard_ns = (unsigned long long)value * 1000ull;
      return 0;
    case KAFMM_OPT_WAIT_REPORT_US:
      if (value < -1 || value > 60000000)
        return fail(P, KAFMM_ERR_ARG, "wait report threshold must be -1 .. 60,000,000 microseconds");
      P.wait.report_ns = value < 0 ? ~0ull : (unsigned long long)value * 1000ull;
      return 0;
    case KAFMM_OPT_TEST_STALL:
      if (value < 0 || value > 1) return fail(P, KAFMM_ERR_ARG, "test stall must be 0 or 1");
      P.stall_test = (int)value;
      return 0;
    case KAFMM_OPT_TC_TILES:
      if (value != 1 && value != 2 && value != 4)
        return fail(P, KAFMM_ERR_ARG, "tensor-core tiles per CTA must be 1, 2 or 4");
      P.tc_tiles = (int)value;
      return 0;
    case KAFMM_OPT_LEAF_STAGE:
      if (value != 0 && (value < 64 || value > 4096))
        return fail(P, KAFMM_ERR_ARG, "leaf staging must be 0 (default) or 64 .. 4096 sources");
      P.leaf_stage = (int)value;
      return 0;
    case KAFMM_OPT_COMPRESS:
      if (value < 0 || value > 2) return fail(P, KAFMM_ERR_ARG, "compress must be 0, 1 or 2");
      if (P.compress_opt != (int)value) {
        P.compress_opt = (int)value;
        configure(P);
        P.have_points = false;
      }
      return 0;
    case KAFMM_OPT_TC_SPLIT:
      if (value != KAFMM_TC_TF32X3 && value != KAFMM_TC_BF16X3 && value != KAFMM_TC_AUTO)
        return fail(P, KAFMM_ERR_ARG, "bad tensor-core split %lld", (long long)value);
      if (P.tc_split_opt != (int)value) {
        P.tc_split_opt = (int)value;
        configure(P);
        P.have_points = false;
      }
      return 0;
    default:
      return fail(P, KAFMM_ERR_ARG, "unknown option %d", key);
  }
}

extern "C" int kafmm_set_domain(kafmm_plan_t pl, const double origin[3], double L) {
  PLAN_CHECK(pl);
  if (!origin || !(L > 0.0)) return fail(P, KAFMM_ERR_ARG, "bad domain");
  for (int d = 0; d < 3; ++d) P.origin[d] = origin[d];
  P.L = L;
  P.have_points = false;
  for (int c = 0; c < WALL_CHILDREN; ++c)
    if (P.wall_child[c]) kafmm_set_domain(P.wall_child[c], origin, L);
  return 0;
}

// Shared body of kafmm_set_points and kafmm_set_points_batched (arguments validated).
static int set_points_impl(Plan& P, const void* y, int64_t ns, const void* x, int64_t nt, int dtype,
                           int n_prob, const int64_t* soff, const int64_t* toff) {
  P.have_points = false;
  const bool wall = P.wall_child[0] != nullptr;
  int rc = wall ? 0 : ensure_ops(P);
  if (rc) return rc;
  g_launches = 0;
  size_t es = dtype == KAFMM_F64 ? 8 : 4;
  const void* yd = y;
  const void* xd = x;
  bool same = (x == y) && (ns == nt);
  for (int k = 0; same && k <= n_prob; ++k) same = soff[k] == toff[k];
  if (ns > 0 && is_host_ptr(y)) {
    CKP(P.io_in.reserve(es * 3 * ns));
    CKP(cudaMemcpyAsync(P.io_in.p, y, es * 3 * ns, cudaMemcpyHostToDevice, P.stream));
    yd = P.io_in.p;
  }
  if (same) {
    xd = yd;
  } else if (nt > 0 && is_host_ptr(x)) {
    CKP(P.io_aux.reserve(es * 3 * nt));
    CKP(cudaMemcpyAsync(P.io_aux.p, x, es * 3 * nt, cudaMemcpyHostToDevice, P.stream));
    xd = P.io_aux.p;
  }
  if (wall) {
    rc = wall_set_points(P, yd, ns, xd, nt, dtype);
    if (rc) return rc;
    P.launches_points = g_launches;
    P.have_points = true;
    return 0;
  }
  rc = build_tree(P, yd, ns, xd, nt, dtype, n_prob, soff, toff);
  if (rc) return rc;
  // tile sizes: the tensor-core kernels take P.tc_boxes target boxes per tile, k_gemm 64 / C
  // (the work lists are laid out on the host by the first evaluation, while S->M runs)
  int nb_tile = P.use_tc ? P.tc_boxes : 64 / P.C;
  rc = worklists_download(P, nb_tile, nb_tile);
  if (rc) return rc;
  P.launches_points = g_launches;
  P.have_points = true;
  return 0;
}

extern "C" int kafmm_set_points(kafmm_plan_t pl, const void* y, int64_t ns, const void* x, int64_t nt,
                                int dtype) {
  PLAN_CHECK(pl);
  if ((dtype != KAFMM_F32 && dtype != KAFMM_F64) || ns < 0 || nt < 0 || ns > (1ll << 31) - 2 ||
      nt > (1ll << 31) - 2 || (ns > 0 && !y) || (nt > 0 && !x))
    return fail(P, KAFMM_ERR_ARG, "kafmm_set_points: bad arguments");
  int64_t soff[2] = {0, ns}, toff[2] = {0, nt};
  return set_points_impl(P, y, ns, x, nt, dtype, 1, soff, toff);
}

extern "C" int kafmm_set_points_batched(kafmm_plan_t pl, int n_prob, const int64_t* src_offsets,
                                        const int64_t* trg_offsets, const void* y, const void* x,
                                        int dtype) {
  PLAN_CHECK(pl);
  NOT_FOR_WALL("kafmm_set_points_batched")
  P.have_points = false;
  if ((dtype != KAFMM_F32 && dtype != KAFMM_F64) || n_prob < 1 || n_prob > KAFMM_MAX_PROBLEMS ||
      !src_offsets || !trg_offsets)
    return fail(P, KAFMM_ERR_ARG, "kafmm_set_points_batched: bad dtype, problem count (1..%d) or offsets",
                KAFMM_MAX_PROBLEMS);
  if (P.bc != KAFMM_BC_OPEN && n_prob > 1)
    return fail(P, KAFMM_ERR_ARG, "batches of several problems need the open boundary condition");
  const int64_t* offs[2] = {src_offsets, trg_offsets};
  for (int w = 0; w < 2; ++w) {
    const int64_t* o = offs[w];
    if (o[0] != 0) return fail(P, KAFMM_ERR_ARG, "kafmm_set_points_batched: offsets must start at 0");
    for (int k = 0; k < n_prob; ++k)
      if (o[k + 1] < o[k])
        return fail(P, KAFMM_ERR_ARG, "kafmm_set_points_batched: offsets decrease at problem %d", k);
    if (o[n_prob] > (1ll << 31) - 2)
      return fail(P, KAFMM_ERR_ARG, "kafmm_set_points_batched: more than 2^31 - 2 points");
  }
  int64_t ns = src_offsets[n_prob], nt = trg_offsets[n_prob];
  if ((ns > 0 && !y) || (nt > 0 && !x)) return fail(P, KAFMM_ERR_ARG, "kafmm_set_points_batched: null points");
  return set_points_impl(P, y, ns, x, nt, dtype, n_prob, src_offsets, trg_offsets);
}

extern "C" int kafmm_eval(kafmm_plan_t pl, const void* s, void* g, int dtype) {
  PLAN_CHECK(pl);
  if (!P.have_points) return fail(P, KAFMM_ERR_STATE, "kafmm_eval before kafmm_set_points");
  if ((dtype != KAFMM_F32 && dtype != KAFMM_F64) || (P.tree.n_src > 0 && !s) || (P.tree.n_trg > 0 && !g))
    return fail(P, KAFMM_ERR_ARG, "kafmm_eval: bad arguments");
  int rc = P.wall_child[0] ? 0 : ensure_ops(P);
  if (rc) return rc;
  size_t es = dtype == KAFMM_F64 ? 8 : 4;
  const void* sd = s;
  void* gd = g;
  bool host_out = P.tree.n_trg > 0 && is_host_ptr(g);
  if (P.tree.n_src > 0 && is_host_ptr(s)) {
    CKP(P.io_in.reserve(es * P.ks * P.tree.n_src));
    CKP(cudaMemcpyAsync(P.io_in.p, s, es * P.ks * P.tree.n_src, cudaMemcpyHostToDevice, P.stream));
    sd = P.io_in.p;
  }
  if (host_out) {
    CKP(P.io_out.reserve(es * P.kt * P.tree.n_trg));
    gd = P.io_out.p;
  }
  // synchronous calls clear the status word and check it at the end; asynchronous ones leave
  // it sticky for kafmm_status (no host synchronisation, so the call can be stream-captured)
  bool check = P.sync || host_out;
  if (check) CKP(cudaMemsetAsync(P.tree.status.p, 0, 4, P.stream));
  long long l0 = g_launches;
  rc = P.wall_child[0] ? wall_eval(P, sd, gd, dtype) : evaluate(P, sd, gd, dtype);
  P.launches_eval = g_launches - l0;
  if (rc) return rc;
  if (host_out)
    CKP(cudaMemcpyAsync(g, gd, es * P.kt * P.tree.n_trg, cudaMemcpyDeviceToHost, P.stream));
  if (!check) return 0;
  unsigned st = 0;
  CKP(cudaMemcpyAsync(&st, P.tree.status.p, 4, cudaMemcpyDeviceToHost, P.stream));
  CKP(cudaStreamSynchronize(P.stream));
  if (st & ST_TIMEOUT) return fail(P, KAFMM_ERR_TIMEOUT, "a bounded device wait expired");
  return 0;
}

extern "C" int kafmm_autotune(kafmm_plan_t pl, const void* s, void* g, int dtype, int64_t* chosen) {
  PLAN_CHECK(pl);
  NOT_FOR_WALL("kafmm_autotune")
  if (!P.have_points) return fail(P, KAFMM_ERR_STATE, "kafmm_autotune before kafmm_set_points");
  if ((dtype != KAFMM_F32 && dtype != KAFMM_F64) || (P.tree.n_src > 0 && !s) || (P.tree.n_trg > 0 && !g))
    return fail(P, KAFMM_ERR_ARG, "kafmm_autotune: bad arguments");
  if ((P.tree.n_src > 0 && is_host_ptr(s)) || (P.tree.n_trg > 0 && is_host_ptr(g)))
    return fail(P, KAFMM_ERR_ARG, "kafmm_autotune takes device pointers only");
  if (int rw = worklists_finish(P)) return rw;
  int best_st = P.tc_stages, best_rg = P.tc_ranges, best_tl = P.wl.m2l_grouped ? 2 : 1,
      best_tp = P.tc_tiles;
  if (P.use_tc) {
    const int stages[2] = {2, 4}, ranges[4] = {1, 2, 4, 8}, tilings[2] = {2, 1}, tiles[3] = {1, 2, 4};
    const int keep_sync = P.sync;
    P.sync = 1;
    float best = 3.4e38f;
    const int n_stages = P.C == 4 ? 2 : 1;   // single-column tables: two stages only
    int built = -1;
    int rc = 0;
    for (int ti = 0; ti < 2 && !rc; ++ti) {
      // the tiling is fixed by the work lists: rebuild them; the host time of the build is
      // part of every set_points, so it counts towards the score
      P.tc_tiling = tilings[ti];
      auto t0 = std::chrono::steady_clock::now();
      rc = build_worklists(P, P.tc_boxes, P.tc_boxes);
      double host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (rc) break;
      built = tilings[ti];
      if (tilings[ti] == 2 && !P.wl.m2l_grouped) continue;   // partials do not fit
      rc = kafmm_eval(pl, s, g, dtype);   // every buffer exists before the timing
      for (int a = 0; a < n_stages && !rc; ++a)
        for (int b = 0; b < 4 && !rc; ++b)
          for (int c = 0; c < 3 && !rc; ++c) {
            P.tc_stages = stages[a];
            P.tc_ranges = ranges[b];
            P.tc_tiles = tiles[c];
            float t = 0.f;
            for (int rep = 0; rep < 2 && !rc; ++rep) {   // best of two evaluations
              rc = kafmm_eval(pl, s, g, dtype);
              float ms = 0.f;
              cudaEventElapsedTime(&ms, P.ev[3], P.ev[7]);
              t = rep == 0 ? ms : std::min(t, ms);
            }
            t += (float)host_ms;
            if (!rc && t < best) {
              best = t;
              best_st = stages[a];
              best_rg = ranges[b];
              best_tl = tilings[ti];
              best_tp = tiles[c];
            }
          }
    }
    P.sync = keep_sync;
    P.tc_tiling = best_tl;
    if (!rc && built != best_tl) rc = build_worklists(P, P.tc_boxes, P.tc_boxes);
    if (rc) return rc;
  }
  P.tc_stages = best_st;
  P.tc_ranges = best_rg;
  P.tc_tiles = best_tp;
  // near field: sources per staging buffer, timed on the leaf phase alone
  int best_ls = P.leaf_stage;
  {
    const int stages_leaf[3] = {256, 640, 1280};
    const int keep_sync = P.sync;
    P.sync = 1;
    float best = 3.4e38f;
    int rc = 0;
    for (int i = 0; i < 3 && !rc; ++i) {
      P.leaf_stage = stages_leaf[i];
      float t = 0.f;
      for (int rep = 0; rep < 3 && !rc; ++rep) {   // first run warms the configuration
        rc = kafmm_eval(pl, s, g, dtype);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, P.ev[6], P.ev[7]);
        if (rep == 1 || (rep == 2 && ms < t)) t = ms;
      }
      if (!rc && t < best) {
        best = t;
        best_ls = stages_leaf[i];
      }
    }
    P.sync = keep_sync;
    if (rc) return rc;
    P.leaf_stage = best_ls;
  }
  if (chosen) {
    chosen[0] = best_st;
    chosen[1] = best_rg;
    chosen[2] = best_tl;
    chosen[3] = best_ls;
    chosen[4] = best_tp;
  }
  return 0;
}

extern "C" int kafmm_status(kafmm_plan_t pl) {
  PLAN_CHECK(pl);
  for (int c = 0; c < WALL_CHILDREN; ++c)
    if (P.wall_child[c]) {
      int rc = kafmm_status(P.wall_child[c]);
      if (rc) return fail(P, rc, "%s", kafmm_last_error(P.wall_child[c]));
    }
  if (!P.tree.status.p) return 0;
  unsigned st = 0;
  CKP(cudaMemcpyAsync(&st, P.tree.status.p, 4, cudaMemcpyDeviceToHost, P.stream));
  CKP(cudaStreamSynchronize(P.stream));
  CKP(cudaMemsetAsync(P.tree.status.p, 0, 4, P.stream));
  CKP(cudaStreamSynchronize(P.stream));
  if (st & ST_TIMEOUT) return fail(P, KAFMM_ERR_TIMEOUT, "a bounded device wait expired");
  return 0;
}

extern "C" int kafmm_rpy_velocity(kafmm_plan_t pl, const void* s, const void* a, const void* g, void* ua,
                                  int dtype) {
  PLAN_CHECK(pl);
  if (P.kernel != KAFMM_RPY) return fail(P, KAFMM_ERR_ARG, "kafmm_rpy_velocity needs the RPY kernel");
  if (!P.have_points) return fail(P, KAFMM_ERR_STATE, "kafmm_rpy_velocity before kafmm_set_points");
  if (P.tree.n_prob > 1) return fail(P, KAFMM_ERR_ARG, "kafmm_rpy_velocity takes one point set, not a batch");
  if ((dtype != KAFMM_F32 && dtype != KAFMM_F64) || (P.tree.n_src > 0 && !s) ||
      (P.tree.n_trg > 0 && (!a || !g || !ua)))
    return fail(P, KAFMM_ERR_ARG, "kafmm_rpy_velocity: bad arguments");
  size_t es = dtype == KAFMM_F64 ? 8 : 4;
  int64_t ns = P.tree.n_src, nt = P.tree.n_trg;
  DevBuf bs, ba, bg, bu;
  const void *sd = s, *ad = a, *gd = g;
  void* ud = ua;
  bool host_out = nt > 0 && is_host_ptr(ua);
  if (ns > 0 && is_host_ptr(s)) {
    CKP(bs.reserve(es * 4 * ns));
    CKP(cudaMemcpyAsync(bs.p, s, es * 4 * ns, cudaMemcpyHostToDevice, P.stream));
    sd = bs.p;
  }
  if (nt > 0 && is_host_ptr(a)) {
    CKP(ba.reserve(es * nt));
    CKP(cudaMemcpyAsync(ba.p, a, es * nt, cudaMemcpyHostToDevice, P.stream));
    ad = ba.p;
  }
  if (nt > 0 && is_host_ptr(g)) {
    CKP(bg.reserve(es * 6 * nt));
    CKP(cudaMemcpyAsync(bg.p, g, es * 6 * nt, cudaMemcpyHostToDevice, P.stream));
    gd = bg.p;
  }
  if (host_out) {
    CKP(bu.reserve(es * 3 * nt));
    ud = bu.p;
  }
  int rc = rpy_velocity(P, sd, ad, gd, ud, dtype);
  if (rc) return rc;
  if (host_out) {
    CKP(cudaMemcpyAsync(ua, ud, es * 3 * nt, cudaMemcpyDeviceToHost, P.stream));
    CKP(cudaStreamSynchronize(P.stream));
  }
  return 0;
}

extern "C" int kafmm_rpy_velocity_noalloc(kafmm_plan_t pl, const void* s, const void* a, const void* g,
                                          void* ua, int dtype) {
  PLAN_CHECK(pl);
  if (P.kernel != KAFMM_RPY) return fail(P, KAFMM_ERR_ARG, "kafmm_rpy_velocity_noalloc needs the RPY kernel");
  if (!P.have_points) return fail(P, KAFMM_ERR_STATE, "kafmm_rpy_velocity_noalloc before kafmm_set_points");
  if (P.tree.n_prob > 1)
    return fail(P, KAFMM_ERR_ARG, "kafmm_rpy_velocity_noalloc takes one point set, not a batch");
  if ((dtype != KAFMM_F32 && dtype != KAFMM_F64) || (P.tree.n_src > 0 && !s) ||
      (P.tree.n_trg > 0 && (!a || !g || !ua)))
    return fail(P, KAFMM_ERR_ARG, "kafmm_rpy_velocity_noalloc: bad arguments");
  // host arrays would need staging buffers, i.e. an allocation: device pointers only
  if ((P.tree.n_src > 0 && is_host_ptr(s)) ||
      (P.tree.n_trg > 0 && (is_host_ptr(a) || is_host_ptr(g) || is_host_ptr(ua))))
    return fail(P, KAFMM_ERR_ARG, "kafmm_rpy_velocity_noalloc takes device pointers only");
  return rpy_velocity_noalloc(P, s, a, g, ua, dtype);
}

extern "C" int kafmm_tree_info(kafmm_plan_t pl, int64_t* info, int n) {
  PLAN_CHECK(pl);
  if (P.wall_child[0]) return kafmm_tree_info(P.wall_child[0], info, n);
  if (!info || n < 0) return fail(P, KAFMM_ERR_ARG, "bad info array");
  if (!P.have_points) return fail(P, KAFMM_ERR_STATE, "no points");
  if (int rw = worklists_finish(P)) return rw;   // the pair counts come with the work lists
  const Tree& T = P.tree;
  int64_t v[10] = {T.nbox, T.nleaf, T.nlevels, T.n_u, T.n_v, T.n_w, T.n_x, T.near_pairs, T.max_leaf_pts,
                   T.n_prob};
  for (int i = 0; i < n && i < 16; ++i) info[i] = i < 10 ? v[i] : 0;
  return 0;
}

namespace kafmm {
__global__ void k_anchor(const uint64_t* key, int n, int32_t* out) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
    uint64_t k = key[b];
    out[3 * b] = (int32_t)compact3(k);
    out[3 * b + 1] = (int32_t)compact3(k >> 1);
    out[3 * b + 2] = (int32_t)compact3(k >> 2);
  }
}
__global__ void k_vtab_csr(const int32_t* vtab, int nbox, const int64_t* off, int32_t* ent) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += gridDim.x * blockDim.x) {
    int64_t o = off[b];
    for (int k = 0; k < 216; ++k) {
      int32_t e = vtab[(int64_t)b * 216 + k];
      if (e != LIST_EMPTY) ent[o++] = e;
    }
  }
}
__global__ void k_vtab_count(const int32_t* vtab, int nbox, int64_t* cnt) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += gridDim.x * blockDim.x) {
    int64_t c = 0;
    for (int k = 0; k < 216; ++k) c += vtab[(int64_t)b * 216 + k] != LIST_EMPTY;
    cnt[b] = c;
  }
}
}  // namespace kafmm

extern "C" int kafmm_get_tree(kafmm_plan_t pl, int32_t* level, int32_t* anchor, int32_t* parent,
                              int8_t* leaf) {
  PLAN_CHECK(pl);
  NOT_FOR_WALL("kafmm_get_tree")
  if (!P.have_points) return fail(P, KAFMM_ERR_STATE, "no points");
  Tree& T = P.tree;
  int nb = T.nbox;
  cudaStream_t st = P.stream;
  if (level) {
    std::vector<int8_t> l8(nb);
    CKP(cudaMemcpyAsync(l8.data(), T.level.p, nb, cudaMemcpyDeviceToHost, st));
    CKP(cudaStreamSynchronize(st));
    for (int i = 0; i < nb; ++i) level[i] = l8[i];
  }
  if (anchor) {
    DevBuf tmp;
    CKP(tmp.reserve(sizeof(int32_t) * 3 * nb));
    KL k_anchor<<<256, 256, 0, st>>>(T.key.as<uint64_t>(), nb, tmp.as<int32_t>());
    CKP(cudaMemcpyAsync(anchor, tmp.p, sizeof(int32_t) * 3 * nb, cudaMemcpyDeviceToHost, st));
    CKP(cudaStreamSynchronize(st));
  }
  if (parent) CKP(cudaMemcpyAsync(parent, T.parent.p, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, st));
  if (leaf) CKP(cudaMemcpyAsync(leaf, T.leaf.p, nb, cudaMemcpyDeviceToHost, st));
  CKP(cudaStreamSynchronize(st));
  return 0;
}

extern "C" int kafmm_get_list(kafmm_plan_t pl, int kind, int64_t* offsets, int32_t* entries,
                              int8_t* shifts) {
  PLAN_CHECK(pl);
  NOT_FOR_WALL("kafmm_get_list")
  if (!P.have_points) return fail(P, KAFMM_ERR_STATE, "no points");
  if (kind < 0 || kind > 3) return fail(P, KAFMM_ERR_ARG, "bad list kind");
  Tree& T = P.tree;
  int nb = T.nbox;
  cudaStream_t st = P.stream;
  std::vector<int64_t> off(nb + 1);
  int64_t n = 0;
  DevBuf doff, dent;
  const int64_t* src_off = nullptr;
  const int32_t* src_ent = nullptr;
  if (kind == 1) {
    CKP(doff.reserve(sizeof(int64_t) * (nb + 1)));
    KL k_vtab_count<<<256, 256, 0, st>>>(T.vtab.as<int32_t>(), nb, doff.as<int64_t>());
    std::vector<int64_t> cnt(nb);
    CKP(cudaMemcpyAsync(cnt.data(), doff.p, sizeof(int64_t) * nb, cudaMemcpyDeviceToHost, st));
    CKP(cudaStreamSynchronize(st));
    off[0] = 0;
    for (int b = 0; b < nb; ++b) off[b + 1] = off[b] + cnt[b];
    n = off[nb];
    CKP(cudaMemcpyAsync(doff.p, off.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, st));
    CKP(dent.reserve(sizeof(int32_t) * (n + 1)));
    KL k_vtab_csr<<<256, 256, 0, st>>>(T.vtab.as<int32_t>(), nb, doff.as<int64_t>(), dent.as<int32_t>());
    src_ent = dent.as<int32_t>();
  } else {
    src_off = kind == 0 ? T.u_off.as<int64_t>() : (kind == 2 ? T.w_off.as<int64_t>() : T.x_off.as<int64_t>());
    src_ent = kind == 0 ? T.u_ent.as<int32_t>() : (kind == 2 ? T.w_ent.as<int32_t>() : T.x_ent.as<int32_t>());
    CKP(cudaMemcpyAsync(off.data(), src_off, sizeof(int64_t) * (nb + 1), cudaMemcpyDeviceToHost, st));
    CKP(cudaStreamSynchronize(st));
    n = off[nb];
  }
  if (offsets) memcpy(offsets, off.data(), sizeof(int64_t) * (nb + 1));
  if (entries || shifts) {
    std::vector<int32_t> e(n);
    if (n) CKP(cudaMemcpyAsync(e.data(), src_ent, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
    CKP(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < n; ++i) {
      if (entries) entries[i] = entry_box(e[i]);
      if (shifts) shifts[i] = (int8_t)entry_shift(e[i]);
    }
  }
  return 0;
}

extern "C" int kafmm_phase_times(kafmm_plan_t pl, double* t, int n) {
  PLAN_CHECK(pl);
  if (P.wall_child[0]) return kafmm_phase_times(P.wall_child[0], t, n);
  if (!t) return fail(P, KAFMM_ERR_ARG, "null array");
  // ev: 0 start of set_points, 1 tree done, 2 lists done, 3 eval start, 4 upward done,
  //     5 M->L done, 6 downward done, 7 eval done
  float ms[8] = {0};
  int pairs[7][2] = {{0, 1}, {1, 2}, {3, 4}, {4, 5}, {5, 6}, {6, 7}, {3, 7}};
  for (int i = 0; i < 7; ++i) {
    float v = 0;
    if (cudaEventElapsedTime(&v, P.ev[pairs[i][0]], P.ev[pairs[i][1]]) != cudaSuccess) {
      cudaGetLastError();
      v = -1;
    }
    ms[i] = v;
  }
  for (int i = 0; i < n && i < 8; ++i) t[i] = i < 7 ? ms[i] : P.host_wl_ms;
  return 0;
}

extern "C" int kafmm_get_counters(kafmm_plan_t pl, int64_t* c, int n) {
  PLAN_CHECK(pl);
  if (P.wall_child[0]) return kafmm_get_counters(P.wall_child[0], c, n);
  if (!c || n < 0) return fail(P, KAFMM_ERR_ARG, "null array");
  if (P.have_points)
    if (int rw = worklists_finish(P)) return rw;
  const bool cm = P.use_tc && P.cmp;
  int64_t v[11] = {P.launches_points, P.launches_eval, P.use_tc ? 1 : 0,
                   P.launches_points + P.launches_eval,
                   P.use_tc ? ((cm ? P.tc_split_cm : P.tc_split) == SPLIT_BF16 ? KAFMM_TC_BF16X3
                                                                               : KAFMM_TC_TF32X3)
                            : -1,
                   P.wl.m2l_grouped ? 2 : 1, P.wl.m2l[1] - P.wl.m2l[0], device_allocations(),
                   cm ? P.rp : 0, cm ? P.r_up : 0, cm ? P.r_dn : 0};
  for (int i = 0; i < n && i < 12; ++i) c[i] = i < 11 ? v[i] : 0;
  return 0;
}

extern "C" int kafmm_get_operator(kafmm_plan_t pl, int slot, double* out) {
  PLAN_CHECK(pl);
  NOT_FOR_WALL("kafmm_get_operator")
  if (!out || slot < 0 || slot >= N_OPS) return fail(P, KAFMM_ERR_ARG, "bad operator slot");
  int rc = ensure_ops(P);
  if (rc) return rc;
  size_t RR = (size_t)P.R * P.R;
  if (P.fp64()) {
    CKP(cudaMemcpy(out, P.ops64.as<double>() + RR * slot, sizeof(double) * RR, cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> tmp(RR);
    CKP(cudaMemcpy(tmp.data(), P.ops32.as<float>() + RR * slot, sizeof(float) * RR, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < RR; ++i) out[i] = tmp[i];
  }
  return 0;
}

extern "C" int kafmm_destroy(kafmm_plan_t pl) {
  if (!pl) return 0;
  Plan* P = reinterpret_cast<Plan*>(pl);
  for (int c = 0; c < WALL_CHILDREN; ++c)
    if (P->wall_child[c]) kafmm_destroy(P->wall_child[c]);
  for (int i = 0; i < 8; ++i)
    if (P->ev[i]) cudaEventDestroy(P->ev[i]);
  if (P->wl_event) {
    cudaEventSynchronize(P->wl_event);
    cudaEventDestroy(P->wl_event);
  }
  if (P->wl_dl_event) {   // copies into the page-locked staging buffer may still be landing
    cudaEventSynchronize(P->wl_dl_event);
    cudaEventDestroy(P->wl_dl_event);
  }
  delete P;
  return 0;
}

extern "C" const char* kafmm_last_error(kafmm_plan_t pl) {
  if (!pl) return g_err.c_str();
  return reinterpret_cast<Plan*>(pl)->err.c_str();
}
