// Plan object and the interfaces between the evaluator's translation units.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace kafmm {

// Device-side view of the octree (boxes numbered level by level, Morton order per level).
struct TreeView {
  int nbox, nlevels, periodic;
  const int* lvl_start;     // [MAX_LEVELS + 1] (device copy)
  const int* prob;          // [nbox] problem of each box (a batch has one root per problem)
  const uint64_t* key;      // cell key (Morton code of the anchor at the box's level)
  const int8_t* level;      // [nbox]
  const int* parent;        // [nbox], -1 for the root
  const int* child;         // [nbox][8], -1 when absent
  const int* sb;            // source range [sb, se) in sorted source order
  const int* se;
  const int* tb;            // target range [tb, te) in sorted target order
  const int* te;
  const int8_t* leaf;       // [nbox] 0/1
};

struct Tree {
  int64_t n_src = 0, n_trg = 0;
  bool same = true;
  // independent problems of one batch: problem k owns sources [src_off[k], src_off[k+1]) and
  // targets [trg_off[k], trg_off[k+1]) of the caller's arrays; a single set has n_prob = 1
  int n_prob = 1;
  std::vector<int64_t> src_off, trg_off;
  DevBuf d_src_off, d_trg_off;
  int nbox = 0, nleaf = 0, nlevels = 0;
  int lvl_start[MAX_LEVELS + 1] = {0};
  int64_t n_u = 0, n_w = 0, n_x = 0, n_v = 0, near_pairs = 0;
  int max_leaf_pts = 0;
  int dtype_pts = KAFMM_F32;       // dtype of the caller's points at set_points
  // sorted points: perm[i] = caller index of sorted point i
  DevBuf src_key, trg_key, src_perm, trg_perm;
  DevBuf src_pos, trg_pos;          // compute-type xyz (float4 or double4, w unused)
  // boxes
  DevBuf d_lvl_start, key, level, parent, child, sb, se, tb, te, leaf, leaves, prob;
  DevBuf leaf_of;                   // [n_src] leaf box of each sorted source point
  // lists, CSR over boxes (entries packed with pack_entry)
  DevBuf u_off, u_ent, w_off, w_ent, x_off, x_ent;
  DevBuf vtab;                      // [nbox][216] source box of each V slot or LIST_EMPTY
  DevBuf vocc;                      // [nbox][32] bytes: V slot occupancy per parent neighbour
  // grouped M->L pairs (box, parent neighbour with V entries) of boxes at levels >= vmin:
  // count and first pair per box, per (neighbour, octant class) totals and their sum
  DevBuf m2l_cnt, m2l_base, m2l_meta;
  unsigned m2l_hist[217] = {0};
  int64_t m2l_npairs = 0;
  DevBuf w_flag;                    // [nbox] 1 if the box appears in some W list
  // scratch of the build
  DevBuf s_keys2, s_vals2, s_hist, t_keys2, t_vals2;
  DevBuf sort_flag;                 // [0] full key sort needed, [1..2] its scan lengths
  DevBuf dense_start;               // dense cell starts of the top levels (sources, targets)
  DevBuf bld_sync;                  // cooperative refinement: barrier words, block totals
  DevBuf bld_key, bld_sb, bld_se, bld_tb, bld_te, bld_parent, bld_child, bld_cnt, bld_nch,
      bld_choff, bld_cb, bld_ctb, bld_prob;
  DevBuf status;                    // unsigned status word
  TreeView view() const;
};

// Work lists of the evaluation, built on the host after each set_points: tiles of boxes that
// share an octant class (int4: offset into boxlist, count, class, 0).
struct WorkLists {
  std::vector<int> boxlist;
  std::vector<int4> tiles;
  int m2l[2] = {0, 0};                       // tile ranges
  // tensor-core M->L tiled per (octant class, parent neighbour g): tile.w = g + 1, tile.x
  // indexes the sorted pair arrays (Plan::m2l_box, m2l_part_sorted); each box's result goes to
  // its own partial and the partials of a box are added in order by Plan::m2l_comb
  bool m2l_grouped = false;
  int64_t m2l_nparts = 0;
  int m2m[MAX_LEVELS][2] = {};
  int l2l[MAX_LEVELS][2] = {};
  int pup[2] = {0, 0}, pdn[2] = {0, 0};
  int root[2] = {0, 0};                      // the root alone (periodic far images)
  int cup[2] = {0, 0}, cx[2] = {0, 0};       // compressed coordinates: leaves, boxes with X entries
  int leaves_n = 0, xbox_off = 0, xbox_n = 0, leafbox_off = 0;  // plain box lists
};

// Child plans of a wall plan: Stokeslet or RPY, Laplace charges + dipoles, (RPY) quadrupoles.
constexpr int WALL_CHILDREN = 3;

struct Plan {
  // problem
  int kernel = 0, bc = 0, p = 0, q = 0;
  int deriv_mode = 0;  // derivative target values: 0 grad, 1 Laplacian, 2 traction
  int prec = KAFMM_PREC_MIXED, variant = KAFMM_ML_L4, near_only = 0, kahan = 0;
  int sync = 1;        // kafmm_eval synchronises and checks the device status (KAFMM_OPT_SYNC)
  int rpy_contact = 0; // KAFMM_OPT_RPY_CONTACT: 0 off, 1 on
  WaitLimits wait;     // KAFMM_OPT_WAIT_LIMIT_US, KAFMM_OPT_WAIT_REPORT_US
  int stall_test = 0;  // KAFMM_OPT_TEST_STALL
  int leaf_stage = 0;  // KAFMM_OPT_LEAF_STAGE: sources per staging buffer of the leaf kernel
  cudaStream_t stream = 0;
  double origin[3] = {0, 0, 0}, L = 1.0;
  int ks = 1, kt = 1;
  int ml_stokes = 0;   // ML-tree kernel: 0 Laplace, 1 Stokeslet
  int C = 1;           // ML columns (4 for the four-channel Laplace table)
  int D = 1;           // rows per surface point (3 for the Stokeslet ML kernel)
  int n = 0;           // points per surface
  int R = 0;           // n * D
  bool ops_ready = false;
  // operators: [N_OPS][R][R] row-major (rows = target check rows, cols = source rows)
  DevBuf ops64, ops32, opstc;       // opstc: [N_M2L][2][R][Rpad] split (hi, lo), tf32 or bf16
  int Rpad = 0;                     // R rounded up to the tensor-core K granularity
  int tc_split = SPLIT_TF32;        // split format of the tensor-core M->L in use
  int tc_split_opt = KAFMM_TC_AUTO; // the requested format (option)
  int tc_rb = 2, tc_boxes = 32;     // row blocks and target boxes per tensor-core CTA
  DevBuf opstc_aux;                 // [N_AUX][2][R][Rpad] tf32 hi/lo of M->M, L->L, pinv factors
  // Compressed coordinates of the mixed form (KAFMM_OPT_COMPRESS): the ML-tree state of a box
  // is its check potential projected on the r leading left singular vectors of the
  // check-to-equivalent matrix (upward U_u, downward U_d; r = singular values above the
  // pseudo-inverse cutoff), every translation P^T T P between those coordinates (rp x rp,
  // rp = max(r_up, r_dn) rounded up to 64); leaves compress their S->M check potentials, and
  // equivalent densities come from V S^+ applied to the coordinates.
  int compress_opt = 2;             // option: use compressed coordinates when the table allows
  bool cmp = false;                 // compressed operators built for this plan
  int rp = 0, r_up = 0, r_dn = 0;
  int tc_split_cm = SPLIT_TF32;     // split format of the compressed M->L
  DevBuf opstc_cm2l;                // [N_M2L][2][rp][rp] M->L in the plan's split format
  DevBuf opstc_caux;                // [N_CAUX][2][rp][rp] tf32: M->M (8), L->L (8), periodic (1)
  DevBuf opstc_cin;                 // [2][2][rp][Rpad] tf32: U_u^T, U_d^T (compress)
  DevBuf opstc_cout;                // [2][2][R][rp] tf32: V_u S_u^+, V_d S_d^+ (decompress)
  DevBuf up_hat, dn_hat;            // [nbox][rp][C] compressed upward / downward state
  DevBuf pvel_shift;                // periodic StokesPVel table: moment partials and shifts
  // TMA descriptors: [operator set][128-byte, 64-byte swizzled rows]; sets: dense M->L, dense
  // aux, compressed M->L, compressed aux, compress, decompress
  alignas(64) unsigned char tmaps[6][2][128];
  bool tmap_ready = false;
  int tc_stages = 2;                // pipeline depth of the tensor-core kernel (2 or 4)
  int tc_ranges = 4;                // most slot ranges (CTAs) per tile of a small grid (1..8)
  int tc_tiling = 0;                // M->L tiles: 0 automatic, 1 whole V lists, 2 per neighbour
  int tc_tiles = 1;                 // consecutive tiles per tensor-core CTA (KAFMM_OPT_TC_TILES)
  size_t dev_mem = 0;               // device memory in bytes (read when the operators are built)
  DevBuf unit64, unit32;            // unit surface [n][3]
  DevBuf tm2l64, tm2l32;            // periodic far-image operator [R][R]
  // tree + data
  Tree tree;
  bool have_points = false;
  DevBuf up_check, dn_check, up_equiv, dn_equiv;   // [nbox][R][C] in compute type
  DevBuf s_sorted;                  // sorted source values, compute type
  DevBuf g_sorted;                  // target values in sorted order
  DevBuf io_in, io_out, io_aux;     // staging for host pointers / dtype conversion
  DevBuf tiles, tile_meta;          // work lists of the gather-GEMM engine
  HostBuf wl_down, wl_up;           // pinned staging of the work-list build (tree in, lists out)
  cudaEvent_t wl_event = nullptr;   // the last work-list upload (the staging buffers are free after it)
  cudaEvent_t wl_dl_event = nullptr;   // the last download of the tree's per-box fields
  bool wl_pending = false;          // downloaded, work lists not laid out yet (worklists_finish)
  int wl_nb = 0, wl_nb_tc = 0;      // boxes per tile of the pending layout
  double host_wl_ms = 0;            // host time of the last work-list build
  DevBuf m2l_parts;                 // partial M->L sums per offset range (tensor-core path)
  // grouped M->L: sorted pairs (keys, partial indices, ping-pong halves), pair boxes before
  // and after sorting, radix histograms, combine list [nbox] (box, first partial, count)
  DevBuf m2l_keys, m2l_vals, m2l_pbox, m2l_box, m2l_hist, m2l_comb;
  const uint32_t* m2l_part_sorted = nullptr;
  int64_t tiles_cap = 0;
  WorkLists wl;
  bool use_tc = false;              // tensor-core M->L available for this plan
  long long launches_points = 0, launches_eval = 0;  // kernel launches of the last calls
  // no-slip wall (KAFMM_BC_WALL): the Stokeslet and Laplace charge + dipole child plans over
  // the sources and their images, and the work arrays of the assembly
  kafmm_plan_t wall_child[WALL_CHILDREN] = {nullptr, nullptr, nullptr};
  DevBuf wall_buf[10];
  cudaEvent_t ev[8] = {0};
  double phase_ms[8] = {0};
  std::string err;

  bool fp64() const { return prec == KAFMM_PREC_FP64; }
  // RPY near field leaves contact pairs to kafmm_rpy_velocity (one shared point set only)
  bool contact_split() const {
    return kernel == KAFMM_RPY && tree.same && rpy_contact == 1;
  }
};

// Sets plan.err and returns code.
int fail(Plan& P, int code, const char* fmt, ...);
int cuda_fail(Plan& P, cudaError_t e, const char* where);

// tree.cu
// Builds the forest of n_prob octrees (one root per problem; src_off / trg_off are host
// arrays of n_prob + 1 offsets into y and x).
int build_tree(Plan& P, const void* y, int64_t ns, const void* x, int64_t nt, int dtype, int n_prob,
               const int64_t* src_off, const int64_t* trg_off);

// operators.cu
int build_operators(Plan& P);

// Sorts the grouped M->L pairs of the current tree (device; see WorkLists::m2l_grouped).
int m2l_pairs_sort(Plan& P);

// eval.cu
int evaluate(Plan& P, const void* s_dev, void* g_dev, int dtype);
int build_worklists(Plan& P, int NB, int NB_TC);
int worklists_download(Plan& P, int NB, int NB_TC);
int worklists_finish(Plan& P);
int rpy_velocity(Plan& P, const void* s_dev, const void* a_dev, const void* g_dev, void* ua_dev,
                 int dtype);
int rpy_velocity_noalloc(Plan& P, const void* s_dev, const void* a_dev, const void* g_dev,
                         void* ua_dev, int dtype);

// wall.cu
int wall_set_points(Plan& P, const void* y, int64_t ns, const void* x, int64_t nt, int dtype);
int wall_eval(Plan& P, const void* s, void* g, int dtype);

}  // namespace kafmm
