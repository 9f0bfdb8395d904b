/*
 * kafmm.h -- C ABI of the GB300 (sm_103a) Kernel Aggregated FMM evaluator.
 *
 * Computes the kernel sum of Yan & Blackwell, "Kernel Aggregated Fast Multipole Method"
 * (arXiv:2010.15155), Eq. kernelsumlinear (Sec. I):
 *
 *     g_i(x_a) = sum_b K_ij(x_a, y_b) s_j(y_b),     a = 1..n_trg,  b = 1..n_src,
 *
 * over an adaptive octree with the U/V/W/X interaction lists (Sec. II, Table tab:ktabdef),
 * using the aggregated kernel tables of Sec. II (Tables tab:ktab_rpy, tab:ktab_reg,
 * tab:ktab_stkdlpvelgrad).  Pairs at zero distance contribute nothing (this removes the self
 * term when sources and targets are the same set).  Viscosity mu = 1.
 *
 * Conventions for every call:
 *   - Return value: 0 on success, a negative KAFMM_ERR_* code otherwise; the message is
 *     available from kafmm_last_error(plan).  No call exits the process or traps the device.
 *   - Arrays are row-major.  Points are [n][3] (x, y, z).  Source values s are [n_src][k_s],
 *     target values g are [n_trg][k_t], with (k_s, k_t) per kernel below.
 *   - Pointers may be device pointers (cudaMalloc / PyTorch CUDA tensors) or host pointers;
 *     host arrays are copied to and from the device inside the call (on the plan's stream,
 *     which is synchronised before a host output is returned).  The caller owns every
 *     buffer it passes; the plan owns the tree, the lists, the operators and all workspace.
 *   - All device work is issued on the plan's stream (KAFMM_OPT_STREAM, default: the legacy
 *     default stream).  Calls on one plan must not run concurrently.
 *   - dtype is KAFMM_F32 or KAFMM_F64 and applies to points, s and g alike.
 */
#ifndef KAFMM_H
#define KAFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kafmm_plan_s* kafmm_plan_t;

/* Kernel summation problems (Table tab:implement).
 *   KAFMM_LAPLACE    q -> phi,               K = 1/(4 pi r)                      k_s=1, k_t=1
 *                    (Sec. II.A)
 *   KAFMM_STOKESLET  f -> u,                 G = (I/r + r r^T/r^3)/(8 pi)        k_s=3, k_t=3
 *                    (Sec. II.B)
 *   KAFMM_RPY        [f, b] -> [u, lap u],   u = (1 + b^2/6 lap) G f             k_s=4, k_t=6
 *                    (Eqs. RPYflow, RPYkernel; source radius b per point; Table tab:ktab_rpy)
 *   KAFMM_STOKES_DL  D -> [p, u],            Eqs. stkdlp, stkdlvel, D_jk at 3j+k k_s=9, k_t=4
 *                    (Sec. II.C, Table tab:ktab_stkdlpvelgrad): the double-layer kernel from
 *                    the sources; the StokesPVel kernel G^P ([f, q] -> [p, u], Eqs. stkslp,
 *                    stkslvel: the fluid source q carries the net flow -1/2 tr D) between and
 *                    from the equivalent surfaces (4 values per surface point).  Check values
 *                    are kept as [h p, u] per box of half-width h, so the translations stay
 *                    level-independent.  Open or triply periodic (periodic: sum of tr D = 0).
 *   KAFMM_STOKES_REG [f, eps] -> u,          regularized Stokeslet               k_s=4, k_t=3
 *                    (Sec. II.B, Table tab:ktab_reg): the flow of f spread by the blob
 *                    15 eps^4 / (8 pi (r^2 + eps^2)^{7/2}),
 *                    8 pi G^eps = [(r^2 + 2 eps^2) I + r r^T] / (r^2 + eps^2)^{3/2}, eps per
 *                    source.  G^eps from the sources (S->M, S->L, S->T), the singular
 *                    Stokeslet elsewhere, always on the G table (KAFMM_OPT_ML_VARIANT is
 *                    ignored).  eps must be far below the smallest leaf box (Sec. II.B).
 *                    Pairs at r = 0 are skipped as for the other kernels; a caller wanting a
 *                    blob's own velocity adds G^eps(0) f = f / (4 pi eps).
 *   KAFMM_LAPLACE_QD [q, d] -> [phi, grad phi, grad grad phi]                     k_s=4, k_t=10
 *                    (Sec. II.A, Table tab:ktab_lapqdpgradgrad): charge q and dipole d per
 *                    source, phi = q/(4 pi r) + d.r/(4 pi r^3); outputs phi, d_x phi, d_y phi,
 *                    d_z phi, then the Hessian xx xy xz yy yz zz.  L and L^D from the sources,
 *                    charges on the equivalent surfaces (Laplace table).  Open boundary only
 *                    (KAFMM_ERR_ARG with KAFMM_BC_PXYZ).
 *   KAFMM_STOKES_PVEL [f, q] -> [p, u],      StokesPVel G^P                      k_s=4, k_t=4
 *                    (Sec. II.C, Eqs. stkslp, stkslvel): force f and fluid source q (twice
 *                    the fluid removed) to pressure and velocity,
 *                    p = r.f/(4 pi r^3), u = G f - r q/(8 pi r^3); G^P for all interactions,
 *                    check values kept as [h p, u] as for KAFMM_STOKES_DL.  Open or
 *                    triply periodic (periodic: sum of f = 0 and sum of q = 0).
 *   Derivative target values (PVelGrad, PVelLaplacian and Traction of Table tab:implement;
 *   the T column of Tables tab:ktab_stkslpvelgrad and tab:ktab_stkdlpvelgrad), from [f, q]
 *   sources (KAFMM_STOKES_PVEL_*, k_s=4) or double-layer D sources (KAFMM_STOKES_DL_*, k_s=9),
 *   on the same StokesPVel ML table, open or triply periodic:
 *     *_GRAD      [p, u, d p / d x_1..3, d u_i / d x_j at 7 + 3 i + j]                 k_t=16
 *     *_LAPL      [p, u, lap u]; lap u is evaluated as grad p (the Stokes equation off the
 *                 sources, mu = 1)                                                       k_t=7
 *     *_TRACTION  sigma_ij = -p delta_ij + d u_i / d x_j + d u_j / d x_i at 3 i + j
 *                 (Eq. stressdef, mu = 1)                                                k_t=9
 *   KAFMM_LAPLACE_QUAD Q -> [phi, grad phi, grad grad phi]                        k_s=9, k_t=10
 *                    (LapQPGradGrad of Table tab:implement): quadrupole Q_jk at 3j+k per source,
 *                    phi = Q_jk d_j d_k (1/(4 pi r)) (derivatives in x); outputs as for
 *                    KAFMM_LAPLACE_QD.  The quadrupole potential from the sources, charges on
 *                    the equivalent surfaces (Laplace table).  Open boundary only. */
typedef enum {
  KAFMM_LAPLACE = 0,
  KAFMM_STOKESLET = 1,
  KAFMM_RPY = 2,
  KAFMM_STOKES_DL = 3,
  KAFMM_STOKES_REG = 4,
  KAFMM_LAPLACE_QD = 5,
  KAFMM_STOKES_PVEL = 6,
  KAFMM_STOKES_PVEL_GRAD = 7,
  KAFMM_STOKES_PVEL_LAPL = 8,
  KAFMM_STOKES_PVEL_TRACTION = 9,
  KAFMM_STOKES_DL_GRAD = 10,
  KAFMM_STOKES_DL_LAPL = 11,
  KAFMM_STOKES_DL_TRACTION = 12,
  KAFMM_LAPLACE_QUAD = 13
} kafmm_kernel;

/* Boundary conditions (Sec. III.B, Table tab:implement).
 * KAFMM_BC_PX / KAFMM_BC_PXY: singly periodic along x / doubly periodic along x and y, with
 * period L (the cube [origin, origin + L)^3; every point must lie inside it, the other axes are
 * open).  For KAFMM_LAPLACE, KAFMM_LAPLACE_QD, KAFMM_LAPLACE_QUAD, KAFMM_STOKESLET, KAFMM_RPY
 * and KAFMM_STOKES_REG (the kernels whose M->L table is Laplace or the Stokeslet G; the
 * StokesPVel-table kernels answer KAFMM_ERR_ARG).  The sources must be neutral in the monopole
 * (sum of q = 0, sum of f = 0; a net charge or force makes the image sum diverge, like log r
 * along a line and like r over a plane).  The result is the limit of the symmetric sums over the
 * images with max|n| <= N (n along the periodic axes), which exists for neutral sources.  The
 * tree's lists wrap along the periodic axes (images with shift -1, 0, 1), and the farther images
 * enter through an operator on the root's multipole density, computed once per plan as the FP64
 * image sum over max|n| = 2 ... N, N = 128 (plane) or 2048 (line), extrapolated in N and
 * projected onto neutral densities.
 * KAFMM_BC_PXYZ: triply periodic in the cube
 * [origin, origin + L)^3; the far images enter through a precomputed operator on the
 * root's multipole density (Sec. III, App. B).  Periodic sums need a zero net source
 * (sum of f = 0 for the Stokeslet, sum of q = 0 for Laplace, both for StokesPVel, sum of
 * tr D = 0 for the double layer); the k = 0 Fourier mode is dropped (zero-mean field).  The
 * StokesPVel table adds the constant pressure and velocity shifts of the source moments its
 * equivalent densities do not carry (the trace of the force dipole, and the split of the
 * potential-dipole field between source dipoles and force quadrupoles).
 * KAFMM_BC_WALL_PX / KAFMM_BC_WALL_PXY (KAFMM_STOKESLET and KAFMM_RPY): the wall below combined
 * with periodicity along x / along x and y (period L): the same image system, its sums taken
 * singly / doubly periodic (their sources and images are neutral by construction, so any net
 * force is allowed; above a plane lattice a net force parallel to the wall drives a uniform
 * flow far from it).
 * KAFMM_BC_WALL (KAFMM_STOKESLET and KAFMM_RPY): a no-slip wall on the plane z = origin_z + L / 2,
 * open elsewhere (Sec. III.C).  Every source and target must lie above it (z in
 * [origin_z + L/2, origin_z + L)), else KAFMM_ERR_DOMAIN; their mirror images fill the lower
 * half of the cube.  The flow is Blake's image system, evaluated as one Stokeslet and two
 * Laplace charge + dipole KAFMM sums over the sources and their images and assembled at the
 * targets (Table tab:rpywall with b = 0):
 *   u = u^S + grad phi^SDZ + x_3 grad phi^SD - [0, 0, phi^SD],  x_3 = height above the wall,
 *   u^S: (f_1, f_2, 0) at y and its negative at the image; phi^SD: charge -f_3/2 at y, charge
 *   f_3/2 and dipole h (-f_1, -f_2, f_3) at the image; phi^SDZ: charge h f_3/2 at y, -h f_3/2
 *   at the image (h: the source's height).  A target on a source gets that source's image
 *   field, not its own.  KAFMM_RPY ([f, b] -> [u, lap u]): the RPY kernel sum above the wall,
 *   u = (1 + b^2/6 lap_y) G_wall f, from four sums (Table tab:rpywall): an RPY sum of (f_12, b)
 *   at y and (-f_12, b) at the image, SD as above, SDZ plus the dipole (b^2/6)(0, 0, f_3) at y
 *   and at the image, and Laplace quadrupoles (b^2/3)[[f_3,0,0],[0,f_3,0],[f_1,f_2,0]] at the
 *   image (printed under "source at y"; at the image the assembly is the definition; spheres
 *   are expected to lie clear of the wall, h > b: the image terms grow like b^2 / h^3 and, in
 *   the FP32 and mixed forms, the four sums then cancel to rounding), with
 *     u = u^S + grad phi^SDZ + x_3 grad(phi^SD + phi^Q) - [0, 0, phi^SD + phi^Q],
 *     lap u = lap u^S + 2 d_3 grad(phi^SD + phi^Q).
 *   The plan keeps child plans (Stokeslet or RPY, Laplace charges + dipoles, and for RPY
 *   Laplace quadrupoles; the same p, q and options); kafmm_tree_info,
 *   kafmm_phase_times and kafmm_get_counters report the first child; batches,
 *   kafmm_autotune, the tree queries, kafmm_get_operator and the RPY velocity calls answer
 *   KAFMM_ERR_ARG. */
typedef enum {
  KAFMM_BC_OPEN = 0,
  KAFMM_BC_PX = 1,
  KAFMM_BC_PXY = 2,
  KAFMM_BC_PXYZ = 3,
  KAFMM_BC_WALL = 4,
  KAFMM_BC_WALL_PX = 5,
  KAFMM_BC_WALL_PXY = 6
} kafmm_bc;

typedef enum { KAFMM_F32 = 0, KAFMM_F64 = 1 } kafmm_dtype;

/* Option keys for kafmm_set_option. */
enum {
  /* Arithmetic of the evaluation (default KAFMM_PREC_MIXED):
   *   KAFMM_PREC_FP64  -- every step in FP64 (the plain reference form);
   *   KAFMM_PREC_FP32  -- FP32 everywhere, every gather-GEMM on CUDA cores;
   *   KAFMM_PREC_MIXED -- FP32 near field and source/target kernels; the gather-GEMMs on
   *                       tcgen05 tensor cores with FP32 accumulation: M->L in split BF16x3
   *                       or TF32x3 (KAFMM_OPT_TC_SPLIT), M->M, L->L and the pseudo-inverse
   *                       factors in TF32x3.  Tables on the tensor cores: the four-channel
   *                       Laplace table and single-column tables with rows per box a multiple
   *                       of 8 (G, Laplace, StokesPVel for even p); others stay on CUDA cores. */
  KAFMM_OPT_PRECISION = 1,
  /* ML-tree kernel table of the Stokeslet and RPY problems (default KAFMM_ML_L4):
   *   KAFMM_ML_G  -- the Stokeslet G on M and L points (Tables tab:ktab_rpy, tab:ktab_reg);
   *   KAFMM_ML_L4 -- four Laplace channels per point (charges f and (y - c).f about the box
   *                  centre c); a linear, low-dimensional ML-tree table in the sense of
   *                  Sec. II.  Ignored for Laplace; periodic boundaries always use KAFMM_ML_G. */
  KAFMM_OPT_ML_VARIANT = 2,
  /* cudaStream_t, passed as an integer. */
  KAFMM_OPT_STREAM = 3,
  /* 1: evaluate only the near field (U-list S->T sums).  Default 0. */
  KAFMM_OPT_NEAR_ONLY = 4,
  /* 1: Kahan-compensated accumulation in the FP32 near field.  Default 0. */
  KAFMM_OPT_KAHAN = 5,
  /* Split format of the tensor-core M->L in KAFMM_PREC_MIXED (default KAFMM_TC_AUTO): each
   * operand x = hi + lo in tf32 (or bf16) and each product hi*hi + hi*lo + lo*hi.  Measured
   * error of the mixed form against the FP64 form (Stokeslet, N = 262144 uniform): TF32x3
   * 4.7e-6..5.7e-6 for p = 6..10; BF16x3 4.2e-5 (p = 6), 1.1e-5 (p = 8), 6.6e-6 (p = 10),
   * 7e-6 against the direct sum at p = 12, at about 0.7x the time.  AUTO takes BF16x3 for
   * p >= 10 and TF32x3 below on check potentials; in compressed coordinates (KAFMM_OPT_COMPRESS)
   * BF16x3 up to 512 compressed rows for p >= 10 and up to 256 rows for p = 8, 9, else TF32x3
   * (the orthonormal projections keep BF16 rounding out of the directions the pseudo-inverses
   * amplify: 512 Stokeslet problems at p = 8, worst problem 6.2e-6 against the FP64 form). */
  KAFMM_OPT_TC_SPLIT = 6,
  /* 1 (default): kafmm_eval synchronises the plan's stream before it returns and reports a
   * device-side timeout as KAFMM_ERR_TIMEOUT.  0: with device arrays kafmm_eval only enqueues
   * work on the plan's stream and returns (no host synchronisation, no device allocation after
   * the first call for the current points), so a second and later call can be captured into a
   * CUDA graph and replayed; device-side timeouts then accumulate in a status word that
   * kafmm_status reports.  Host arrays are always handled synchronously. */
  KAFMM_OPT_SYNC = 7,
  /* Pipeline depth of the tensor-core gather-GEMM (mixed form): 2 stages of 96 KB (operand rows
   * of 128 bytes, 64 bf16 / 32 tf32 k-values per stage) or 4 stages of 48 KB (64-byte rows, half
   * the k-values per stage).  Both issue the same MMAs in the same order and give bit-identical
   * results.  Default 2: 4 measured slower on GB300 (Stokeslet N = 262144: M->L 7.1 ms against
   * 5.3 ms at p = 10, 33 ms against 25 ms at p = 8). */
  KAFMM_OPT_TC_STAGES = 8,
  /* Most slot ranges a tile of the tensor-core gather-GEMM is split into when the grid would
   * not fill the GPU (M->L offsets, M->M child octants; partial sums combined in a fixed
   * order): 1, 2, 4 (default) or 8. */
  KAFMM_OPT_TC_RANGES = 9,
  /* RPY with one shared point set: 1 = kafmm_eval leaves the U-list pairs within contact
   * (r <= b_i + b_j, the radii of the two points) out of the kernel sum and
   * kafmm_rpy_velocity adds their whole pair mobility; 0 (default) = the kernel sum holds every
   * pair and kafmm_rpy_velocity corrects contact pairs by (overlap form - far form), as
   * Sec. II.B describes.  Use 1 for sphere velocities of dense suspensions in the FP32 and
   * mixed forms: the far form of very close pairs (a^2 / r^3) is orders of magnitude larger
   * than the velocity and cancels in the correction beyond FP32 precision (2^20 clustered
   * spheres, mixed form, sampled velocities vs brute force: 2.5e-4 with 0, 1.3e-5 with 1; FP64
   * form 1.7e-6).  With 1, kafmm_eval's [u, lap u] is the kernel sum without those pairs; set it
   * before kafmm_eval and keep it for the matching kafmm_rpy_velocity. */
  KAFMM_OPT_RPY_CONTACT = 10,
  /* How the tensor-core M->L groups target boxes into tiles (applied at the next
   * kafmm_set_points): 1 = tiles of one octant class carry whole V lists (every offset any of
   * their boxes has); 2 = tiles of one octant class and one neighbour of the parent (the 8
   * children of that colleague, Sec. II), each box's result a partial sum added to its
   * downward check in neighbour order by a combine pass; 0 (default) = 2 when the partials
   * (R x C floats per box and neighbour) fit in a quarter of the device memory, else 1.
   * Adaptive V lists are sparse and differ from box to box (2^18 clustered points: 45 of 189
   * offsets per box on average, 5735 distinct occupancies in 8810 boxes), so whole-list tiles
   * compute mostly empty columns (M->L of 2^20 clustered RPY points: 44.7 ms with 1, 22.6 ms
   * with 2; Stokeslet N = 262144 uniform, p = 10: 5.39 -> 4.42 ms).  kafmm_autotune times
   * both. */
  KAFMM_OPT_TC_TILING = 11,
  /* Limit of every device-side wait on an asynchronous copy or a pipeline stage, in
   * microseconds (default 2,000,000 = 2 s; 1 .. 60,000,000).  A wait that runs out records a
   * timeout (KAFMM_ERR_TIMEOUT from kafmm_eval or kafmm_status); the kernel then issues no
   * further copy, waits once more (same limit) for its copies in flight, skips the rest of its
   * work and returns, so the device stays usable.  No kernel traps. */
  KAFMM_OPT_WAIT_LIMIT_US = 12,
  /* Test aid (default -1 = off): a device-side wait that lasted at least this many
   * microseconds (0: every wait) records a timeout as above but completes normally, so the
   * results are unchanged while the status reaches the host. */
  KAFMM_OPT_WAIT_REPORT_US = 13,
  /* Test aid (default 0): 1 makes every block of the near-field kernel first wait on a barrier
   * that nothing completes, so the wait runs out after KAFMM_OPT_WAIT_LIMIT_US and the block
   * takes the wind-down path above (kafmm_eval returns KAFMM_ERR_TIMEOUT; the results of that
   * call are not valid). */
  KAFMM_OPT_TEST_STALL = 14,
  /* Mixed form on the tensor cores (default 2): 1 runs the ML tree in compressed coordinates,
   * 0 in check potentials (R rows per box).  The pseudo-inverse of Sec. II keeps the r singular
   * values above its cutoff, and every use of a check potential passes through it, so a box's
   * state can be its projection on the r leading left singular vectors (U^T times the check
   * potential) without changing the result in exact arithmetic: M->L, M->M, L->L and the
   * periodic operator become r x r matrices (r padded to 64; p = 10, Laplace table: 256 instead
   * of 488 rows, 256 instead of 512 k-values), the leaves' S->M potentials and the X-list
   * potentials are projected once, and the equivalent densities come from V S^+ applied to the
   * projections.  2 (default): as 1, and when rounding the larger rank down to a multiple of 64
   * keeps at least 90 % of it, only that many leading singular vectors are kept (p = 10: 192 of
   * 202), so no k-value of the tensor-core tiles is padding (Stokeslet N = 262144, p = 10:
   * M->L 1.27 -> 1.07 ms, error against the FP64 form 3.6e-6 -> 3.4e-6).  Applied at the next
   * kafmm_set_points (operators rebuilt). */
  KAFMM_OPT_COMPRESS = 15,
  /* Sources per staging buffer of the near-field kernel (two buffers: the copies of one batch
   * of U-list sources are in flight while the previous batch is evaluated).  0 (default): 20 KB
   * per buffer (640 FP32 Stokeslet sources); 64 .. 4096 otherwise; never fewer than the points
   * of one equivalent surface.  kafmm_autotune times 256, 640 and 1280. */
  KAFMM_OPT_LEAF_STAGE = 16,
  /* Consecutive tiles one CTA of the tensor-core gather-GEMM processes in turn: 1 (default),
   * 2 or 4.  With more than one, the TMEM allocation and barrier set-up are paid once per CTA
   * and a tile's output writes overlap the next tile's MMAs; fewer are used when the grid would
   * no longer fill the GPU twice.  Results are bit-identical for every value.
   * kafmm_autotune times all three. */
  KAFMM_OPT_TC_TILES = 17
};
enum { KAFMM_TC_TF32X3 = 0, KAFMM_TC_BF16X3 = 1, KAFMM_TC_AUTO = 2 };
enum { KAFMM_PREC_FP64 = 0, KAFMM_PREC_FP32 = 1, KAFMM_PREC_MIXED = 2 };
enum { KAFMM_ML_G = 0, KAFMM_ML_L4 = 1 };

/* Error codes. */
enum {
  KAFMM_OK = 0,
  KAFMM_ERR_ARG = -1,     /* invalid argument (sizes, enum values, null pointers)     */
  KAFMM_ERR_DOMAIN = -2,  /* a point outside [origin, origin + L)^3, or NaN / Inf     */
  KAFMM_ERR_CUDA = -3,    /* a CUDA runtime error (message holds the CUDA text)       */
  KAFMM_ERR_TIMEOUT = -4, /* a bounded device wait expired                           */
  KAFMM_ERR_NOMEM = -5,   /* device allocation failed                                */
  KAFMM_ERR_STATE = -6    /* call out of order (eval before set_points, ...)          */
};

/* Creates a plan: kernel, boundary condition, multipole order p (the paper's m, Sec. III:
 * 6(p-1)^2 + 2 equivalent points per surface, 2 <= p <= 16) and the leaf size q (a box is
 * split while it holds more than q points, Sec. III; 1 <= q <= 4096).  Builds the FP64
 * translation operators on the current CUDA device (pseudo-inverses by one-sided Jacobi
 * SVD, Sec. II; the periodic operator by Ewald lattice sums (PXYZ) or extrapolated image sums
 * (PX, PXY)).  *out receives the plan. */
int kafmm_plan(kafmm_kernel kernel, kafmm_bc bc, int p, int max_pts_per_leaf,
               kafmm_plan_t* out);

/* Sets one option (keys above).  Changing PRECISION or ML_VARIANT after kafmm_plan
 * rebuilds the operators; after set_points it also invalidates the tree (set_points must
 * be called again). */
int kafmm_set_option(kafmm_plan_t plan, int key, int64_t value);

/* The cube that holds all points: [origin, origin + L)^3 (default origin 0, L = 1). */
int kafmm_set_domain(kafmm_plan_t plan, const double origin[3], double L);

/* Sets sources y [n_src][3] and targets x [n_trg][3] (x == y with n_trg == n_src means one
 * shared set).  Builds the octree and the U/V/W/X lists on the device: Morton keys, radix
 * sort, level-by-level refinement, list construction (Sec. II, Sec. III).  Points outside
 * the domain give KAFMM_ERR_DOMAIN.  The plan keeps sorted copies; the caller's arrays
 * are not retained. */
int kafmm_set_points(kafmm_plan_t plan, const void* y, int64_t n_src, const void* x,
                     int64_t n_trg, int dtype);

/* Largest problem count of kafmm_set_points_batched. */
#define KAFMM_MAX_PROBLEMS 65536

/* Sets a batch of n_prob independent problems at once, each its own kernel sum of
 * Eq. kernelsumlinear (the paper evaluates one sum per call; a batch runs many uneven ones
 * in the same launches).  Problem k has the sources
 * y[src_offsets[k] .. src_offsets[k+1]) and the targets x[trg_offsets[k] .. trg_offsets[k+1]),
 * all in the same cube [origin, origin + L)^3, and interacts with nothing outside itself.
 * src_offsets and trg_offsets are HOST arrays of n_prob + 1 nondecreasing entries starting at
 * 0 (empty problems allowed); y and x are the concatenated points (host or device, as in
 * kafmm_set_points; x == y with equal offsets means one shared set per problem).  One forest is
 * built, one root per problem, and every later call (kafmm_eval, the tree queries) covers the
 * whole batch in the same launches as one problem: s and g of kafmm_eval are the concatenated
 * values in the same order.  1 <= n_prob <= KAFMM_MAX_PROBLEMS; n_prob > 1 needs
 * KAFMM_BC_OPEN and is not accepted by the RPY velocity calls (KAFMM_ERR_ARG). */
int kafmm_set_points_batched(kafmm_plan_t plan, int n_prob, const int64_t* src_offsets,
                             const int64_t* trg_offsets, const void* y, const void* x, int dtype);

/* Evaluates g [n_trg][k_t] from s [n_src][k_s] for the current points (overwrites g).
 * Upward pass S->M, M->M; downward pass M->L (V), S->L (X), L->L; leaves L->T, M->T (W),
 * S->T (U) -- Sec. II, Fig. kifmmgraph. */
int kafmm_eval(kafmm_plan_t plan, const void* s, void* g, int dtype);

/* Autotuner: for the current points and the source values s (device arrays; g receives the
 * values of the last trial), times kafmm_eval for every combination of KAFMM_OPT_TC_TILING
 * (2, 1; the work lists are rebuilt for each and the host time of that build is added to the
 * score), KAFMM_OPT_TC_STAGES (2, 4) and KAFMM_OPT_TC_RANGES (1, 2, 4, 8), best of two runs
 * each (tensor-core plans only), then the near-field staging KAFMM_OPT_LEAF_STAGE (256, 640,
 * 1280 sources per buffer) on the leaf phase alone, and keeps the fastest in the plan; with
 * KAFMM_OPT_TC_TILES (1, 2, 4) in the tensor-core combinations.  chosen (host, may be NULL,
 * 5 entries) receives {stages, ranges, tiling, leaf stage, tiles per CTA}.  Call it again
 * when the tree changes much. */
int kafmm_autotune(kafmm_plan_t plan, const void* s, void* g, int dtype, int64_t* chosen);

/* Synchronises the plan's stream and reports (then clears) the device status accumulated by
 * asynchronous kafmm_eval calls (KAFMM_OPT_SYNC = 0): KAFMM_ERR_TIMEOUT if a bounded device
 * wait expired in any of them, else 0. */
int kafmm_status(kafmm_plan_t plan);

/* RPY only (Eq. RPYtrgvel and the overlap post-processing of Sec. II.B): from the kernel
 * sum g = [u, lap u] ([n_trg][6], as returned by kafmm_eval) and the target radii a
 * [n_trg], writes the sphere velocities ua [n_trg][3] = u + a^2/6 lap u, corrected for every
 * overlapping pair (|x - y| <= a + b) by the difference between the overlap-regularised
 * pair mobility and the far form.  Requires the source values s of the last kafmm_eval
 * ([n_src][4], passed again) so the pass can read forces and radii. */
int kafmm_rpy_velocity(kafmm_plan_t plan, const void* s, const void* a, const void* g,
                       void* ua, int dtype);

/* Same result as kafmm_rpy_velocity, for callers that cannot allocate device memory during
 * the call: for instance an application whose own pool allocator has reserved the device
 * memory up front, or one that must not trigger the implicit device-wide synchronisation of
 * cudaMalloc / cudaFree while other streams run.  The paper has no counterpart: this is a
 * library convenience.  It calls no cudaMalloc, cudaFree or allocating library routine
 * (counter 7 of kafmm_get_counters does not move); its work arrays live in one fixed 32 MiB
 * device array that every GPU loading the library holds until the process exits.  Limit: the
 * work arrays take 32 bytes per source and 8 per target in FP64 (16 and 4 in FP32) plus 2 MiB
 * of cell table, so about 780,000 points of one shared set in FP64 and 1.5 million in FP32;
 * larger sets return KAFMM_ERR_ARG with the sizes in the message (use kafmm_rpy_velocity).
 * All pointers must be device pointers (host arrays would need staging copies).  The first
 * call in a CUDA context (once per device, and again after cudaDeviceReset replaced the
 * context) looks the array up with that device current; make that first call before any
 * stream capture.  Every call uses the same array and keeps its contents, so calls that
 * overlap on the GPU (other threads, other streams) race. */
int kafmm_rpy_velocity_noalloc(kafmm_plan_t plan, const void* s, const void* a, const void* g,
                               void* ua, int dtype);

/* Tree and list statistics of the current points (host array info[n], up to 16 entries):
 * 0 boxes, 1 leaves, 2 levels, 3 U entries, 4 V entries, 5 W entries, 6 X entries,
 * 7 near-field pairs (sum over U of n_trg(B) n_src(A)), 8 max points in a leaf,
 * 9 problems (1 unless set by kafmm_set_points_batched). */
int kafmm_tree_info(kafmm_plan_t plan, int64_t* info, int n);

/* Copies the tree to host arrays (each may be NULL): level[nbox], anchor[nbox][3],
 * parent[nbox], leaf[nbox] (0/1), and the list kind (0 U, 1 V, 2 W, 3 X) as CSR:
 * offsets[nbox + 1], entries[n_entries] = source box index, shifts[n_entries] = image
 * shift code (sx+1) + 3 (sy+1) + 9 (sz+1).  Boxes are numbered level by level, in Morton
 * order inside a level (a batch: ordered by problem, then Morton; the root of problem k is
 * box k).  Sizes come from kafmm_tree_info. */
int kafmm_get_tree(kafmm_plan_t plan, int32_t* level, int32_t* anchor, int32_t* parent,
                   int8_t* leaf);
int kafmm_get_list(kafmm_plan_t plan, int kind, int64_t* offsets, int32_t* entries,
                   int8_t* shifts);

/* Times of the phases of the last set_points + eval, in milliseconds (CUDA events on the
 * plan's stream): 0 tree, 1 lists, 2 upward, 3 M->L, 4 downward rest, 5 near field,
 * 6 whole eval; 7 host time of set_points' work-list build (tiles of the gather-GEMMs, read
 * back from the tree; the device waits meanwhile).  Host array t[n], up to 8 entries. */
int kafmm_phase_times(kafmm_plan_t plan, double* t, int n);

/* Counters of the last calls (host array c[n], up to 12 entries): 0 kernel launches of the
 * last kafmm_set_points, 1 kernel launches of the last kafmm_eval, 2 whether M->L ran on the
 * tcgen05 tensor cores (0/1), 3 launches of set_points + eval, 4 the split format in use
 * (KAFMM_TC_TF32X3 or KAFMM_TC_BF16X3; -1 without tensor cores), 5 the M->L tiling of the
 * current points (1 whole V lists, 2 per parent neighbour; see KAFMM_OPT_TC_TILING), 6 the
 * number of M->L tiles, 7 device allocations (cudaMalloc) the library has made in this process
 * so far, over all plans, 8 rows of the compressed coordinates (0: check potentials; see
 * KAFMM_OPT_COMPRESS), 9 and 10 the singular values kept by the upward and downward
 * pseudo-inverses. */
int kafmm_get_counters(kafmm_plan_t plan, int64_t* c, int n);

/* Copies one precomputed translation operator to the host as FP64 (row-major R x R, R = the
 * ML rows of the plan: 6(p-1)^2+2, times 3 for the Stokeslet G table, times 4 for the
 * StokesPVel table).  slot: 0..342 M->L by
 * offset (ox+3) + 7(oy+3) + 49(oz+3); 343..350 M->M by child octant; 351..358 L->L by child
 * octant; 359/360 the upward pseudo-inverse factors S^+U^T and V; 361/362 the downward ones;
 * 363 the periodic far-image operator.  All are composed with the pseudo-inverse and
 * described in units of the box half-width.  Values come from the plan's precision (FP32
 * plans return their FP32 operators widened). */
int kafmm_get_operator(kafmm_plan_t plan, int slot, double* out);

/* Measurement aid, not part of the method (the paper has no counterpart): runs one
 * micro-benchmark on the current CUDA device and writes its rate to *rate (operations per
 * second) and the duration of the timed launch to *ms (may be NULL).  what: 0 FP32 FMA
 * (2 flop each), 1 MUFU reciprocal square root (one operation each), 2 FP64 FMA (2 flop each),
 * 3 tcgen05 MMA kind::tf32 and 4 kind::f16 with bf16 operands (dense flops, M = 128, N = 256,
 * one CTA per SM).  These are the denominators of the near-field, FP64 and TF32 rooflines.
 * Returns KAFMM_ERR_ARG for another value of what. */
int kafmm_measure_peak(int what, double* rate, double* ms);

/* Releases the plan and all device memory it owns. */
int kafmm_destroy(kafmm_plan_t plan);

/* Last error message of the plan (or of the last failed kafmm_plan when plan is NULL). */
const char* kafmm_last_error(kafmm_plan_t plan);

#ifdef __cplusplus
}
#endif
#endif /* KAFMM_H */
