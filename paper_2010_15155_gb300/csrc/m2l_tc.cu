// M->L translations on the tcgen05 tensor cores (sm_103a) in split precision (BF16x3 or
// TF32x3) with FP32 accumulation in tensor memory.
//
// The V list of a box B (Sec. II: children of the parent's colleagues not adjacent to B) lies
// at up to 189 of the 316 offsets o in [-3,3]^3 \ [-1,1]^3; with the pseudo-inverse folded in,
// each offset is one dense operator T_o (R x R) applied to the check potentials of the source
// box.  Output-stationary form: a CTA owns 2 x 128 check rows x 32 target boxes of one octant
// class (4 channels each -> N = 128 columns; one TMEM accumulator per 128-row block) and
// accumulates
//     D[rows, (box, ch)] = sum_o T_o[rows, :] * shift_o(up_check[box + o])[:, ch]
// over all offsets.  A (the operator) arrives by TMA (128B swizzle, K-major); B (gathered,
// re-referenced to the target centre and split into hi/lo) is written to shared memory by
// producer warps in the same canonical layout: one warp per source box and k-chunk, each lane
// two (bf16) or one (tf32) consecutive k of all four channels, so the gather is coalesced and
// every 32-bit store instruction fills one whole swizzled 128-byte row (conflict-free).  Each operand is split x = hi + lo in the
// MMA format (tf32 or bf16) and each product is taken as hi*hi + hi*lo + lo*hi.
// A group of k-values (counted over the tile's offsets in order; its length is chosen per
// table on the host) is accumulated in a fresh TMEM accumulator and then added into a TMEM sum
// by the epilogue warps, so no FP32 accumulation chain inside the tensor core is longer than
// one group.
//
// Warp roles (448 threads): 0-3 epilogue (TMEM lane quarters), 4-11 B producers, 12 TMA,
// 13 TMEM allocation + MMA issue.  Every wait is bounded (%globaltimer, 2 s by default); on
// expiry the kernel records ST_TIMEOUT and winds down without trapping.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "plan.cuh"
#include "tcgen05.cuh"

namespace kafmm {

namespace tc {

// A CTA owns RB row blocks of BM = 128 operator rows and NB = 64 / RB target boxes
// (BN = 256 / RB columns, four channels per box): all row blocks multiply the same gathered B
// tile, so every B element the producers build feeds RB x 3 MMAs.  RB = 2 when the number of
// row blocks is even, else 1 (a lone last block would waste a pair's B tile).  Shared memory
// per stage (96 KB) and TMEM (RB x BN accumulator + running-sum columns) are the same for both.
//
// Pipeline: the operand rows of a stage are SWB bytes wide, stored with the SWB-byte swizzle:
// SWB = 128 gives two stages of 96 KB, SWB = 64 four stages of 48 KB (half the k per stage,
// twice the stages in flight, the same MMAs in the same order).
//
// Single-column tables (the Stokeslet G table and the Laplace table, CH = 1): a CTA owns
// BN = 256 / RB target boxes, one column each, and the B producers copy contiguous k-runs of
// each source box (no re-reference: those tables have no centre-dependent channel).
template <int RB, int SWB, int CH>
struct Shape {
  static constexpr int BN = 256 / RB, NB = BN / CH;
  static constexpr int A_TILE = BM * SWB;                // 128 rows per split and row block
  static constexpr int A_STAGE = RB * 2 * A_TILE;        // A hi/lo of all row blocks
  static constexpr int B_TILE = BN * SWB;                // BN rows per split
  static constexpr int STAGE_BYTES = A_STAGE + 2 * B_TILE;
  static constexpr int STAGES = 196608 / STAGE_BYTES;
  static_assert(STAGE_BYTES == 768 * SWB, "96 KB (SWB 128) or 48 KB (SWB 64) per stage");
};
// dynamic shared memory: 192 KB of stages + alignment
constexpr int SMEM_BYTES = 196608 + 1024;   // stages + alignment to 1024 bytes
// non-M->L modes drain the TMEM accumulator into the running sum after every 64 k-values (one
// 128-byte chunk): the pseudo-inverse factors sum with heavy cancellation, and accumulating two
// such chunks per drain measured 1.3e-5 against the FP64 form at p = 8 (8.7e-6 with one;
// Stokeslet N = 262144)
template <int SWB>
constexpr int aux_drain() { return 128 / SWB; }
// M->L accumulation groups.  The tensor core's FP32 accumulation loses accuracy over long
// chains of these cancelling sums.  Single-column tables drain every 256 k-values: the
// Stokeslet G table at p = 12 (2184 k per offset), TF32x3, measured 1.5e-5 against the FP32
// CUDA-core form with one drain per offset, 2.2e-6 with one per 256 k (1 % slower) and 1.3e-6
// with one per 64 k.  The four-channel table (488 k per offset at p = 10) drains after one
// offset in TF32x3 and after two in BF16x3 (measured 7.6e-6 against the FP64 form at p = 10;
// one drain per 256 k gives 6.1e-6 but costs 5 % of the M->L time).  A group may span two
// offsets (the sum is linear).
constexpr int M2L_GROUP_K = 256;
// Most tiles one CTA processes in turn (KAFMM_OPT_TC_TILES): the TMEM allocation and barrier
// set-up are paid once, and a tile's output writes overlap the next tile's MMAs.
constexpr int TC_TMAX = 4;
constexpr int THREADS = 448;
constexpr int NPROD = 256;
constexpr int W_TMA = 12, W_MMA = 13;

constexpr uint32_t TMEM_COLS = 512;         // [0,256) accumulators, [256,512) running sums
constexpr uint32_t SUM_COL = 256;           // row block r: accumulator r*BN, sum SUM_COL + r*BN

// Modes of the gather-GEMM: target box b (of a tile), slots s, out[b] (+)= sum_s
// T_s * shift_s(in[src(b, s)]):
//   TC_M2L    s = V slot of the parent's 6^3 neighbourhood, src = V entry, T = M->L(offset)
//   TC_M2M    s = child octant, src = child s (b a parent), T = M->M(s)
//   TC_L2L    one slot, src = parent of b, T = L->L(octant class of b)
//   TC_APPLY  one slot, src = b, T = a fixed operator (pseudo-inverse factor), no shift
// shift_s re-references the fourth channel from the source box centre to the target's.
enum TcMode { TC_M2L = 0, TC_M2M = 1, TC_L2L = 2, TC_APPLY = 3 };
// Output: TC_STORE out = value (or the partial of offset range z), TC_ADD out += value,
// TC_SCALE out = value x half-width of b.
enum TcWrite { TC_STORE = 0, TC_ADD = 1, TC_SCALE = 2 };

struct Args {
  TreeView t;
  double L;
  const float* up;        // input [nbox][R][CH]
  float* dn;              // output [nbox][R][CH]; with nsplit > 1: [nsplit] partials
  int64_t part_stride;    // floats between partial buffers
  int nsplit;
  const int4* tiles;
  const int* boxlist;
  const int32_t* vtab;
  unsigned* status;
  WaitLimits lim;
  // Rout: operator rows = output rows per box; Rin: input rows per box (the k extent); Rop:
  // rows per operator in the tensor map (Rout, or more with padding)
  int Rout, Rin, Rop, nchunk;
  int mode, write;
  int op;                 // TC_APPLY: operator index in the tensor map
  int group;              // TC_M2L: k-chunks per TMEM accumulation group
  // TC_M2L tiles of one parent neighbour (tile.w = g + 1): box j of the tile writes partial
  // part[tile.x + j] of dn (R x CH floats each) instead of its own box
  const int* part;
  int qrow4;              // StokesPVel table, TC_SCALE: rows 4k+3 (q) take the half-width twice
  int ntiles;             // tiles of the launch
  int tpc;                // consecutive tiles per CTA (1 .. TC_TMAX)
};

// Slots of a mode (upper bound of the slot index), the operator of slot s in the tensor map
// (M->L map for TC_M2L, the auxiliary map otherwise) and the re-reference shift of slot s in
// units of the target box's side.
__device__ __forceinline__ int mode_slots(int mode) {
  return mode == TC_M2L ? 216 : (mode == TC_M2M ? 8 : 1);
}
__device__ __forceinline__ int slot_op(const Args& a, int s, int cls) {
  if (a.mode == TC_M2L) {
    int ox = s % 6 - 2 - (cls & 1), oy = (s / 6) % 6 - 2 - ((cls >> 1) & 1), oz = s / 36 - 2 - ((cls >> 2) & 1);
    return m2l_index(ox, oy, oz);
  }
  if (a.mode == TC_M2M) return OP_M2M - OP_M2M + s;
  if (a.mode == TC_L2L) return OP_L2L - OP_M2M + cls;
  return a.op;
}
__device__ __forceinline__ void slot_shift(int mode, int s, int cls, float& fx, float& fy, float& fz) {
  if (mode == TC_M2L) {
    fx = (float)(s % 6 - 2 - (cls & 1));
    fy = (float)((s / 6) % 6 - 2 - ((cls >> 1) & 1));
    fz = (float)(s / 36 - 2 - ((cls >> 2) & 1));
  } else if (mode == TC_M2M) {  // child centre - parent centre
    fx = (s & 1) ? 0.25f : -0.25f;
    fy = (s & 2) ? 0.25f : -0.25f;
    fz = (s & 4) ? 0.25f : -0.25f;
  } else if (mode == TC_L2L) {  // parent centre - child centre
    fx = (cls & 1) ? -0.5f : 0.5f;
    fy = (cls & 2) ? -0.5f : 0.5f;
    fz = (cls & 4) ? -0.5f : 0.5f;
  } else {
    fx = fy = fz = 0.f;
  }
}
// Source box of target b at slot s, or -1.
__device__ __forceinline__ int slot_src(const Args& a, int b, int s) {
  if (b < 0) return -1;
  if (a.mode == TC_M2L) {
    int32_t e = a.vtab[(int64_t)b * 216 + s];
    return e != LIST_EMPTY ? entry_box(e) : -1;
  }
  if (a.mode == TC_M2M) return a.t.child[b * 8 + s];
  if (a.mode == TC_L2L) return a.t.parent[b];
  return b;
}

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Bounded parity wait: false (ST_TIMEOUT recorded, the CTA's bail flag set) once lim.hard_ns
// passed, or when another warp has already bailed; a wait of lim.report_ns or longer that
// completes records ST_TIMEOUT too (report only).
__device__ __forceinline__ bool wait_parity(uint64_t* bar, uint32_t parity, unsigned* status,
                                            int* bail, const WaitLimits& lim) {
  const uint32_t addr = smem_u32(bar);
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(addr, parity)) {
      if (lim.report_ns != ~0ull && global_ns() - t0 >= lim.report_ns)
        atomicOr(status, (unsigned)ST_TIMEOUT);
      return true;
    }
    if (*(volatile int*)bail) return false;
    if (global_ns() - t0 > lim.hard_ns) {
      atomicOr(status, (unsigned)ST_TIMEOUT);
      *(volatile int*)bail = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// Read-only 256-bit load of two consecutive float4 (address 32-byte aligned).
__device__ __forceinline__ void ld_nc_v8(const float4* p, float4& a, float4& b) {
  asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
               : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
               : "l"(p));
}

__device__ __forceinline__ void st_shared_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.b32 [%0], %1;\n" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, const uint32_t (&v)[4]) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "r"(v[0]), "r"(v[1]), "r"(v[2]),
               "r"(v[3])
               : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}

template <int SPLIT, int RB, int SWB, int CH>
__global__ void __launch_bounds__(THREADS, 1)
    k_m2l_tc(const __grid_constant__ CUtensorMap tmap, Args a) {
  constexpr int BK = SWB / Fmt<SPLIT>::ES, MK = Fmt<SPLIT>::MK;
  using S = Shape<RB, SWB, CH>;
  constexpr int BN = S::BN, NB = S::NB, B_BYTES = S::B_TILE, A_BYTES = S::A_TILE,
                A_STAGE = S::A_STAGE, STAGE_BYTES = S::STAGE_BYTES, STAGES = S::STAGES;
  constexpr int PROD_WARPS = NPROD / 32;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full[4], empty[4], acc_full, acc_empty;
  __shared__ uint32_t tmem_base;
  __shared__ int bail;
  // the CTA's tiles (a.tpc consecutive tiles): box records, active slots and the prefix tables
  // that map the CTA's iteration index (tile after tile, slot after slot, k-chunk after k-chunk)
  // and its accumulation groups to their tile
  __shared__ int sbox[TC_TMAX][NB];
  __shared__ int sout[TC_TMAX][NB];          // output record of box j (its box, or its partial)
  __shared__ float sside[TC_TMAX][NB];
  __shared__ int slots_all[TC_TMAX * 216];
  __shared__ int slot_any[216];
  __shared__ int t_n[TC_TMAX], t_s0[TC_TMAX], t_cls[TC_TMAX], t_it0[TC_TMAX + 1], t_g0[TC_TMAX + 1];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int R = a.Rout, Rin = a.Rin;
  const int row0 = blockIdx.y * (RB * BM);
  // row blocks of this CTA that hold operator rows (the last pair may have only one)
  const int nrb = min(RB, (R - row0 + BM - 1) / BM);
  const int T = min(a.tpc, TC_TMAX);
  const int nchunk = a.nchunk;
  // accumulation groups: iterations accumulated in TMEM before the epilogue adds them into the
  // running sum (M->L: a.group chunks; other modes: one 128-byte chunk); a group never spans
  // two tiles
  const int GI = a.mode == TC_M2L ? a.group : aux_drain<SWB>();
  const int nsmax = mode_slots(a.mode);

  if (threadIdx.x == 0) {
    bail = 0;
    for (int st = 0; st < STAGES; ++st) {
      mbar_init(&full[st], PROD_WARPS + 1);   // one arrival per producer warp + the TMA's
      mbar_init(&empty[st], 1);
    }
    mbar_init(&acc_full, 1);
    mbar_init(&acc_empty, 128);
  }
  int s_run = 0;   // entries of slots_all used so far (warp 0)
  for (int t = 0; t < T; ++t) {
    const int ti = blockIdx.x * T + t;
    const int4 tile = ti < a.ntiles ? a.tiles[ti] : make_int4(0, 0, 0, 0);
    const int cls = tile.z;
    const int grp = a.mode == TC_M2L ? tile.w - 1 : -1;   // parent neighbour, -1 = whole V lists
    for (int j = threadIdx.x; j < NB; j += THREADS) {
      int b = j < tile.y ? a.boxlist[tile.x + j] : -1;
      sbox[t][j] = b;
      sout[t][j] = grp >= 0 && b >= 0 ? a.part[tile.x + j] : b;
      sside[t][j] = b >= 0 ? (float)(a.L / (double)(1 << a.t.level[b])) : 0.f;
    }
    for (int k = threadIdx.x; k < 216; k += THREADS) slot_any[k] = 0;
    if (threadIdx.x == 0) t_cls[t] = cls;
    __syncthreads();
    // active slots: some box of the tile has a source there; candidates: the 8 children of
    // parent neighbour grp, or all slots of the mode
    const int ncand = grp >= 0 ? 8 : nsmax;
    for (int e = threadIdx.x; e < ncand * NB; e += THREADS) {
      int k = e / NB, j = e % NB;
      if (grp >= 0)
        k = (2 * (grp % 3) + (k & 1)) + 6 * (2 * ((grp / 3) % 3) + ((k >> 1) & 1)) +
            36 * (2 * (grp / 9) + (k >> 2));
      bool inner = false;
      if (a.mode == TC_M2L) {
        int ox = k % 6 - 2 - (cls & 1), oy = (k / 6) % 6 - 2 - ((cls >> 1) & 1),
            oz = k / 36 - 2 - ((cls >> 2) & 1);
        inner = abs(ox) <= 1 && abs(oy) <= 1 && abs(oz) <= 1;
      }
      if (!inner && slot_src(a, sbox[t][j], k) >= 0) slot_any[k] = 1;
    }
    __syncthreads();
    if (warp == 0) {  // active offsets (ballot compaction), then this CTA's share (blockIdx.z)
      int* list = slots_all + s_run;
      int ns = 0;
      for (int k0 = 0; k0 < nsmax; k0 += 32) {
        const int k = k0 + lane;
        const bool on = k < nsmax && slot_any[k];
        const unsigned m = __ballot_sync(0xffffffffu, on);
        if (on) list[ns + __popc(m & ((1u << lane) - 1u))] = k;
        ns += __popc(m);
      }
      __syncwarp();
      const int z = blockIdx.z, nz = a.nsplit;
      const int q0 = (int)((int64_t)ns * z / nz), q1 = (int)((int64_t)ns * (z + 1) / nz);
      int tmp[7];   // the share moves to the front (at most 216 entries, 7 per lane)
      int cnt = 0;
      for (int k = q0 + lane; k < q1; k += 32) tmp[cnt++] = list[k];
      __syncwarp();
      cnt = 0;
      for (int k = q0 + lane; k < q1; k += 32) list[k - q0] = tmp[cnt++];
      if (lane == 0) {
        t_n[t] = q1 - q0;
        t_s0[t] = s_run;
      }
      s_run += q1 - q0;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    t_it0[0] = 0;
    t_g0[0] = 0;
    for (int t = 0; t < T; ++t) {
      const int n_it = t_n[t] * nchunk;
      t_it0[t + 1] = t_it0[t] + n_it;
      t_g0[t + 1] = t_g0[t] + (n_it + GI - 1) / GI;
    }
  }
  if (warp == W_MMA) {  // TMEM allocation (whole warp)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int total = t_it0[T];
  // tile of iteration it (iterations run tile after tile), its slot and its k-chunk
  auto tile_of = [&](int it) {
    int t = 0;
    while (t + 1 < T && it >= t_it0[t + 1]) ++t;
    return t;
  };
  auto slot_of = [&](int t, int it) { return slots_all[t_s0[t] + (it - t_it0[t]) / nchunk]; };
  auto chunk_of = [&](int t, int it) { return (it - t_it0[t]) % nchunk; };

  if (warp == W_TMA) {
    // ---------------- TMA producer of A (operator rows, hi and lo) ----------------
    if (lane == 0) {
      for (int it = 0; it < total; ++it) {
        int st = it % STAGES;
        if (it >= STAGES && !wait_parity(&empty[st], ((it / STAGES) - 1) & 1, a.status, &bail, a.lim)) break;
        const int t = tile_of(it);
        int s = slot_of(t, it), c = chunk_of(t, it);
        int op = slot_op(a, s, t_cls[t]);
        unsigned char* base = smem + st * STAGE_BYTES;
        uint32_t bar = smem_u32(&full[st]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar),
                     "r"(nrb * 2 * A_BYTES)
                     : "memory");
        for (int r = 0; r < nrb; ++r)
          for (int h = 0; h < 2; ++h) {
            int y = (op * 2 + h) * a.Rop + row0 + r * BM;
            int x = c * BK;
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], "
                "[%1, {%2, %3}], [%4];\n" ::"r"(smem_u32(base + (r * 2 + h) * A_BYTES)),
                "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(x), "r"(y), "r"(bar)
                : "memory");
          }
      }
    }
  } else if (warp >= 4 && warp < W_TMA) {
    if constexpr (CH == 1) {
      // ---------------- B producers, single-column tables: gather, split, swizzle ----------------
      // Row n of B = target box n of the tile: the BK k-values of this chunk of its source box,
      // contiguous in memory.  LPR lanes share a row, each loading 8 consecutive k (32 bytes)
      // and writing its 16-byte chunk(s) of the swizzled row (one per 8 bf16, two per 8 tf32);
      // a warp instruction covers BPI boxes, so the loads are contiguous runs and each
      // shared-memory phase of 8 lanes fills whole 128-byte rows (conflict-free).
      static_assert(SWB == 128, "single-column tables use 128-byte rows");
      constexpr int LPR = BK / 8;                      // lanes per row
      constexpr int BPI = 32 / LPR;                    // boxes per warp instruction (4 or 8)
      constexpr int UPW = NB / PROD_WARPS;             // boxes per producer warp per stage
      constexpr int LPS = UPW / BPI;                   // boxes per lane per stage
      constexpr int UH = LPS / 2;                      // boxes per lane per half stage
      static_assert(UH >= 1 && LPS == 2 * UH, "two half stages");
      const int pw = warp - 4;
      const int bsel = lane / LPR, wd = lane % LPR;
      auto box_of = [&](int ul) { return pw * UPW + ul * BPI + bsel; };
      int srcb[LPS];
      int cur_slot = -1;
      auto load_half = [&](int it, int h, float4 (&q)[UH][2]) {
        const int t = tile_of(it);
        int s = slot_of(t, it), c = chunk_of(t, it);
        if (t * 256 + s != cur_slot) {
#pragma unroll
          for (int ul = 0; ul < LPS; ++ul) srcb[ul] = slot_src(a, sbox[t][box_of(ul)], s);
          cur_slot = t * 256 + s;
        }
        const int k0 = c * BK + wd * 8;
        const bool kin = k0 < Rin;   // Rin a multiple of 8: a lane's 8 k are all in or all out
#pragma unroll
        for (int u = 0; u < UH; ++u) {
          int sb = srcb[h * UH + u];
          if (sb >= 0 && kin) {
            ld_nc_v8(reinterpret_cast<const float4*>(a.up + (int64_t)sb * Rin + k0), q[u][0], q[u][1]);
          } else {
            q[u][0] = make_float4(0.f, 0.f, 0.f, 0.f);
            q[u][1] = q[u][0];
          }
        }
      };
      auto store_half = [&](int it, int h, const float4 (&q)[UH][2]) {
        const int st = it % STAGES;
        const uint32_t bhi = smem_u32(smem + st * STAGE_BYTES + A_STAGE);
        const uint32_t blo = bhi + B_BYTES;
#pragma unroll
        for (int u = 0; u < UH; ++u) {
          const int n = box_of(h * UH + u);
          const uint32_t row = (uint32_t)(n * SWB);
          const float v[8] = {q[u][0].x, q[u][0].y, q[u][0].z, q[u][0].w,
                              q[u][1].x, q[u][1].y, q[u][1].z, q[u][1].w};
          if (SPLIT == SPLIT_TF32) {
#pragma unroll
            for (int g = 0; g < 2; ++g) {
              uint32_t hw[4], lw[4];
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                float hf = tf32_rn(v[4 * g + t]);
                hw[t] = __float_as_uint(hf);
                lw[t] = __float_as_uint(tf32_rn(v[4 * g + t] - hf));
              }
              const uint32_t off = row + ((uint32_t)((2 * wd + g) ^ (n & 7)) << 4);
              st_shared_v4(bhi + off, hw);
              st_shared_v4(blo + off, lw);
            }
          } else {
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * t], v[2 * t + 1]);
              float2 hf = __bfloat1622float2(h2);
              hw[t] = *reinterpret_cast<uint32_t*>(&h2);
              lw[t] = pack_bf16(v[2 * t] - hf.x, v[2 * t + 1] - hf.y);
            }
            const uint32_t off = row + ((uint32_t)(wd ^ (n & 7)) << 4);
            st_shared_v4(bhi + off, hw);
            st_shared_v4(blo + off, lw);
          }
        }
      };
      float4 qa[UH][2], qb[UH][2];
      if (total > 0) load_half(0, 0, qa);
      for (int it = 0; it < total; ++it) {
        int st = it % STAGES;
        load_half(it, 1, qb);
        int ok_wait = 1;
        if (lane == 0 && it >= STAGES)
          ok_wait = wait_parity(&empty[st], ((it / STAGES) - 1) & 1, a.status, &bail, a.lim) ? 1 : 0;
        if (!__shfl_sync(0xffffffffu, ok_wait, 0)) break;
        store_half(it, 0, qa);
        if (it + 1 < total) load_half(it + 1, 0, qa);
        store_half(it, 1, qb);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncwarp();
        if (lane == 0) arrive(&full[st]);
      }
    } else {
      // ---------------- B producers: gather, re-reference, split, swizzle ----------------
      // Work unit = one target box j of the tile: the BK k-values of this chunk of its source
      // box's four channels.  Lane l takes EPL consecutive k (two for bf16, one for tf32), i.e.
      // one 32-bit word of each of the 8 rows (4 channels x hi/lo) at word l of the 128-byte
      // row: the warp's loads are contiguous and each store instruction writes a full row.
      constexpr int EPL = 4 / Fmt<SPLIT>::ES;          // k values per lane (one 32-bit word)
      constexpr int WPR = SWB / 4;                     // 32-bit words per operand row
      constexpr int BPI = 32 / WPR;                    // boxes per warp instruction (1 or 2)
      constexpr int UPW = NB / PROD_WARPS;             // boxes per producer warp per stage
      constexpr int LPS = UPW / BPI;                   // boxes per lane per stage
      constexpr int UH = LPS / 2;                      // boxes per lane per half stage
      static_assert(UH >= 1 && LPS == 2 * UH, "two half stages");
      const int pw = warp - 4;
      const int bsel = lane / WPR;                     // which of the BPI boxes the lane serves
      const int wd = lane % WPR;                       // the lane's word of the row
      // Lane box ul (0..LPS-1) is u = bsel + BPI ul of the warp's boxes, j = pw + 8u, with rows
      // n = 4j + ch = (4 pw + ch) + 32u: the swizzled row of (u, ch) sits 32 u SWB bytes after that
      // of (0, ch), and the chunk swizzle depends on n & 7 only.  With two boxes per instruction
      // the second writes channel ch ^ 1 (rows of opposite parity: the other 64-byte bank half).
      auto swz_off = [&](int n) -> uint32_t {
        int x = SWB == 128 ? (n & 7) : ((n >> 1) & 3);
        return (uint32_t)((n >> 3) * (8 * SWB) + (n & 7) * SWB + ((((wd >> 2) ^ x) & (SWB / 16 - 1)) << 4) +
                          (wd & 3) * 4);
      };
      uint32_t roff[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        int ch = BPI == 2 ? (i ^ bsel) : i;
        roff[i] = swz_off(4 * pw + ch) + (uint32_t)(32 * SWB * bsel);
      }
      // source box (flat index into up) of each of this lane's boxes for the current slot, or -1
      int srcb[LPS];
      int cur_slot = -1;
      auto box_of = [&](int ul) { return pw + PROD_WARPS * (bsel + BPI * ul); };
      auto set_slot = [&](int t, int s) {
#pragma unroll
        for (int ul = 0; ul < LPS; ++ul) srcb[ul] = slot_src(a, sbox[t][box_of(ul)], s);
      };
      // Software pipeline over half stages (UH boxes per lane each): the loads of the next half
      // are in flight while the current half is converted, including the first half of the next
      // stage (registers only: no shared-memory stage is needed to issue them).
      auto load_half = [&](int it, int h, float4 (&q)[UH][EPL]) {
        const int t = tile_of(it);
        int s = slot_of(t, it), c = chunk_of(t, it);
        if (t * 256 + s != cur_slot) {
          set_slot(t, s);
          cur_slot = t * 256 + s;
        }
        const int k0 = c * BK + wd * EPL;
        const bool kin = k0 < Rin;   // Rin and k0 even: a bf16 pair is all in or out
#pragma unroll
        for (int u = 0; u < UH; ++u) {
          int sb = srcb[h * UH + u];
          bool ok = sb >= 0 && kin;
          const float4* p = reinterpret_cast<const float4*>(a.up) + (int64_t)(ok ? sb : 0) * Rin + k0;
          if (EPL == 2) {
            if (ok) {
              ld_nc_v8(p, q[u][0], q[u][EPL - 1]);
            } else {
              q[u][0] = make_float4(0.f, 0.f, 0.f, 0.f);
              q[u][EPL - 1] = q[u][0];
            }
          } else {
            q[u][0] = ok ? __ldg(p) : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
      };
      auto store_half = [&](int it, int h, const float4 (&q)[UH][EPL]) {
        const int t = tile_of(it);
        int s = slot_of(t, it);
        float ox, oy, oz;
        slot_shift(a.mode, s, t_cls[t], ox, oy, oz);
        const int st = it % STAGES;
        const uint32_t bhi = smem_u32(smem + st * STAGE_BYTES + A_STAGE);
        const uint32_t blo = bhi + B_BYTES;
#pragma unroll
        for (int u = 0; u < UH; ++u) {
          const int ul = h * UH + u;
          float side = sside[t][box_of(ul)];
          float sx = ox * side, sy = oy * side, sz = oz * side;
          float v[4][EPL];
#pragma unroll
          for (int t = 0; t < EPL; ++t) {
            v[0][t] = q[u][t].x;
            v[1][t] = q[u][t].y;
            v[2][t] = q[u][t].z;
            v[3][t] = q[u][t].w + sx * q[u][t].x + sy * q[u][t].y + sz * q[u][t].z;
          }
          uint32_t hw[4], lw[4];
#pragma unroll
          for (int ch = 0; ch < 4; ++ch) {
            if (SPLIT == SPLIT_TF32) {
              float hf = tf32_rn(v[ch][0]);
              hw[ch] = __float_as_uint(hf);
              lw[ch] = __float_as_uint(tf32_rn(v[ch][0] - hf));
            } else {
              __nv_bfloat162 h2 = __floats2bfloat162_rn(v[ch][0], v[ch][EPL - 1]);
              float2 hf = __bfloat1622float2(h2);
              hw[ch] = *reinterpret_cast<uint32_t*>(&h2);
              lw[ch] = pack_bf16(v[ch][0] - hf.x, v[ch][EPL - 1] - hf.y);
            }
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            uint32_t h_ = hw[i], l_ = lw[i];
            if (BPI == 2 && bsel) {
              h_ = hw[i ^ 1];
              l_ = lw[i ^ 1];
            }
            const uint32_t off = roff[i] + (uint32_t)(32 * SWB * BPI) * ul;
            st_shared_u32(bhi + off, h_);
            st_shared_u32(blo + off, l_);
          }
        }
      };
      float4 qa[UH][EPL], qb[UH][EPL];
      if (total > 0) load_half(0, 0, qa);
      for (int it = 0; it < total; ++it) {
        int st = it % STAGES;
        load_half(it, 1, qb);
        // lane 0 waits for the stage to be free; the warp leaves the loop together on a timeout
        int ok_wait = 1;
        if (lane == 0 && it >= STAGES)
          ok_wait = wait_parity(&empty[st], ((it / STAGES) - 1) & 1, a.status, &bail, a.lim) ? 1 : 0;
        if (!__shfl_sync(0xffffffffu, ok_wait, 0)) break;
        store_half(it, 0, qa);
        if (it + 1 < total) load_half(it + 1, 0, qa);
        store_half(it, 1, qb);
        // each lane orders its shared-memory writes before the async proxy (the MMAs) reads
        // them; lane 0 then arrives once for the warp
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncwarp();
        if (lane == 0) arrive(&full[st]);
      }
    }
  } else if (warp == W_MMA) {
    // ---------------- MMA issue (one thread) ----------------
    if (lane == 0) {
      bool ok = true;
      for (int t = 0; t < T && ok; ++t) {
        for (int G = t_g0[t]; G < t_g0[t + 1]; ++G) {
          if (G > 0 && !wait_parity(&acc_empty, (G - 1) & 1, a.status, &bail, a.lim)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const int it_beg = t_it0[t] + (G - t_g0[t]) * GI, it_end = min(t_it0[t + 1], it_beg + GI);
          for (int it = it_beg; it < it_end; ++it) {
            int st = it % STAGES;
            if (!wait_parity(&full[st], (it / STAGES) & 1, a.status, &bail, a.lim)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            uint32_t base = smem_u32(smem + st * STAGE_BYTES);
            uint32_t bhi = base + A_STAGE, blo = bhi + B_BYTES;
            bool first = it == it_beg;
            for (int r = 0; r < nrb; ++r) {
              uint32_t ahi = base + r * 2 * A_BYTES, alo = ahi + A_BYTES;
              uint32_t d = tmem + (uint32_t)(r * BN);
#pragma unroll
              for (int kk = 0; kk < BK / MK; ++kk) {
                uint32_t ko = kk * 32;  // MK elements = 32 bytes in both formats and swizzles
                mma<SPLIT, BN>(d, sdesc<SWB>(ahi + ko), sdesc<SWB>(bhi + ko), (first && kk == 0) ? 0u : 1u);
                mma<SPLIT, BN>(d, sdesc<SWB>(ahi + ko), sdesc<SWB>(blo + ko), 1u);
                mma<SPLIT, BN>(d, sdesc<SWB>(alo + ko), sdesc<SWB>(bhi + ko), 1u);
              }
            }
            commit(&empty[st]);
          }
          if (!ok) break;
          commit(&acc_full);
        }
      }
    }
  } else {
    // ---------------- epilogue: drain each offset into the running sum ----------------
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    float x[32], y[32];
    float4* dst = reinterpret_cast<float4*>(a.dn + a.part_stride * blockIdx.z);
    bool stop = false;
    for (int t = 0; t < T && !stop; ++t) {
      for (int G = t_g0[t]; G < t_g0[t + 1]; ++G) {
        // lane 0 waits; the warp stays converged for the .sync.aligned TMEM accesses
        int ok_wait = lane == 0 ? (wait_parity(&acc_full, G & 1, a.status, &bail, a.lim) ? 1 : 0) : 0;
        if (!__shfl_sync(0xffffffffu, ok_wait, 0)) {
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const bool first = G == t_g0[t];   // the tile's first group starts its running sum
        for (int q = 0; q < nrb * (BN / 32); ++q) {   // row block q / (BN / 32), 32 columns each
          tmem_ld32(tmem + lane_base + q * 32, x);
          if (!first) tmem_ld32(tmem + lane_base + SUM_COL + q * 32, y);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
          if (!first) {
#pragma unroll
            for (int u = 0; u < 32; ++u) x[u] += y[u];
          }
          tmem_st32(tmem + lane_base + SUM_COL + q * 32, x);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        arrive(&acc_empty);   // the MMAs of the next group (this or the next tile) may start
      }
      if (stop) break;
      // write tile t (the MMAs of tile t + 1 proceed meanwhile): row = row0 + 128 r + lane
      // quarter + lane, columns (box j, channel); every CTA writes its partial (zeros when it had
      // no offsets) so the combine is fixed-order
      if (blockIdx.x * T + t >= a.ntiles) continue;
      const int do_write = __shfl_sync(0xffffffffu, (!*(volatile int*)&bail) ? 1 : 0, 0);
      if (!do_write) break;
      const bool has = t_n[t] > 0;
      for (int q = 0; q < nrb * (BN / 32); ++q) {
        int row = row0 + (q / (BN / 32)) * BM + (warp & 3) * 32 + lane;
        int qc = q % (BN / 32);
        if (has) {
          tmem_ld32(tmem + lane_base + SUM_COL + q * 32, x);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        } else {
#pragma unroll
          for (int u = 0; u < 32; ++u) x[u] = 0.f;
        }
        if constexpr (CH == 1) {
          if (row < R) {
            // column u = box 32 qc + u; a warp writes 32 consecutive rows of one box per store
            float* dst1 = a.dn + a.part_stride * blockIdx.z;
#pragma unroll
            for (int u = 0; u < 32; ++u) {
              if (sbox[t][qc * 32 + u] < 0) continue;
              float* o = dst1 + (int64_t)sout[t][qc * 32 + u] * R + row;
              float v = x[u];
              if (a.write == TC_ADD) {
                v += *o;
              } else if (a.write == TC_SCALE) {
                const float h = 0.5f * sside[t][qc * 32 + u];
                v *= (a.qrow4 && (row & 3) == 3) ? h * h : h;
              }
              *o = v;
            }
          }
        } else if (row < R) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            if (sbox[t][qc * 8 + jj] < 0) continue;
            float4 v = make_float4(x[4 * jj], x[4 * jj + 1], x[4 * jj + 2], x[4 * jj + 3]);
            float4* o = dst + (int64_t)sout[t][qc * 8 + jj] * R + row;
            if (a.write == TC_ADD) {
              float4 w = *o;
              v.x += w.x;
              v.y += w.y;
              v.z += w.z;
              v.w += w.w;
            } else if (a.write == TC_SCALE) {
              float al = 0.5f * sside[t][qc * 8 + jj];
              v.x *= al;
              v.y *= al;
              v.z *= al;
              v.w *= al;
            }
            *o = v;
          }
        }
      }
      // the next tile's first drain overwrites the running sum: its reads above are complete
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == W_MMA) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS)
                 : "memory");
  }
}

// dn[b] (+)= sum of the partial sums over the slot ranges, in range order (boxes of the tiles
// only); add = 0 stores.
__global__ void k_combine_parts(const float4* __restrict__ parts, int64_t part_stride4, int nsplit,
                                float4* __restrict__ dn, const int4* __restrict__ tiles, int ntiles,
                                const int* __restrict__ boxlist, int R, int add) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int4 tile = tiles[t];
    for (int e = threadIdx.x; e < tile.y * R; e += blockDim.x) {
      int b = boxlist[tile.x + e / R], r = e % R;
      int64_t i = (int64_t)b * R + r;
      float4 v = parts[i];
      for (int z = 1; z < nsplit; ++z) {
        float4 w = parts[i + part_stride4 * z];
        v.x += w.x;
        v.y += w.y;
        v.z += w.z;
        v.w += w.w;
      }
      if (add) {
        float4 d = dn[i];
        v.x += d.x;
        v.y += d.y;
        v.z += d.z;
        v.w += d.w;
      }
      dn[i] = v;
    }
  }
}

// Grouped M->L: dn[box] (+)= sum of the box's partials (one per parent neighbour, in
// neighbour order).  comb = (box, first partial, count) for every box; R4 = float4 per box.
__global__ void k_combine_groups(const float4* __restrict__ parts, const int4* __restrict__ comb,
                                 int ncomb, float4* __restrict__ dn, int R4, int add) {
  for (int i = blockIdx.x; i < ncomb; i += gridDim.x) {
    const int4 c = comb[i];
    if (c.z == 0) continue;   // a box without V entries (or below the M->L levels)
    for (int r = threadIdx.x; r < R4; r += blockDim.x) {
      const float4* p = parts + (int64_t)c.y * R4 + r;
      float4 v = p[0];
      for (int k = 1; k < c.z; ++k) {
        float4 w = p[(int64_t)k * R4];
        v.x += w.x;
        v.y += w.y;
        v.z += w.z;
        v.w += w.w;
      }
      float4* o = dn + (int64_t)c.x * R4 + r;
      if (add) {
        float4 d = *o;
        v.x += d.x;
        v.y += d.y;
        v.z += d.z;
        v.w += d.w;
      }
      *o = v;
    }
  }
}

}  // namespace tc

// Tables on the tensor cores: the four-channel Laplace table (Laplace ML kernel, C = 4) and
// the single-column tables (C = 1) whose rows per box are a multiple of 8 (32-byte loads).
bool tc_table(const Plan& P) {
  return (P.C == 4 && !P.ml_stokes) || (P.C == 1 && P.R % 8 == 0);
}

bool tc_supported(Plan& P) {
  if (P.prec != KAFMM_PREC_MIXED || !tc_table(P) || !P.opstc.p) return false;
  int rows = (P.R + tc::BM - 1) / tc::BM;
  // compressed coordinates: every operator set shares the tiles, so a CTA always owns two
  // 128-row blocks (the last CTA of an odd block count runs one)
  P.tc_rb = P.cmp ? 2 : (rows % 2 == 0 ? 2 : 1);
  P.tc_boxes = 256 / P.tc_rb / P.C;
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  cudaGetLastError();
  return major == 10 && minor == 3;
}

// Tensor map over a split operator array of total_rows rows ([op][2][rows][colpad], tf32 or
// bf16), swb-byte swizzle, boxes of 128 rows x swb bytes.
static int make_tmap(Plan& P, CUtensorMap* map, void* base, int64_t total_rows, int colpad, bool tf32,
                     int swb) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return fail(P, KAFMM_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  int es = tf32 ? 4 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)colpad, (cuuint64_t)total_rows};
  cuuint64_t strides[1] = {(cuuint64_t)colpad * es};
  cuuint32_t box[2] = {(cuuint32_t)(swb / es), tc::BM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(map, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                      2, base, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE,
                      swb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(P, KAFMM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return 0;
}

// Operator sets of the tensor-core gather-GEMM: the map, the rows per operator, the padded k
// extent, the input rows per box and the output rows per box.
struct OpSet {
  int map, rop, kpad, rin, rout;
};
static OpSet op_set(const Plan& P, int opset, bool m2l) {
  switch (opset) {
    case TCO_CMP: return {m2l ? 2 : 3, P.rp, P.rp, P.rp, P.rp};
    case TCO_CIN: return {4, P.rp, P.Rpad, P.R, P.rp};
    case TCO_COUT: return {5, P.R, P.rp, P.rp, P.R};
    default: return {m2l ? 0 : 1, P.R, P.Rpad, P.R, P.R};
  }
}

static int tc_prepare(Plan& P) {
  if (P.tmap_ready) return 0;
  const bool ml_tf32 = P.tc_split == SPLIT_TF32, cm_tf32 = P.tc_split_cm == SPLIT_TF32;
  for (int sw = 0; sw < 2; ++sw) {   // 128- and 64-byte swizzled rows
    int swb = sw == 0 ? 128 : 64;
    auto map = [&](int k) { return reinterpret_cast<CUtensorMap*>(P.tmaps[k][sw]); };
    int rc = make_tmap(P, map(0), P.opstc.p, (int64_t)N_M2L * 2 * P.R, P.Rpad, ml_tf32, swb);
    if (!rc) rc = make_tmap(P, map(1), P.opstc_aux.p, (int64_t)N_AUX * 2 * P.R, P.Rpad, true, swb);
    if (!rc && P.cmp) {
      rc = make_tmap(P, map(2), P.opstc_cm2l.p, (int64_t)N_M2L * 2 * P.rp, P.rp, cm_tf32, swb);
      if (!rc) rc = make_tmap(P, map(3), P.opstc_caux.p, (int64_t)N_CAUX * 2 * P.rp, P.rp, true, swb);
      if (!rc) rc = make_tmap(P, map(4), P.opstc_cin.p, (int64_t)2 * 2 * P.rp, P.Rpad, true, swb);
      if (!rc) rc = make_tmap(P, map(5), P.opstc_cout.p, (int64_t)2 * 2 * P.R, P.rp, true, swb);
    }
    if (rc) return rc;
  }
  cudaError_t e = cudaSuccess;
  for (auto fn : {tc::k_m2l_tc<SPLIT_TF32, 1, 128, 4>, tc::k_m2l_tc<SPLIT_TF32, 2, 128, 4>,
                  tc::k_m2l_tc<SPLIT_BF16, 1, 128, 4>, tc::k_m2l_tc<SPLIT_BF16, 2, 128, 4>,
                  tc::k_m2l_tc<SPLIT_TF32, 1, 64, 4>, tc::k_m2l_tc<SPLIT_TF32, 2, 64, 4>,
                  tc::k_m2l_tc<SPLIT_BF16, 1, 64, 4>, tc::k_m2l_tc<SPLIT_BF16, 2, 64, 4>,
                  tc::k_m2l_tc<SPLIT_TF32, 1, 128, 1>, tc::k_m2l_tc<SPLIT_TF32, 2, 128, 1>,
                  tc::k_m2l_tc<SPLIT_BF16, 1, 128, 1>, tc::k_m2l_tc<SPLIT_BF16, 2, 128, 1>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES);
  if (e != cudaSuccess) return cuda_fail(P, e, "cudaFuncSetAttribute(k_m2l_tc)");
  P.tmap_ready = true;
  return 0;
}

// One gather-GEMM on the tensor cores over the operator set opset (TCO_*).  TC_M2L: the
// operator in the plan's split format, several offset ranges per tile when the grid is small.
// Other modes: TF32x3 (op = index of the operator in its set for TC_APPLY), one range.
int tc_gemm_launch(Plan& P, int mode, int opset, const int4* tiles, int ntiles, const int* boxlist,
                   const float* in, float* out, int op, int write, cudaStream_t st) {
  int rc = tc_prepare(P);
  if (rc) return rc;
  const bool m2l = mode == tc::TC_M2L;
  const OpSet os = op_set(P, opset, m2l);
  // 64-byte rows, four stages : 128-byte rows, two (single-column tables: always two)
  const int sw = P.tc_stages == 4 && P.C == 4 ? 1 : 0;
  const CUtensorMap& map = *reinterpret_cast<const CUtensorMap*>(P.tmaps[os.map][sw]);
  const int split = m2l ? (opset == TCO_CMP ? P.tc_split_cm : P.tc_split) : SPLIT_TF32;
  int rows = (os.rout + P.tc_rb * tc::BM - 1) / (P.tc_rb * tc::BM);   // CTAs per tile
  // slot ranges per tile (M->L offsets, M->M child octants): enough CTAs to fill the 152 SMs
  // over several waves; the ranges' partial sums are combined in fixed order
  // grouped M->L tiles (one parent neighbour each) write per-box partials, combined below
  const bool grouped = m2l && P.wl.m2l_grouped;
  const bool splittable = (m2l && !grouped) || mode == tc::TC_M2M;
  int nsplit = 1;
  while (splittable && nsplit < P.tc_ranges && (int64_t)ntiles * rows * nsplit < 152 * 6) nsplit *= 2;
  int64_t part_stride = (int64_t)P.tree.nbox * os.rout * P.C;
  if (nsplit > 1 || grouped) {
    size_t bytes = grouped ? sizeof(float) * (size_t)P.wl.m2l_nparts * os.rout * P.C + 256
                           : sizeof(float) * part_stride * nsplit + 256;
    cudaError_t e = P.m2l_parts.reserve(bytes);
    if (e != cudaSuccess) return cuda_fail(P, e, "M->L partial buffers");
  }
  tc::Args a;
  a.t = P.tree.view();
  a.L = P.L;
  a.up = in;
  // one offset range: straight into the output; several: partial buffers, combined below
  a.dn = nsplit > 1 || grouped ? P.m2l_parts.as<float>() : out;
  a.part_stride = nsplit > 1 ? part_stride : 0;
  a.nsplit = nsplit;
  a.part = grouped ? reinterpret_cast<const int*>(P.m2l_part_sorted) : nullptr;
  // StokesPVel table: the q rows of an equivalent density take the half-width twice
  a.qrow4 = P.D == 4 && os.rout == P.R ? 1 : 0;
  a.tiles = tiles;
  a.boxlist = boxlist;
  a.vtab = P.tree.vtab.as<int32_t>();
  a.status = P.tree.status.as<unsigned>();
  a.lim = P.wait;
  a.Rout = os.rout;
  a.Rin = os.rin;
  a.Rop = os.rop;
  a.mode = mode;
  a.write = nsplit > 1 || grouped ? tc::TC_STORE : write;
  a.op = m2l ? 0 : op;
  // consecutive tiles per CTA: the option, kept while the grid still fills the 152 SMs twice
  int tpc = std::max(1, std::min(P.tc_tiles, tc::TC_TMAX));
  while (tpc > 1 && (int64_t)((ntiles + tpc - 1) / tpc) * rows * nsplit < 152 * 2) tpc /= 2;
  a.ntiles = ntiles;
  a.tpc = tpc;
  dim3 grid((ntiles + tpc - 1) / tpc, rows, nsplit);
  const int swb = sw ? 64 : 128;
  const int bk = swb / (split == SPLIT_TF32 ? tc::Fmt<SPLIT_TF32>::ES : tc::Fmt<SPLIT_BF16>::ES);
  a.nchunk = os.kpad / bk;
  a.group = P.C == 1 ? tc::M2L_GROUP_K / bk : (split == SPLIT_BF16 ? 2 : 1) * a.nchunk;
  if (a.group < 1) a.group = 1;
#define KAFMM_TC_LAUNCH(SP, RBv, SW) \
  KL tc::k_m2l_tc<SP, RBv, SW, 4><<<grid, tc::THREADS, tc::SMEM_BYTES, st>>>(map, a)
#define KAFMM_TC_LAUNCH1(SP, RBv) \
  KL tc::k_m2l_tc<SP, RBv, 128, 1><<<grid, tc::THREADS, tc::SMEM_BYTES, st>>>(map, a)
  if (P.C == 1) {
    if (split == SPLIT_TF32 && P.tc_rb == 2) KAFMM_TC_LAUNCH1(SPLIT_TF32, 2);
    else if (split == SPLIT_TF32) KAFMM_TC_LAUNCH1(SPLIT_TF32, 1);
    else if (P.tc_rb == 2) KAFMM_TC_LAUNCH1(SPLIT_BF16, 2);
    else KAFMM_TC_LAUNCH1(SPLIT_BF16, 1);
  } else if (swb == 128) {
    if (split == SPLIT_TF32 && P.tc_rb == 2) KAFMM_TC_LAUNCH(SPLIT_TF32, 2, 128);
    else if (split == SPLIT_TF32) KAFMM_TC_LAUNCH(SPLIT_TF32, 1, 128);
    else if (P.tc_rb == 2) KAFMM_TC_LAUNCH(SPLIT_BF16, 2, 128);
    else KAFMM_TC_LAUNCH(SPLIT_BF16, 1, 128);
  } else {
    if (split == SPLIT_TF32 && P.tc_rb == 2) KAFMM_TC_LAUNCH(SPLIT_TF32, 2, 64);
    else if (split == SPLIT_TF32) KAFMM_TC_LAUNCH(SPLIT_TF32, 1, 64);
    else if (P.tc_rb == 2) KAFMM_TC_LAUNCH(SPLIT_BF16, 2, 64);
    else KAFMM_TC_LAUNCH(SPLIT_BF16, 1, 64);
  }
#undef KAFMM_TC_LAUNCH
#undef KAFMM_TC_LAUNCH1
  if (grouped && P.tree.nbox > 0)
    KL tc::k_combine_groups<<<std::min(P.tree.nbox, 152 * 8), 128, 0, st>>>(
        P.m2l_parts.as<float4>(), P.m2l_comb.as<int4>(), P.tree.nbox,
        reinterpret_cast<float4*>(out), os.rout * P.C / 4, write == tc::TC_ADD ? 1 : 0);
  if (nsplit > 1)   // a box holds Rout * C floats = Rout * C / 4 float4 (Rout * C a multiple of 8)
    KL tc::k_combine_parts<<<std::min(ntiles, 152 * 4), 256, 0, st>>>(
        P.m2l_parts.as<float4>(), part_stride / 4, nsplit, reinterpret_cast<float4*>(out), tiles, ntiles,
        boxlist, os.rout * P.C / 4, write == tc::TC_ADD ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(P, e, "k_m2l_tc launch");
  return 0;
}

}  // namespace kafmm
