// Shared definitions of the KAFMM evaluator (CUDA, sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

#include "../../include/kafmm.h"

namespace kafmm {

// Periodic axes of a boundary condition: bit 0 = x, bit 1 = y, bit 2 = z (PX, PXY, PXYZ).
inline int periodic_mask(int bc) {
  return bc == KAFMM_BC_PX ? 1 : (bc == KAFMM_BC_PXY ? 3 : (bc == KAFMM_BC_PXYZ ? 7 : 0));
}

// Count of kernel launches issued by this thread (reported per set_points + eval).
extern thread_local long long g_launches;
#define KL ++::kafmm::g_launches,
// Count of device allocations (cudaMalloc) made by the library in this process.
long long device_allocations();
void count_device_allocation();

constexpr int MAX_LEVEL = 20;        // finest octree level; keys carry 20 bits per axis
constexpr int MAX_LEVELS = MAX_LEVEL + 1;
constexpr double PI = 3.14159265358979323846;

// Surface radii in units of the box half-width (Ying, Biros & Zorin 2004): upward
// equivalent / check, downward equivalent / check.
constexpr double ALPHA_UE = 1.05, ALPHA_UC = 2.95, ALPHA_DE = 2.95, ALPHA_DC = 1.05;
// Relative singular-value cutoffs of the check-to-equivalent pseudo-inverses: 1e-9 for the
// FP64 form (lowest FP64 error against the direct sum for p = 8..12); 1e-7 (about twice the
// FP32 unit roundoff) for the FP32 and mixed forms, where a smaller cutoff only amplifies
// rounding -- for the Stokeslet the normal density is an exact null mode of the single layer.
constexpr double PINV_RCOND_FP64 = 1e-9, PINV_RCOND_FP32 = 1e-7;

// Operator slots: 343 M->L offsets (ox,oy,oz) in [-3,3]^3 (the 27 inner ones unused), then
// 8 M->M octants, 8 L->L octants, and the upward / downward pseudo-inverses in factored form
// pinv = V (S^+ U^T): slot *1 holds S^+ U^T, slot *2 holds V.  Applying the two factors in turn
// keeps the rounding of a short format confined to the directions the pseudo-inverse
// amplifies; the product matrix itself, rounded to FP32, loses all accuracy.
constexpr int OP_M2L = 0, N_M2L = 343;
constexpr int OP_M2M = OP_M2L + N_M2L;
constexpr int OP_L2L = OP_M2M + 8;
constexpr int OP_UP1 = OP_L2L + 8;
constexpr int OP_UP2 = OP_UP1 + 1;
constexpr int OP_DN1 = OP_UP2 + 1;
constexpr int OP_DN2 = OP_DN1 + 1;
constexpr int OP_PER = OP_DN2 + 1;  // periodic far-image operator of the root (composed)
constexpr int N_OPS = OP_PER + 1;
// operators of the non-M->L tensor-core modes (M->M, L->L, pseudo-inverse factors), kept in
// their own TF32 split array: aux index = slot - OP_M2M
constexpr int N_AUX = OP_PER - OP_M2M;

// Operators of the compressed coordinates besides M->L: 8 M->M, 8 L->L, the periodic one.
constexpr int N_CAUX = 17, CAUX_PER = 16;

// Operator sets of the tensor-core gather-GEMM: the dense operators (R x R), the translations
// between compressed coordinates (rp x rp), compress (rp x R) and decompress (R x rp).
enum { TCO_DENSE = 0, TCO_CMP = 1, TCO_CIN = 2, TCO_COUT = 3 };

// Split formats of the tensor-core M->L.
enum { SPLIT_TF32 = 0, SPLIT_BF16 = 1 };

__host__ __device__ inline int m2l_index(int ox, int oy, int oz) {
  return (ox + 3) + 7 * (oy + 3) + 49 * (oz + 3);
}

// Shift code of a periodic image: (sx+1) + 3(sy+1) + 9(sz+1); 13 = no shift.
__host__ __device__ inline int shift_code(int sx, int sy, int sz) {
  return (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1);
}
__host__ __device__ inline void shift_decode(int c, int& sx, int& sy, int& sz) {
  sx = c % 3 - 1;
  sy = (c / 3) % 3 - 1;
  sz = c / 9 - 1;
}

// List entry: source box index in the low 27 bits, shift code in the high 5 (codes >= 16 set
// the sign bit, so entries are compared with LIST_EMPTY, never with 0).
constexpr int32_t LIST_EMPTY = -1;  // box 2^27 - 1 with shift code 31: not a valid entry
__host__ __device__ inline int32_t pack_entry(int box, int sc) { return box | (sc << 27); }
__host__ __device__ inline int entry_box(int32_t e) { return e & ((1 << 27) - 1); }
__host__ __device__ inline int entry_shift(int32_t e) { return (int)((uint32_t)e >> 27); }

// 3 x 20-bit interleave: bit 3i = x_i, 3i+1 = y_i, 3i+2 = z_i.
__host__ __device__ inline uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0xFFFFF;
  x = (x | (x << 32)) & 0x001F00000000FFFFull;
  x = (x | (x << 16)) & 0x001F0000FF0000FFull;
  x = (x | (x << 8)) & 0x100F00F00F00F00Full;
  x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}
__host__ __device__ inline uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x | (x >> 2)) & 0x10C30C30C30C30C3ull;
  x = (x | (x >> 4)) & 0x100F00F00F00F00Full;
  x = (x | (x >> 8)) & 0x001F0000FF0000FFull;
  x = (x | (x >> 16)) & 0x001F00000000FFFFull;
  x = (x | (x >> 32)) & 0xFFFFFull;
  return (uint32_t)x;
}
__host__ __device__ inline uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

// ---- device buffers -----------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  // Grows to at least nbytes (contents not preserved). Returns a CUDA error code.
  cudaError_t reserve(size_t nbytes) {
    if (nbytes <= bytes && p) return cudaSuccess;
    release();
    size_t nb = nbytes < 256 ? 256 : nbytes;
    count_device_allocation();
    cudaError_t e = cudaMalloc(&p, nb);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    bytes = nb;
    return cudaSuccess;
  }
  template <class T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

// Page-locked host staging buffer (grows, never shrinks; contents not preserved on growth).
struct HostBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ~HostBuf() { release(); }
  void release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
  }
  cudaError_t reserve(size_t nbytes) {
    if (nbytes <= bytes && p) return cudaSuccess;
    release();
    size_t nb = nbytes < 4096 ? 4096 : nbytes + nbytes / 4;
    cudaError_t e = cudaMallocHost(&p, nb);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    bytes = nb;
    return cudaSuccess;
  }
  template <class T>
  T* as(size_t byte_off = 0) const { return reinterpret_cast<T*>(static_cast<char*>(p) + byte_off); }
};

// Status word written by kernels (never trapped on): bit 0 domain error, bit 1 timeout,
// bit 2 capacity overflow, bit 3 non-finite value.
enum { ST_DOMAIN = 1, ST_TIMEOUT = 2, ST_OVERFLOW = 4, ST_NONFINITE = 8 };

// Limits of the device-side waits (nanoseconds of %globaltimer).  A wait that has not
// completed after hard_ns gives up: the kernel records ST_TIMEOUT and winds down.  report_ns
// only reports: a wait that took report_ns or longer records ST_TIMEOUT and still completes
// normally (a test sets it to 0 to see the status reach the host without changing what runs).
struct WaitLimits {
  unsigned long long hard_ns = 2000000000ull;
  unsigned long long report_ns = ~0ull;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(addr), "r"(phase), "r"(100000u)  // suspend up to 0.1 ms per try (woken on completion)
      : "memory");
  return ok != 0;
}

// Bounded mbarrier wait: true once the phase completed, false (ST_TIMEOUT recorded) when
// lim.hard_ns passed first.
__device__ inline bool mbar_wait_bounded(uint64_t* bar, uint32_t phase, unsigned* status,
                                         const WaitLimits& lim) {
  uint32_t addr = (uint32_t)__cvta_generic_to_shared(bar);
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(addr, phase)) {
      if (lim.report_ns != ~0ull && global_ns() - t0 >= lim.report_ns)
        atomicOr(status, (unsigned)ST_TIMEOUT);
      return true;
    }
    if (global_ns() - t0 > lim.hard_ns) {
      atomicOr(status, (unsigned)ST_TIMEOUT);
      return false;
    }
  }
}

__device__ inline void mbar_init(uint64_t* bar, unsigned count) {
  uint32_t addr = (uint32_t)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(addr), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  uint32_t addr = (uint32_t)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(addr), "r"(bytes)
               : "memory");
}

// 1-D bulk copy global -> shared completing on an mbarrier (16-byte aligned, size % 16 == 0).
__device__ inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
          "r"(d),
      "l"(src), "r"(bytes), "r"(b)
      : "memory");
}

}  // namespace kafmm
