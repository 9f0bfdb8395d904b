// tcgen05 building blocks shared by the tensor-core kernels (sm_103a): UMMA shared-memory and
// instruction descriptors, the MMA issue, commit to an mbarrier, and TMEM loads / stores.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace kafmm {
namespace tc {

constexpr int BM = 128;   // rows of one MMA (M) and of one TMEM accumulator block

// Split formats: an SWB-byte swizzle row holds SWB / ES elements; one MMA consumes MK of them
// (32 bytes in both formats).
template <int SPLIT>
struct Fmt;
template <>
struct Fmt<SPLIT_TF32> {  // kind::tf32, K = 8 per instruction
  static constexpr int ES = 4, MK = 8;
  static constexpr uint32_t AB = 2;
};
template <>
struct Fmt<SPLIT_BF16> {  // kind::f16 with bf16 operands, K = 16 per instruction
  static constexpr int ES = 2, MK = 16;
  static constexpr uint32_t AB = 1;
};
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// K-major UMMA shared-memory descriptor (SM100 format, version 1) for SWB-byte swizzled rows:
// start >> 4, LBO = 16 B (unused for swizzled K-major), SBO = 8 rows x SWB bytes, layout
// SWIZZLE_128B (2) or SWIZZLE_64B (4).
template <int SWB>
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(16 >> 4) << 16;
  d |= (uint64_t)((8 * SWB) >> 4) << 32;
  d |= (uint64_t)1 << 46;       // descriptor version
  d |= (uint64_t)(SWB == 128 ? 2 : 4) << 61;
  return d;
}

// Instruction descriptor: D = F32, A/B format (bf16 = 1, tf32 = 2), K-major both, N = 256,
// M = 128.
template <int SPLIT, int BN>
__device__ __forceinline__ constexpr uint32_t idesc() {
  return (1u << 4) | (Fmt<SPLIT>::AB << 7) | (Fmt<SPLIT>::AB << 10) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}

template <int SPLIT, int BN>
__device__ __forceinline__ void mma(uint32_t dt, uint64_t a, uint64_t b, uint32_t acc) {
  if (SPLIT == SPLIT_TF32)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
        "l"(a), "l"(b), "r"(idesc<SPLIT, BN>()), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
        "l"(a), "l"(b), "r"(idesc<SPLIT, BN>()), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t* r = reinterpret_cast<uint32_t*>(v);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float* v) {
  const uint32_t* r = reinterpret_cast<const uint32_t*>(v);
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
      "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]),
      "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]),
      "r"(r[30]), "r"(r[31])
      : "memory");
}

}  // namespace tc
}  // namespace kafmm
