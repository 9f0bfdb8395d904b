// Micro-benchmarks of the arithmetic rates the rooflines of the evaluator are taken against:
// FP32 FMA and MUFU reciprocal square root (the near field), FP64 FMA (the plain reference
// form), and the tcgen05 MMA issue rate in TF32 and BF16 (the split-precision gather-GEMMs).
// Every kernel runs a fixed amount of independent work per thread (or per CTA) so the timed
// launch is bound by the unit measured; the results feed no computation of the method.
#include "tcgen05.cuh"

namespace kafmm {

// 8 independent FMA chains per thread; 2 flop per FMA.
__global__ void __launch_bounds__(256) k_peak_ffma(int iters, float b, float c, float* out) {
  float a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fmaf(a[i], b, c);
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  if (s == 1234.5f) out[blockIdx.x] = s;   // keeps the chains live
}

__global__ void __launch_bounds__(256) k_peak_dfma(int iters, double b, double c, double* out) {
  double a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = (double)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  if (s == 1234.5) out[blockIdx.x] = s;
}

// 8 independent chains of MUFU rsqrt (x -> 1/sqrt(x) stays positive and finite).
__global__ void __launch_bounds__(256) k_peak_rsqrt(int iters, float* out) {
  float a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = 1.0f + (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < 8; ++i) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(a[i]));
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  if (s == 1234.5f) out[blockIdx.x] = s;
}

// One CTA per SM: one thread issues iters x 4 MMAs (M = 128, N = 256, one 128-byte K row of
// A and B per 4 instructions) into one TMEM accumulator, then commits and waits (bounded).
// The operands are zeros in shared memory; only the issue rate is measured.
template <int SPLIT>
__global__ void __launch_bounds__(128, 1) k_peak_mma(int iters, unsigned* status) {
  constexpr int BN = 256, MK = tc::Fmt<SPLIT>::MK;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t done;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < (tc::BM + BN) * 128 / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  if (threadIdx.x == 0) mbar_init(&done, 1);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     tc::smem_u32(&tmem_base)),
                 "r"(256)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;
  if (threadIdx.x == 0) {
    const uint32_t a = tc::smem_u32(smem), b = a + tc::BM * 128;
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int kk = 0; kk < 128 / (MK * tc::Fmt<SPLIT>::ES); ++kk)
        tc::mma<SPLIT, BN>(tmem, tc::sdesc<128>(a + kk * 32), tc::sdesc<128>(b + kk * 32),
                           (it | kk) ? 1u : 0u);
    tc::commit(&done);
    WaitLimits lim;
    mbar_wait_bounded(&done, 0, status, lim);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(256) : "memory");
  }
}

}  // namespace kafmm

using namespace kafmm;

extern "C" int kafmm_measure_peak(int what, double* rate, double* ms) {
  if (!rate || what < 0 || what > 4) return KAFMM_ERR_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return KAFMM_ERR_CUDA;
  }
  DevBuf out;
  if (out.reserve(sizeof(double) * 4096) != cudaSuccess) return KAFMM_ERR_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int smem_mma = (tc::BM + 256) * 128 + 1024;
  if (what >= 3) {
    cudaFuncSetAttribute(k_peak_mma<SPLIT_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_mma);
    cudaFuncSetAttribute(k_peak_mma<SPLIT_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_mma);
  }
  const int blocks = nsm * 8, threads = 256;
  double ops = 0.0;
  float t = 0.f;
  for (int rep = 0; rep < 3; ++rep) {   // the first launch warms up; the last one is kept
    int iters = 0;
    cudaEventRecord(e0);
    if (what == 0) {
      iters = 1 << 16;
      k_peak_ffma<<<blocks, threads>>>(iters, 0.999f, 1e-3f, out.as<float>());
      ops = 2.0 * 8 * (double)iters * blocks * threads;
    } else if (what == 1) {
      iters = 1 << 14;
      k_peak_rsqrt<<<blocks, threads>>>(iters, out.as<float>());
      ops = 8.0 * (double)iters * blocks * threads;
    } else if (what == 2) {
      iters = 1 << 12;
      k_peak_dfma<<<blocks, threads>>>(iters, 0.999, 1e-3, out.as<double>());
      ops = 2.0 * 8 * (double)iters * blocks * threads;
    } else {
      iters = 1 << 14;
      const int split = what == 3 ? SPLIT_TF32 : SPLIT_BF16;
      const int mk = split == SPLIT_TF32 ? 8 : 16;
      if (split == SPLIT_TF32)
        k_peak_mma<SPLIT_TF32><<<nsm, 128, smem_mma>>>(iters, out.as<unsigned>());
      else
        k_peak_mma<SPLIT_BF16><<<nsm, 128, smem_mma>>>(iters, out.as<unsigned>());
      ops = 2.0 * tc::BM * 256 * mk * 4.0 * (double)iters * nsm;
    }
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&t, e0, e1);
  }
  cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return KAFMM_ERR_CUDA;
  *rate = ops / (t * 1e-3);
  if (ms) *ms = t;
  return 0;
}
