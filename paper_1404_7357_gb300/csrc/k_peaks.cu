// Arithmetic peaks of the device, measured by kernels that keep one pipe of every
// SM busy (cfft_measure_peak).  The roofline fractions of the tabulation stages
// divide by these: the FP32 FMA pipe (CUDA cores), the FP64 FMA pipe, and the
// fifth-generation tensor cores in the two kinds the library could use for its
// contractions, kind::tf32 (the one it uses, three products per term) and
// kind::f16 with bf16 operands (a cross-check against a cuBLAS bf16 GEMM).
//
// FMA kernels: every thread runs kChains independent multiply-add chains
// x <- x * a + b with |a| < 1, so the values stay finite and no chain waits on
// another; 4 blocks of 256 threads per SM.  The result is stored only when it
// equals an impossible value, so that the compiler keeps every FMA while the
// stores stay out of the timing.
//
// Tensor kernel: one CTA per SM (its shared-memory request leaves no room for a
// second); one thread issues M = 128, N = 256 MMAs over a
// 128-byte-deep K slice of A and B in shared memory (no-swizzle K-major core
// matrices), accumulating into 256 fp32 columns of tensor memory, then commits
// once to an mbarrier and waits with a bound.  A wait that runs out sets the
// error flag; the CTA then waits (again bounded) before it frees tensor memory.
#include <algorithm>

#include "../../include/cfft.h"
#include "cfft_common.cuh"
#include "tc_sm100.cuh"

namespace cfft {
namespace {

constexpr int kChains = 8;
constexpr int kFmaThreads = 256;
constexpr int kFmaBlocksPerSm = 4;
constexpr uint32_t kPeakPolls = 1u << 26;

template <class T>
__global__ void __launch_bounds__(kFmaThreads) fma_peak_kernel(int iters, T a, T b, T* out) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// kind: 0 = tf32 (K = 8 per MMA), 1 = bf16 (K = 16 per MMA); both read 32 bytes of
// K per row per MMA, so the descriptors are the same
constexpr int kMmaM = 128, kMmaN = 256, kSliceBytes = 128;   // K bytes per row in shared memory

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__global__ void __launch_bounds__(128) mma_peak_kernel(int n_mma, int kind, float* out, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t taddr_s;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int s_fail;
  unsigned char* A = smem;                                  // 128 rows x 128 B
  unsigned char* B = smem + kMmaM * kSliceBytes;            // 256 rows x 128 B
  const int tid = threadIdx.x;
  // operands: small finite values (a fixed bit pattern per 32-bit word)
  uint32_t* w = reinterpret_cast<uint32_t*>(smem);
  const int words = (kMmaM + kMmaN) * kSliceBytes / 4;
  for (int i = tid; i < words; i += blockDim.x) {
    const uint32_t h = (uint32_t)(i * 2654435761u) >> 9;
    w[i] = kind == 0 ? (0x3c000000u | (h & 0x007fe000u))           // tf32 in [2^-7, 2^-6)
                     : (0x3c003c00u | (h & 0x007f007fu));          // two bf16 in [2^-7, 2^-6)
  }
  if (tid == 0) {
    s_fail = 0;
    tc::mbar_init(&mbar, 1);
  }
  tc::fence_proxy_async();
  __syncthreads();
  if (tid < 32) {
    tc::tmem_alloc(&taddr_s, kMmaN);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = taddr_s;
  if (tid == 0) {
    const uint32_t idesc = kind == 0
                               ? tc::idesc_tf32(kMmaM, kMmaN)
                               : ((1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kMmaN >> 3) << 17) |
                                  ((uint32_t)(kMmaM >> 4) << 24));
    const uint32_t a0 = tc::smem_u32(A), b0 = tc::smem_u32(B);
    const uint32_t sbo = (kSliceBytes / 16) * 128;
    for (int i = 0; i < n_mma; ++i) {
      const uint32_t ko = (uint32_t)(i & 3) * 256;
      const uint64_t da = tc::sdesc(a0 + ko, 128, sbo), db = tc::sdesc(b0 + ko, 128, sbo);
      if (kind == 0)
        tc::mma_tf32(tmem, da, db, idesc, i > 0 ? 1u : 0u);
      else
        mma_f16(tmem, da, db, idesc, i > 0 ? 1u : 0u);
    }
    tc::mma_commit(&mbar);
    if (!tc::mbar_wait(&mbar, 0, kPeakPolls)) {
      s_fail = 1;
      tc::mbar_wait(&mbar, 0, kPeakPolls);   // bounded: let issued products drain
    }
  }
  __syncthreads();
  tc::fence_after_sync();
  if (!s_fail) {
    // one accumulator column per warp lane group: keeps the products observable
    float v[8];
    tc::tmem_ld8(tmem + ((uint32_t)(32 * (tid >> 5)) << 16), v);
    if (v[0] == -12345.678f) out[blockIdx.x * blockDim.x + tid] = v[0];
  } else if (tid == 0) {
    atomicOr(err, 16);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid < 32) tc::tmem_dealloc(tmem, kMmaN);
}

}  // namespace
}  // namespace cfft

using namespace cfft;

extern "C" cfft_status cfft_measure_peak(int device, int which, int reps, double* tflops,
                                         double* best_ms) {
  if (!tflops || which < 0 || which > 3 || reps < 1 || reps > 100) return CFFT_ERR_ARG;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return CFFT_ERR_ARG;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return CFFT_ERR_CUDA;
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return CFFT_ERR_CUDA;
  cfft_status status = CFFT_OK;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void* out = nullptr;
  int* err = nullptr;
  const int sms = current_sm_count();
  const int fma_blocks = sms * kFmaBlocksPerSm;
  const size_t out_bytes = (size_t)std::max(fma_blocks * kFmaThreads, sms * 128) * sizeof(double);
  // 48 KB of operands, but 116 KB requested: two CTAs never share an SM, so each
  // tensor-memory allocation (256 of the SM's 512 columns) succeeds at once
  const size_t mma_smem = 116 * 1024;
  // work per launch, sized for about 10-40 ms at the nominal rates
  const int fp32_iters = 16384, fp64_iters = 512, mma_count = 32768;
  double flops = 0.0;
  auto launch = [&]() -> cudaError_t {
    switch (which) {
      case 0:
        fma_peak_kernel<float><<<fma_blocks, kFmaThreads, 0, st>>>(fp32_iters, 0.999f, 1e-3f,
                                                                   reinterpret_cast<float*>(out));
        break;
      case 1:
        fma_peak_kernel<double><<<fma_blocks, kFmaThreads, 0, st>>>(fp64_iters, 0.999, 1e-3,
                                                                    reinterpret_cast<double*>(out));
        break;
      default:
        mma_peak_kernel<<<sms, 128, mma_smem, st>>>(mma_count, which - 2, reinterpret_cast<float*>(out), err);
        break;
    }
    return cudaGetLastError();
  };
  if (which <= 1) {
    const int iters = which == 0 ? fp32_iters : fp64_iters;
    flops = 2.0 * kChains * 16.0 * iters * (double)fma_blocks * kFmaThreads;
  } else {
    const int k = which == 2 ? 8 : 16;
    flops = 2.0 * kMmaM * kMmaN * k * (double)mma_count * sms;
  }
  do {
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMalloc(&out, out_bytes) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess ||
        cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) {
      status = CFFT_ERR_CUDA;
      break;
    }
    if (which >= 2 && cudaFuncSetAttribute(mma_peak_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)mma_smem) != cudaSuccess) {
      status = CFFT_ERR_CUDA;
      break;
    }
    if (launch() != cudaSuccess) {   // warm-up (clocks up, code loaded)
      status = CFFT_ERR_CUDA;
      break;
    }
    float best = 1e30f;
    for (int r = 0; r < reps && status == CFFT_OK; ++r) {
      float ms = 0.f;
      if (cudaEventRecord(e0, st) != cudaSuccess || launch() != cudaSuccess ||
          cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        status = CFFT_ERR_CUDA;
      else
        best = std::min(best, ms);
    }
    if (status != CFFT_OK) break;
    int flag = 0;
    if (cudaMemcpy(&flag, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      status = CFFT_ERR_CUDA;
      break;
    }
    if (flag) {
      status = CFFT_ERR_TIMEOUT;
      break;
    }
    *tflops = flops / (best * 1e-3) / 1e12;
    if (best_ms) *best_ms = best;
  } while (false);
  if (out) cudaFree(out);
  if (err) cudaFree(err);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaGetLastError();
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return status;
}
