// Shared pieces of the tensor-core MBF spectra (Eq. 11 as a GEMM): chunking of
// the basis dimension, the TF32 head/tail split of an FP32 value, the rooftop shape factor
// and the column layout of the accumulator.  The B operand (a constant of the
// element) is built on the host by spectra_tc_bmatrix.
#pragma once

#include "cfft_common.cuh"

namespace cfft {

constexpr int kTcBasis = 8;                // basis functions per K chunk
constexpr int kTcK = 4 * kTcBasis;         // K per chunk (floats: Re E, Im E, Re E', Im E')
constexpr uint32_t kTcPolls = 1u << 26;    // bound of every mbarrier wait

// columns of one (side, class) group: 2 M reals (re, im per MBF), padded to 8 so that
// every group starts on an 8-column boundary of the accumulator
__host__ __device__ constexpr int tc_group_cols(int m) { return 2 * m > 8 ? 2 * m : 8; }

// MBF count as compiled (1, 2, 4, 8; padding columns of Q are zero)
__host__ __device__ inline int tc_mbf_pad(int n_mbf) { return n_mbf <= 1 ? 1 : n_mbf <= 2 ? 2 : n_mbf <= 4 ? 4 : 8; }

// x = hi + lo exactly, hi with 11 significant bits (a TF32 value, nearest to x, ties
// away from zero: half a TF32 unit added to the magnitude bits, then the 13 low bits
// cleared), lo = x - hi (exact, at most 12 significant bits).  The tensor core reads
// lo to TF32 precision, so the product uses x to within 2^-11 |lo| <= 2^-22 |x|.
// Two integer operations and one rounded subtraction.
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
  lo = __fsub_rn(x, hi);
}

// closed-form rooftop transform a sinc^2(k_u a/2) sinc(k_v w/2) at complex k
__device__ __forceinline__ cpx<float> rooftop_factor(const ShapeClass& c, cpx<float> kx, cpx<float> ky) {
  const float a = (float)c.p1, w = (float)c.p2;
  const cpx<float> ku = c.dir == 0 ? kx : ky;
  const cpx<float> kv = c.dir == 0 ? ky : kx;
  const cpx<float> s1 = csinc(mk(ku.re * a * 0.5f, ku.im * a * 0.5f));
  const cpx<float> s2 = csinc(mk(kv.re * w * 0.5f, kv.im * w * 0.5f));
  return a * (s1 * s1 * s2);
}

}  // namespace cfft
