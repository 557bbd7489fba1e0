// Weights of the ES ("exponential of semicircle") interpolation kernel for the FP32-mixed
// back-projection, and its Fourier transform for the spectral precorrection.
//
// phi(x) = exp(beta (sqrt(1 - (2x/w)^2) - 1)) on |x| <= w/2.  A function band-limited to
// |omega| <= pi / sigma (grid units) is recovered at any u from samples of its spectrally
// precorrected form, G'(k) = sum_j c_j / phi_hat(omega_j) exp(-i omega_j k), as
// sum_k G'(k) phi(u - k): the Poisson sum of e^{-i omega k} phi(u - k) is
// sum_m phi_hat(omega + 2 pi m) e^{-i (omega + 2 pi m) u}, and the terms m != 0 (the
// aliasing error) are below 2e-6 (w = 6) and 1e-8 (w = 8) of the m = 0 term for sigma = 4.
// Against Lagrange interpolation of the same accuracy this halves the taps (12 -> 6).
#pragma once
#include "es_kernel.cuh"

namespace cfft {

template <int TAPS>
struct EsTable;
template <>
struct EsTable<6> {
  static constexpr int kDeg = 7;
  __device__ static __forceinline__ float c(int m, int d) { return kEsPoly6[m][d]; }
};
template <>
struct EsTable<8> {
  static constexpr int kDeg = 9;
  __device__ static __forceinline__ float c(int m, int d) { return kEsPoly8[m][d]; }
};

// the TAPS weights phi(f + TAPS/2 - 1 - m), m = 0..TAPS-1, of a stencil whose base is
// floor(u), f = u - floor(u) in [0, 1): one polynomial in f per tap (Horner)
template <int TAPS>
__device__ __forceinline__ void es_weights(float f, float* w) {
  constexpr int D = EsTable<TAPS>::kDeg;
#pragma unroll
  for (int m = 0; m < TAPS; ++m) {
    float v = EsTable<TAPS>::c(m, D);
#pragma unroll
    for (int d = D - 1; d >= 0; --d) v = fmaf(v, f, EsTable<TAPS>::c(m, d));
    w[m] = v;
  }
}

// 1 / phi_hat(omega) for complex omega = wr + i wi (grid units), phi of width `width`
// (6 or 8): phi_hat(omega) = 2 int_0^{w/2} phi(x) cos(omega x) dx by Gauss-Legendre,
// cos((wr + i wi) x) = cos(wr x) cosh(wi x) - i sin(wr x) sinh(wi x)
__device__ __forceinline__ float2 es_precorrection(float wr, float wi, int width) {
  const float* qx = width == 8 ? kEsQuadX8 : kEsQuadX6;
  const float* qw = width == 8 ? kEsQuadW8 : kEsQuadW6;
  float re = 0.f, im = 0.f;
  for (int q = 0; q < kEsQuad; ++q) {
    const float x = qx[q];
    float sv, cv;
    sincosf(wr * x, &sv, &cv);
    re = fmaf(qw[q], cv * coshf(wi * x), re);
    im = fmaf(-qw[q], sv * sinhf(wi * x), im);
  }
  re *= 2.f;
  im *= 2.f;
  const float inv = 1.f / (re * re + im * im);
  return make_float2(re * inv, -im * inv);
}

}  // namespace cfft
