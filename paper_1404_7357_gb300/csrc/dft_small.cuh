// Small in-register DFTs (forward, W_N = exp(-2 pi i / N)) shared by the FFT
// passes and the folded angular transforms.
#pragma once

#include "cfft_common.cuh"

namespace cfft {

// 4-point DFT in place
template <class T>
__device__ __forceinline__ void dft4(cpx<T>& x0, cpx<T>& x1, cpx<T>& x2, cpx<T>& x3) {
  const cpx<T> s02 = x0 + x2, d02 = x0 - x2, s13 = x1 + x3, d13 = x1 - x3;
  const cpx<T> mid = mk(d13.im, -d13.re);  // -i (x1 - x3)
  x0 = s02 + s13;
  x1 = d02 + mid;
  x2 = s02 - s13;
  x3 = d02 - mid;
}

// 8-point DFT in place: r = 2 r1 + r0, radix-4 over r1, twiddle W_8^{r0 s0}, radix-2 over r0
template <class T>
__device__ __forceinline__ void dft8(cpx<T>* v) {
  cpx<T> a[2][4];
#pragma unroll
  for (int r0 = 0; r0 < 2; ++r0) {
#pragma unroll
    for (int r1 = 0; r1 < 4; ++r1) a[r0][r1] = v[2 * r1 + r0];
    dft4(a[r0][0], a[r0][1], a[r0][2], a[r0][3]);
  }
  const T h = (T)0.70710678118654752440;
  a[1][1] = mk(h * (a[1][1].re + a[1][1].im), h * (a[1][1].im - a[1][1].re));     // * W_8
  a[1][2] = mk(a[1][2].im, -a[1][2].re);                                            // * W_8^2
  a[1][3] = mk(h * (a[1][3].im - a[1][3].re), -h * (a[1][3].re + a[1][3].im));    // * W_8^3
#pragma unroll
  for (int s0 = 0; s0 < 4; ++s0) {
    v[s0] = a[0][s0] + a[1][s0];
    v[s0 + 4] = a[0][s0] - a[1][s0];
  }
}

}  // namespace cfft
