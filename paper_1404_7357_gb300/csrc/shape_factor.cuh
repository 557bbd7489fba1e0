// Closed-form transform S_c(k) of the shape class of an element's basis functions, at
// complex k (the analytic extension of Eq. 18): rooftop a sinc^2(k_u a / 2) sinc(k_v w / 2),
// cosine strip 2 pi L cos(k_x L / 2) / (pi^2 - k_x^2 L^2) sinc(k_y W / 2).  Both are even in
// k.  Used by the SIMT integrand and by the Cartesian spectrum.
#pragma once

#include "cfft_common.cuh"

namespace cfft {

template <class T>
__device__ __forceinline__ cpx<T> shape_factor(const ShapeClass& c, cpx<T> kx, cpx<T> ky) {
  if (c.kind == 0) {
    const T a = (T)c.p1, w = (T)c.p2;
    cpx<T> ku = c.dir == 0 ? kx : ky;
    cpx<T> kv = c.dir == 0 ? ky : kx;
    cpx<T> s1 = csinc(mk(ku.re * a * (T)0.5, ku.im * a * (T)0.5));
    cpx<T> s2 = csinc(mk(kv.re * w * (T)0.5, kv.im * w * (T)0.5));
    return a * (s1 * s1 * s2);
  }
  // cosine strip along x: cos(u) / (pi^2/4 - u^2) = sinc(pi/2 - u) / (pi/2 + u),
  // with u = kx L/2 mirrored into Re u >= 0 (the factor is even in u)
  const T len = (T)c.p1, wid = (T)c.p2;
  cpx<T> u = mk(kx.re * len * (T)0.5, kx.im * len * (T)0.5);
  if (u.re < (T)0) u = mk(-u.re, -u.im);
  const T hp = (T)1.5707963267948966;
  cpx<T> num = csinc(mk(hp - u.re, -u.im));
  cpx<T> along = cdiv(num, mk(hp + u.re, u.im));
  along = ((T)1.5707963267948966 * len) * along;  // (pi L / 2)
  cpx<T> across = csinc(mk(ky.re * wid * (T)0.5, ky.im * wid * (T)0.5));
  return along * across;
}

}  // namespace cfft
