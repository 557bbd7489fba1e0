// The effective homogeneous medium and its image through the ground plane: the part of
// the grounded-slab Green's function that Sections II and III-A move to Z^h (treated
// there in the space domain), so that the tabulated remainder Z^l decays faster in beta.
// Reading: a current sheet in a homogeneous medium of permittivity eps_eff (mu_0), the
// ground plane h below it, which is a matched line in parallel with a shorted line of the
// same medium:
//   Z = Z_c (1 - exp(-2 j kz h)) / 2,  Z_c^TE = k0 Z0 / kz,  Z_c^TM = Z0 kz / (k0 eps_eff),
//   kz = -j sqrt(beta^2 - eps_eff k0^2)  (Im kz <= 0, the radiation condition),
// and in the form G = P I - R k k^T of the slab: P = -Z_TE, R beta^2 = Z_TM - Z_TE.  With
// eps_eff = (eps_r + 1) / 2 the large-beta TM term (the charge term, growing like beta)
// equals the slab's, so the remainder loses its dominant part; for eps_r = 1 the slab is
// free space above a ground plane and the remainder vanishes.
// (1 - exp(-2 j kz h)) / kz = 2 j h exp(-j kz h) sinc(kz h) keeps Z_TE regular at kz = 0.
#pragma once

#include "cfft_common.cuh"

namespace cfft {

struct GreenExt {
  cpx<double> p, rb2;              // P and R beta^2 of the extracted part
  cpx<double> dp[2], drb2[2];      // their derivatives: [0] d/d eps_r, [1] d/d h
};

__device__ inline GreenExt ext_green(cpx<double> bc, double eps_eff, double deps_eff, double hs, double k0,
                                     bool derivs) {
  constexpr double kZ0 = 376.730313668;
  GreenExt g;
  const cpx<double> b2 = bc * bc;
  const double k02 = k0 * k0;
  cpx<double> arg = mk(b2.re - eps_eff * k02, b2.im);
  if (arg.im == 0.0) arg.im = 0.0;   // +0: real beta below the medium's wavenumber gives kz > 0
  const cpx<double> r = csqrt_(arg);
  const cpx<double> kz = mk(r.im, -r.re);   // -j sqrt(.)
  const cpx<double> u = mk(kz.re * hs, kz.im * hs);
  // exp(-j u) = exp(u.im) (cos u.re - j sin u.re)
  const double eu = exp(u.im);
  double su, cu;
  sincos(u.re, &su, &cu);
  const cpx<double> emj = mk(eu * cu, -eu * su);
  const cpx<double> s = emj * csinc(u);                     // exp(-j kz h) sinc(kz h)
  const cpx<double> zte = mk(0.0, k0 * kZ0 * hs) * s;       // j k0 Z0 h S
  const cpx<double> ztm = (mk(0.0, kZ0 * hs / (k0 * eps_eff)) * s) * (kz * kz);
  g.p = mk(-zte.re, -zte.im);
  g.rb2 = ztm - zte;
  if (derivs) {
    const cpx<double> e2 = emj * emj;                        // exp(-2 j kz h)
    const cpx<double> f = mk(1.0 - e2.re, -e2.im);
    // d/d h: df/dh = 2 j kz E
    const cpx<double> dte_h = mk(0.0, k0 * kZ0) * e2;
    const cpx<double> dtm_h = (mk(0.0, kZ0 / (k0 * eps_eff)) * e2) * (kz * kz);
    // d/d eps_r through eps_eff: dkz = k0^2 deps / (2 kz), df = 2 j h E dkz
    const cpx<double> dkz = cdiv(mk(0.5 * k02 * deps_eff, 0.0), kz);
    const cpx<double> df = (mk(0.0, 2.0 * hs) * e2) * dkz;
    const cpx<double> dte_e = (0.5 * k0 * kZ0) * (cdiv(df, kz) - cdiv(f * dkz, kz * kz));
    const cpx<double> dtm_e = (0.5 * kZ0 / k0) * ((1.0 / eps_eff) * (dkz * f + kz * df) -
                                                  (deps_eff / (eps_eff * eps_eff)) * (kz * f));
    g.dp[0] = mk(-dte_e.re, -dte_e.im);
    g.drb2[0] = dtm_e - dte_e;
    g.dp[1] = mk(-dte_h.re, -dte_h.im);
    g.drb2[1] = dtm_h - dte_h;
  }
  return g;
}

}  // namespace cfft
