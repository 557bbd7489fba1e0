// Contour nodes (Eq. 8) and the grounded-slab Green's function along them.
//
// One thread per rectangle-rule node j (Eq. 23): beta_R = (j + 1/2) step,
// beta_I the parabola of peak `height` on [0, beta_p] (Fig. 1), and the
// Jacobian weight step * (1 + i dbeta_I/dbeta_R).  The grounded-slab dyadic
// of Eq. 6/10 is written as G = P(beta) I - R(beta) k k^T: for a horizontally
// isotropic slab every tangential dyadic has this form, so only two scalars
// per node are needed and the angular dependence enters through k alone.
// With exp(+j w t), k1 = sqrt(eps_r k0^2 - beta^2) (any branch: G is even in
// k1), k2 = -j sqrt(beta^2 - k0^2) (Im k2 <= 0), c = cos k1 h, s = sin k1 h:
//   Te = k1 c + j k2 s,  Tm = eps_r k2 c + j k1 s   (TE / TM denominators)
//   P = -j Z0/k0 s (eps_r k0^2 k2 c + j k0^2 k1 s) / (Te Tm)
//   R = -j Z0/k0 s (k2 c + j k1 s) / (Te Tm)
// Everything here is float64: the denominators near the surface-wave poles and
// the branch-point square roots are where float32 loses the most digits.
#include "cfft_common.cuh"
#include "es_weights.cuh"
#include "green_ext.cuh"

namespace cfft {

namespace {

constexpr double kEta0 = 376.730313668;  // free-space wave impedance, ohm

__device__ __forceinline__ void contour_node(const ContourArgs& a, const ContourData& d, int j) {
  double br = (j + 0.5) * a.step;
  double bi = 0.0, slope = 0.0;
  if (br < a.beta_p) {
    double ip2 = 1.0 / (a.beta_p * a.beta_p);
    bi = 4.0 * a.height * br * (a.beta_p - br) * ip2;
    slope = 4.0 * a.height * (a.beta_p - 2.0 * br) * ip2;
  }
  cpx<double> bc = mk(br, bi);
  cpx<double> w = mk(a.step, a.step * slope);
  cpx<double> b2 = bc * bc;
  double k02 = a.k0 * a.k0;
  cpx<double> k1 = csqrt_(mk(a.eps_r * k02 - b2.re, -b2.im));
  cpx<double> arg2 = mk(b2.re - k02, b2.im);
  if (arg2.im == 0.0) arg2.im = 0.0;  // +0: real beta < k0 gives k2 > 0 (outgoing)
  cpx<double> r2 = csqrt_(arg2);
  cpx<double> k2 = mk(r2.im, -r2.re);  // -j * sqrt(.)
  cpx<double> sn, cs;
  csincos(mk(k1.re * a.hs, k1.im * a.hs), &sn, &cs);
  cpx<double> j1 = mk(0.0, 1.0);
  cpx<double> te = k1 * cs + j1 * (k2 * sn);
  cpx<double> tm = a.eps_r * (k2 * cs) + j1 * (k1 * sn);
  // C = -j eta0/k0 * s / (Te Tm)
  cpx<double> cfac = cdiv(mk(0.0, -kEta0 / a.k0) * sn, te * tm);
  cpx<double> p = cfac * ((a.eps_r * k02) * (k2 * cs) + j1 * (k02 * (k1 * sn)));
  cpx<double> r = cfac * (k2 * cs + j1 * (k1 * sn));
  GreenExt ge{};
  if (a.extract) {
    ge = ext_green(bc, a.eps_eff, a.deps_eff, a.hs, a.k0, d.dp_eps != nullptr);
    p = p - ge.p;
  }
  d.beta_c[j] = make_double2(bc.re, bc.im);
  d.weight[j] = make_double2(w.re, w.im);
  cpx<double> bw = bc * w;
  d.bw[j] = make_double2(bw.re, bw.im);
  d.bi_rel[j] = a.height > 0.0 ? bi / a.height : 0.0;
  if (d.bi_rel_f) d.bi_rel_f[j] = (float)d.bi_rel[j];
  d.green_p[j] = make_double2(p.re, p.im);
  cpx<double> rb2 = r * b2;  // R beta_c^2: the k k^T term is R beta_c^2 u u^T
  if (a.extract) rb2 = rb2 - ge.rb2;
  d.green_r[j] = make_double2(rb2.re, rb2.im);
  if (d.dp_eps) {
    // derivatives with respect to eps_r (dk1 = k0^2 / (2 k1)) and h (k2 does not
    // depend on either): c' = -s (k1 h)', s' = c (k1 h)', then the quotient rule
    // on C = -j eta0/k0 s / (Te Tm) and the products P = C N_P, R = C N_R
    for (int which = 0; which < 2; ++which) {
      const bool eps = which == 0;
      cpx<double> dk1 = eps ? cdiv(mk(0.5 * k02, 0.0), k1) : mk(0.0, 0.0);
      cpx<double> darg = eps ? mk(dk1.re * a.hs, dk1.im * a.hs) : k1;  // d(k1 h)
      cpx<double> dc = mk(0.0, 0.0) - sn * darg;
      cpx<double> ds = cs * darg;
      double de = eps ? 1.0 : 0.0;
      cpx<double> dte = dk1 * cs + k1 * dc + j1 * (k2 * ds);
      cpx<double> dtm = de * (k2 * cs) + a.eps_r * (k2 * dc) + j1 * (dk1 * sn + k1 * ds);
      cpx<double> tt = te * tm;
      cpx<double> dtt = dte * tm + te * dtm;
      // dC = -j eta0/k0 (ds Te Tm - s d(Te Tm)) / (Te Tm)^2
      cpx<double> dcf = cdiv(mk(0.0, -kEta0 / a.k0) * (ds * tt - sn * dtt), tt * tt);
      cpx<double> np = (a.eps_r * k02) * (k2 * cs) + j1 * (k02 * (k1 * sn));
      cpx<double> dnp = (de * k02) * (k2 * cs) + (a.eps_r * k02) * (k2 * dc) +
                        j1 * (k02 * (dk1 * sn + k1 * ds));
      cpx<double> nr = k2 * cs + j1 * (k1 * sn);
      cpx<double> dnr = k2 * dc + j1 * (dk1 * sn + k1 * ds);
      cpx<double> dp = dcf * np + cfac * dnp;
      cpx<double> dr = (dcf * nr + cfac * dnr) * b2;
      if (a.extract) {
        dp = dp - ge.dp[which];
        dr = dr - ge.drb2[which];
      }
      (eps ? d.dp_eps : d.dp_h)[j] = make_double2(dp.re, dp.im);
      (eps ? d.dr_eps : d.dr_h)[j] = make_double2(dr.re, dr.im);
    }
  }
  if (d.prec) {
    // precorrection of the transform input for the ES back-projection: the node's
    // demodulated frequency in grid units, omega = (beta_c - beta_max / 2) ds
    d.prec[j] = es_precorrection((float)((br - 0.5 * a.beta_max) * a.ds), (float)(bi * a.ds), a.es_width);
  }
}

__global__ void contour_kernel(ContourArgs a, ContourData d) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < a.n) contour_node(a, d, j);
}

// batched form: block b covers nodes map[b].y .. + 255 of item map[b].x
__global__ void contour_batch_kernel(const ContourArgs* items, const ContourData* data,
                                     const int2* map) {
  const int2 bm = map[blockIdx.x];
  const ContourArgs a = items[bm.x];
  const ContourData d = data[bm.x];
  int j = bm.y + threadIdx.x;
  if (j < a.n) contour_node(a, d, j);
}

template <class T>
__global__ void twiddle_kernel(cpx<T>* tw, int len) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= len) return;
  double s, c;
  sincospi(-2.0 * (double)t / (double)len, &s, &c);
  tw[t] = mk((T)c, (T)s);
}

// table of class (90, 90) = class (0, 0) times (-i)^q: both elements rotated by
// the same angle theta multiply harmonic q by exp(-i q theta)
template <class T>
__global__ void class_phase_kernel(cpx<T>* table, int pairs, int n_harm, int q_max,
                                   int n_rho) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t per_class = (int64_t)pairs * n_harm * n_rho;
  if (idx >= per_class) return;
  int qi = (int)((idx / n_rho) % n_harm);
  int q = qi - q_max;
  int m = ((q % 4) + 4) % 4;  // (-i)^q = (-i)^(q mod 4)
  cpx<T> v = table[idx];
  cpx<T> o;
  if (m == 0) o = v;
  else if (m == 1) o = mk(v.im, -v.re);     // -i v
  else if (m == 2) o = mk(-v.re, -v.im);    // -v
  else o = mk(-v.im, v.re);                 // +i v
  table[3 * per_class + idx] = o;
}

template <class T>
__global__ void nonfinite_kernel(const cpx<T>* buf, int64_t count, int* flag) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (; i < count; i += stride) {
    cpx<T> v = buf[i];
    bad |= !isfinite(v.re) || !isfinite(v.im);
  }
  if (bad) atomicOr(flag, 1);
}

}  // namespace

void launch_contour(const ContourArgs& a, const ContourData& d, cudaStream_t s) {
  contour_kernel<<<(a.n + 255) / 256, 256, 0, s>>>(a, d);
}

void launch_contour_batch(const ContourArgs* items, const ContourData* data, const int2* map,
                          int n_blocks, cudaStream_t s) {
  contour_batch_kernel<<<n_blocks, 256, 0, s>>>(items, data, map);
}

template <class T>
void launch_twiddle(cpx<T>* tw, int len, cudaStream_t s) {
  twiddle_kernel<T><<<(len + 255) / 256, 256, 0, s>>>(tw, len);
}

template <class T>
void launch_class_phase(cpx<T>* table, int pairs, int n_harm, int q_max, int n_rho,
                        cudaStream_t s) {
  int64_t n = (int64_t)pairs * n_harm * n_rho;
  class_phase_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(table, pairs, n_harm,
                                                                     q_max, n_rho);
}

template <class T>
void launch_nonfinite(const cpx<T>* buf, int64_t count, int* flag, cudaStream_t s) {
  int blocks = (int)((count + 255) / 256);
  if (blocks > 4 * current_sm_count()) blocks = 4 * current_sm_count();
  if (blocks < 1) blocks = 1;
  nonfinite_kernel<T><<<blocks, 256, 0, s>>>(buf, count, flag);
}

template void launch_twiddle<float>(cpx<float>*, int, cudaStream_t);
template void launch_twiddle<double>(cpx<double>*, int, cudaStream_t);
template void launch_class_phase<float>(cpx<float>*, int, int, int, int, cudaStream_t);
template void launch_class_phase<double>(cpx<double>*, int, int, int, int, cudaStream_t);
template void launch_nonfinite<float>(const cpx<float>*, int64_t, int*, cudaStream_t);
template void launch_nonfinite<double>(const cpx<double>*, int64_t, int*, cudaStream_t);

}  // namespace cfft
