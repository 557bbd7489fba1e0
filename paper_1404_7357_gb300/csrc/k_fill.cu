// Reduced-matrix fill by interpolation in the reaction table (Section III-B-3).
//
// For test element m and basis element n, Delta = r_m - r_n = rho (cos phi,
// sin phi) and the rotation class cls of (rot_m, rot_n); every MBF pair (a, b)
// of the block Z'_mn (Eq. 3) is
//   Z'[(m, a), (n, b)] = sum_q exp(i q phi) Z^{cls}_ab,q(rho)
// with Z_ab,q(rho) interpolated by a taps-point Lagrange stencil on the
// table's uniform rho grid.  Rows below rho = 0 come from the parity of the
// harmonics, Z_q(-rho) = (-1)^q Z_q(rho) (J_q(-x) = (-1)^q J_q(x)); near
// rho_max the stencil is shifted inward.  rho and the stencil position are
// formed in float64 from float64 positions (an error of 1e-5 wavelength in rho
// is already a 1e-4 phase error at the top of the spectrum); exp(i phi) is
// (Delta_x, Delta_y) / rho and exp(i q phi) follows by recurrence.
// One thread per element pair; the lanes of a warp take consecutive basis
// elements n so that each output row segment is written contiguously.
#include "cfft_common.cuh"

namespace cfft {

namespace {

constexpr int kMaxM = 8;
constexpr int kMaxTaps = 16;

template <class T, class TO>
__global__ void __launch_bounds__(128) fill_kernel(FillArgs<T, TO> a) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (n >= a.n_el || m >= a.n_el) return;
  const int M = a.n_mbf;
  const int pairs = M * M;
  const double dx = a.pos[2 * m] - a.pos[2 * n];
  const double dy = a.pos[2 * m + 1] - a.pos[2 * n + 1];
  const double rho = sqrt(dx * dx + dy * dy);
  cpx<TO>* zrow = a.z + (size_t)m * M * a.ld + (size_t)n * M;
  if (!(rho <= a.rho_max * (1.0 + 1e-12))) {
    atomicOr(a.err, 1);
    for (int ia = 0; ia < M; ++ia)
      for (int ib = 0; ib < M; ++ib) zrow[(size_t)ia * a.ld + ib] = mk((TO)0, (TO)0);
    return;
  }
  cpx<T> e1 = rho > 0.0 ? mk((T)(dx / rho), (T)(dy / rho)) : mk((T)1, (T)0);
  const int cls = (a.n_cls == 1 || a.rot == nullptr) ? 0 : 2 * (a.rot[m] != 0) + (a.rot[n] != 0);
  // stencil rows i0 .. i0 + taps - 1, weights at x = u - i0
  const double u = rho * a.inv_d_rho;
  int i0 = (int)floor(u) - (a.taps / 2 - 1);
  if (i0 + a.taps > a.n_rho) i0 = a.n_rho - a.taps;
  const T x = (T)(u - (double)i0);
  T w[kMaxTaps];
  {
    T pre = (T)1;
#pragma unroll
    for (int t = 0; t < kMaxTaps; ++t)
      if (t < a.taps) {
        w[t] = pre;
        pre *= (x - (T)t);
      }
    T suf = (T)1;
#pragma unroll
    for (int t = kMaxTaps - 1; t >= 0; --t)
      if (t < a.taps) {
        // 1 / prod_{s != t} (t - s) = (-1)^(taps-1-t) / (t! (taps-1-t)!)
        T den = (T)1;
        for (int s2 = 1; s2 <= t; ++s2) den *= (T)s2;
        for (int s2 = 1; s2 <= a.taps - 1 - t; ++s2) den *= (T)s2;
        if ((a.taps - 1 - t) & 1) den = -den;
        w[t] *= suf / den;
        suf *= (x - (T)t);
      }
  }
  const cpx<T>* tab = a.table + (size_t)cls * pairs * a.n_harm * a.n_rho;
  // exp(i q phi) for q = -q_max: conj(e1)^q_max
  cpx<T> zq = mk((T)1, (T)0);
  for (int k = 0; k < a.q_max; ++k) zq = zq * conj(e1);
  for (int ia = 0; ia < M; ++ia) {
    cpx<T> acc[kMaxM];
#pragma unroll
    for (int ib = 0; ib < kMaxM; ++ib) acc[ib] = mk((T)0, (T)0);
    cpx<T> ph = zq;
    for (int qi = 0; qi < a.n_harm; ++qi) {
      const int q = qi - a.q_max;
      const bool odd = (q & 1) != 0;
#pragma unroll
      for (int ib = 0; ib < kMaxM; ++ib) {
        if (ib < M) {
          const cpx<T>* row = tab + ((size_t)(ia * M + ib) * a.n_harm + qi) * a.n_rho;
          cpx<T> v = mk((T)0, (T)0);
#pragma unroll
          for (int t = 0; t < kMaxTaps; ++t) {
            if (t < a.taps) {
              int r = i0 + t;
              T wt = w[t];
              if (r < 0) {
                r = -r;
                if (odd) wt = -wt;
              }
              v = v + wt * row[r];
            }
          }
          cmac(acc[ib], ph, v);
        }
      }
      ph = ph * e1;
    }
#pragma unroll
    for (int ib = 0; ib < kMaxM; ++ib)
      if (ib < M) zrow[(size_t)ia * a.ld + ib] = mk((TO)acc[ib].re, (TO)acc[ib].im);
  }
}

}  // namespace

template <class T, class TO>
cudaError_t launch_fill(const FillArgs<T, TO>& a, cudaStream_t s) {
  if (a.n_mbf > kMaxM || a.taps > kMaxTaps || a.taps < 2) return cudaErrorInvalidValue;
  dim3 grid((a.n_el + 127) / 128, a.n_el);
  fill_kernel<T, TO><<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_fill<float, float>(const FillArgs<float, float>&, cudaStream_t);
template cudaError_t launch_fill<float, double>(const FillArgs<float, double>&, cudaStream_t);
template cudaError_t launch_fill<double, double>(const FillArgs<double, double>&, cudaStream_t);
template cudaError_t launch_fill<double, float>(const FillArgs<double, float>&, cudaStream_t);

}  // namespace cfft
