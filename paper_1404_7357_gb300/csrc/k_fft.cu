// Taylor-expanded contour transform by batched, pruned, zero-padded FFTs.
//
// Along the contour beta_c,j = beta_R,j + i beta_I,j the transform in beta
//   g_q(s) = sum_j Y_q[j] exp(-i beta_c,j s)
//          = sum_j Y_q[j] exp(beta_I,j s) exp(-i beta_R,j s)
// is not a Fourier sum because of the real exponential (Section III-B-3).  The
// real exponential is expanded in a Taylor series (Eq. 22) and every term is a
// plain DFT with the Delta-dependence moved outside the sum (Eq. 23):
//   g_q(s) = sum_n (H s)^n / n! * sum_j (beta_I,j / H)^n Y_q[j] exp(-i beta_R,j s)
// with H the contour height (so (beta_I/H)^n <= 1 and (H s)^n/n! stays small).
// On the grid s_k = k ds, ds = 2 pi / (P step), P = sigma * n (zero padding by
// sigma) and beta_R,j = (j + 1/2) step, each inner sum is a length-P DFT of the
// zero-padded sequence times the half-sample phase exp(-i pi k / P).  Only
// |k| <= K is needed (|s| <= rho_max plus the interpolation stencil), and the
// sequence is non-zero only for j < n (and, for n >= 1, only where beta_I > 0),
// so the length-P transform is decomposed (k = D t + k2, D = P / L):
//   X[D t + k2] = sum_{j'<L} W_L^{j' t} [ sum_m x_{j'+mL} W_P^{(j'+mL) k2} ]
// i.e. for every residue k2 one length-L FFT of a folded, pre-twiddled input.
// One CTA owns one (series, k2): it loops over the Taylor terms, runs each
// length-L FFT in shared memory (radix-4 Stockham passes staged through
// registers), and accumulates (H s_k)^n/n! times the needed outputs.  The
// result is written demodulated by exp(+i beta_max s / 2) so that the
// back-projection interpolates a function whose spectrum is centred on zero:
//   grid[series][k + K] = g_q(s_k) exp(i pi k / sigma),   k = -K..K.
#include "cfft_common.cuh"

namespace cfft {

namespace {

template <class T>
__device__ __forceinline__ cpx<T> powi_scale(T b, int n) {
  // b^n by binary exponentiation (returned in .re)
  T r = (T)1, x = b;
  while (n > 0) {
    if (n & 1) r *= x;
    x *= x;
    n >>= 1;
  }
  return mk(r, (T)0);
}

template <class T, int LOG2L, int NT>
__device__ __forceinline__ void fft_inplace(cpx<T>* buf, const cpx<T>* __restrict__ tw) {
  constexpr int L = 1 << LOG2L;
  constexpr int VPT = L / NT;  // values per thread per pass
  static_assert(VPT >= 4 && VPT % 4 == 0, "at least one radix-4 butterfly per thread");
  const int tid = threadIdx.x;
  int p = 1;
  if (LOG2L & 1) {
    constexpr int T2 = L / 2;
    cpx<T> v[VPT];
#pragma unroll
    for (int b = 0; b < VPT / 2; ++b) {
      int i = tid + NT * b;
      v[2 * b] = buf[i];
      v[2 * b + 1] = buf[i + T2];
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < VPT / 2; ++b) {
      int i = tid + NT * b;  // span 1: no twiddle, output index 2 i
      buf[2 * i] = v[2 * b] + v[2 * b + 1];
      buf[2 * i + 1] = v[2 * b] - v[2 * b + 1];
    }
    __syncthreads();
    p = 2;
  }
  for (; p < L; p *= 4) {
    constexpr int T4 = L / 4;
    cpx<T> v[VPT];
#pragma unroll
    for (int b = 0; b < VPT / 4; ++b) {
      int i = tid + NT * b;
#pragma unroll
      for (int r = 0; r < 4; ++r) v[4 * b + r] = buf[i + r * T4];
    }
    __syncthreads();
    const int stride = L / (4 * p);
#pragma unroll
    for (int b = 0; b < VPT / 4; ++b) {
      int i = tid + NT * b;
      int k = i & (p - 1);
      cpx<T> x0 = v[4 * b];
      cpx<T> x1 = v[4 * b + 1] * tw[k * stride];
      cpx<T> x2 = v[4 * b + 2] * tw[2 * k * stride];
      cpx<T> x3 = v[4 * b + 3] * tw[3 * k * stride];
      cpx<T> s02 = x0 + x2, d02 = x0 - x2, s13 = x1 + x3, d13 = x1 - x3;
      cpx<T> mid = mk(d13.im, -d13.re);  // -i (x1 - x3)
      int j = (i - k) * 4 + k;
      buf[j] = s02 + s13;
      buf[j + p] = d02 + mid;
      buf[j + 2 * p] = s02 - s13;
      buf[j + 3 * p] = d02 - mid;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int floor_div(int a, int b) {  // b > 0
  int q = a / b;
  return (a % b != 0 && a < 0) ? q - 1 : q;
}

template <class T, int LOG2L, int NT>
__global__ void __launch_bounds__(NT) fft_taylor_kernel(FftArgs<T> a) {
  constexpr int L = 1 << LOG2L;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  const int series = blockIdx.x;
  const int k2 = blockIdx.y;
  const int D = a.n_sub;
  const int K = a.grid_half;
  const int t_lo = -floor_div(K + k2, D);     // ceil((-K - k2) / D)
  const int t_hi = floor_div(K - k2, D);
  const int n_out = t_hi - t_lo + 1;
  cpx<T>* acc = buf + L;
  T* fac = reinterpret_cast<T*>(acc + n_out);
  const int tid = threadIdx.x;
  const int64_t P = a.fft_len;
  const cpx<T>* y = a.y + (size_t)series * a.n;

  for (int o = tid; o < n_out; o += NT) {
    acc[o] = mk((T)0, (T)0);
    fac[o] = (T)1;
  }
  for (int n = 0; n <= a.taylor; ++n) {
    const int lim = n == 0 ? a.n : a.n_active;
    // ---- fold + pre-twiddle W_P^{j k2} + Taylor weight (beta_I/H)^n
    for (int jp = tid; jp < L; jp += NT) {
      cpx<T> v = mk((T)0, (T)0);
      for (int j = jp; j < lim; j += L) {
        cpx<T> x = y[j];
        if (n > 0) x = powi_scale<T>((T)a.bi_rel[j], n).re * x;
        if (k2 != 0) {
          int64_t e = ((int64_t)j * k2) % P;
          T s, c;
          sincospi_((T)(-2.0 * (double)e / (double)P), &s, &c);
          x = x * mk(c, s);
        }
        v = v + x;
      }
      buf[jp] = v;
    }
    __syncthreads();
    fft_inplace<T, LOG2L, NT>(buf, a.twiddle);
    // ---- accumulate the needed outputs: k = k2 + D t, |k| <= K
    for (int o = tid; o < n_out; o += NT) {
      int t = t_lo + o;
      int idx = t & (L - 1);  // t mod L (two's complement)
      cpx<T> v = buf[idx];
      T f = fac[o];
      acc[o] = acc[o] + f * v;
      int k = k2 + D * t;
      fac[o] = f * (T)(a.ds_height * (double)k) / (T)(n + 1);
    }
    __syncthreads();
  }
  // ---- half-sample phase exp(-i pi k / P) and demodulation exp(+i pi k / sigma)
  cpx<T>* out = a.grid + (size_t)series * (2 * K + 1);
  const int64_t two_p = 2 * P;
  for (int o = tid; o < n_out; o += NT) {
    int k = k2 + D * (t_lo + o);
    // pi k (1/sigma - 1/P) = pi k (n - 1) / P, reduced exactly modulo 2 pi
    int64_t e = ((int64_t)k * (int64_t)(a.n - 1)) % two_p;
    if (e < 0) e += two_p;
    cpx<T> ph = expipi<T>((double)e / (double)P);
    out[k + K] = acc[o] * ph;
  }
}

template <class T, int LOG2L>
cudaError_t launch_l(const FftArgs<T>& a, cudaStream_t s) {
  constexpr int L = 1 << LOG2L;
  constexpr int NT = (L / 4 < 512) ? L / 4 : 512;
  const int D = a.n_sub;
  const int n_out_max = (2 * a.grid_half + 1) / D + 2;
  size_t smem = (size_t)L * sizeof(cpx<T>) + (size_t)n_out_max * (sizeof(cpx<T>) + sizeof(T)) + 16;
  cudaError_t e = cudaFuncSetAttribute(fft_taylor_kernel<T, LOG2L, NT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.series, D);
  fft_taylor_kernel<T, LOG2L, NT><<<grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

template <class T>
cudaError_t launch_fft(const FftArgs<T>& a, cudaStream_t s) {
  switch (a.log2_sub) {
    case 6: return launch_l<T, 6>(a, s);
    case 7: return launch_l<T, 7>(a, s);
    case 8: return launch_l<T, 8>(a, s);
    case 9: return launch_l<T, 9>(a, s);
    case 10: return launch_l<T, 10>(a, s);
    case 11: return launch_l<T, 11>(a, s);
    case 12: return launch_l<T, 12>(a, s);
    case 13: return launch_l<T, 13>(a, s);
    case 14:
      if constexpr (sizeof(T) == 4) return launch_l<T, 14>(a, s);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_fft<float>(const FftArgs<float>&, cudaStream_t);
template cudaError_t launch_fft<double>(const FftArgs<double>&, cudaStream_t);

}  // namespace cfft
