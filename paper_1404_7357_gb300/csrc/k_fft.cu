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

// Twiddles exp(-2 pi i t / L) as hi[t >> 7] * lo[t & 127] from two small shared tables
// (the full table would evict the L1 that shared memory leaves free).
template <class T>
__device__ __forceinline__ cpx<T> tw2(const cpx<T>* thi, const cpx<T>* tlo, int t) {
  return thi[t >> 7] * tlo[t & 127];
}

template <class T, int LOG2L, int NT>
__device__ __forceinline__ void fft_inplace(cpx<T>* buf, const cpx<T>* thi, const cpx<T>* tlo) {
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
      cpx<T> x1 = v[4 * b + 1];
      cpx<T> x2 = v[4 * b + 2];
      cpx<T> x3 = v[4 * b + 3];
      if (k != 0) {
        x1 = x1 * tw2(thi, tlo, k * stride);
        x2 = x2 * tw2(thi, tlo, 2 * k * stride);
        x3 = x3 * tw2(thi, tlo, 3 * k * stride);
      }
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


// one (series, k2) task: all Taylor terms of one residue class of the outputs
template <class T, int LOG2L, int NT>
__device__ __forceinline__ void fft_taylor_task(const FftArgs<T>& a, int series, int k2,
                                                unsigned char* smem_raw) {
  constexpr int L = 1 << LOG2L;
  const int D = a.n_sub;
  const int K = a.grid_half;
  const int t_lo = -floor_div(K + k2, D);     // ceil((-K - k2) / D)
  const int t_hi = floor_div(K - k2, D);
  const int n_out = t_hi - t_lo + 1;
  const int n = a.n;
  const int n_hi = (n + 127) >> 7;
  const int tid = threadIdx.x;
  const int64_t P = a.fft_len;
  // shared layout: FFT buffer | pre-twiddle lo, hi | FFT twiddle hi, lo | acc | fac | sk
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* plo = buf + L;            // exp(-2 pi i r k2 / P), r < 128
  cpx<T>* phi = plo + 128;          // exp(-2 pi i 128 m k2 / P), m < n_hi
  cpx<T>* thi = phi + n_hi;         // exp(-2 pi i 128 m / L), m < L / 128
  cpx<T>* tlo = thi + 128;          // exp(-2 pi i r / L), r < 128
  cpx<T>* acc = tlo + 128;
  T* fac = reinterpret_cast<T*>(acc + n_out);
  T* skv = fac + n_out;
  const cpx<T>* y = a.y + (size_t)series * n;

  // ---- per-task tables (float64 argument reduction, once)
  for (int r = tid; r < 128; r += NT) {
    double sv, cv;
    sincospi(-2.0 * (double)(((int64_t)r * k2) % P) / (double)P, &sv, &cv);
    plo[r] = mk((T)cv, (T)sv);
    sincospi(-2.0 * (double)r / (double)L, &sv, &cv);
    tlo[r] = mk((T)cv, (T)sv);
    if (r < ((L >> 7) > 0 ? (L >> 7) : 1)) {
      sincospi(-2.0 * (double)(128 * r) / (double)L, &sv, &cv);
      thi[r] = mk((T)cv, (T)sv);
    }
  }
  for (int m = tid; m < n_hi; m += NT) {
    double sv, cv;
    sincospi(-2.0 * (double)(((int64_t)m * 128 * k2) % P) / (double)P, &sv, &cv);
    phi[m] = mk((T)cv, (T)sv);
  }
  for (int o = tid; o < n_out; o += NT) {
    acc[o] = mk((T)0, (T)0);
    fac[o] = (T)1;
    skv[o] = (T)(a.ds_height * (double)(k2 + D * (t_lo + o)));
  }
  __syncthreads();
  for (int nt = 0; nt <= a.taylor; ++nt) {
    const int lim = nt == 0 ? n : a.n_active;
    // ---- fold + pre-twiddle W_P^{j k2} + Taylor weight (beta_I/H)^n
    for (int jp = tid; jp < L; jp += NT) {
      cpx<T> v = mk((T)0, (T)0);
      for (int j = jp; j < lim; j += L) {
        cpx<T> x = y[j];
        if (nt > 0) {
          T b;
          if constexpr (sizeof(T) == 4) b = a.bi_rel_f[j];
          else b = a.bi_rel[j];
          x = powi_scale<T>(b, nt).re * x;
        }
        if (k2 != 0) x = x * (phi[j >> 7] * plo[j & 127]);
        v = v + x;
      }
      buf[jp] = v;
    }
    __syncthreads();
    fft_inplace<T, LOG2L, NT>(buf, thi, tlo);
    // ---- accumulate the needed outputs: k = k2 + D t, |k| <= K
    const T inv = (T)1 / (T)(nt + 1);
    for (int o = tid; o < n_out; o += NT) {
      int t = t_lo + o;
      int idx = t & (L - 1);  // t mod L (two's complement)
      cpx<T> v = buf[idx];
      T f = fac[o];
      acc[o] = acc[o] + f * v;
      fac[o] = f * skv[o] * inv;
    }
    __syncthreads();
  }
  // ---- half-sample phase exp(-i pi k / P) and demodulation exp(+i pi k / sigma)
  cpx<T>* out = a.grid + (size_t)series * (2 * K + 1);
  const int64_t two_p = 2 * P;
  for (int o = tid; o < n_out; o += NT) {
    int k = k2 + D * (t_lo + o);
    // pi k (1/sigma - 1/P) = pi k (n - 1) / P, reduced exactly modulo 2 pi
    int64_t e = ((int64_t)k * (int64_t)(n - 1)) % two_p;
    if (e < 0) e += two_p;
    cpx<T> ph = expipi<T>((double)e / (double)P);
    out[k + K] = acc[o] * ph;
  }
}

template <class T, int LOG2L, int NT>
__global__ void __launch_bounds__(NT) fft_taylor_kernel(FftArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fft_taylor_task<T, LOG2L, NT>(a, blockIdx.x, blockIdx.y, smem_raw);
}

// persistent form: CTAs pull (item, series, k2) tasks from a counter until none is left
template <class T, int LOG2L, int NT>
__global__ void __launch_bounds__(NT) fft_taylor_batch_kernel(const FftArgs<T>* items,
                                                              const int4* tasks, int n_tasks,
                                                              int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_task;
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= n_tasks) break;
    const int4 tk = tasks[t];
    const FftArgs<T> a = items[tk.x];
    fft_taylor_task<T, LOG2L, NT>(a, tk.y, tk.z, smem_raw);
    __syncthreads();
  }
}

template <class T, int LOG2L>
cudaError_t launch_l(const FftArgs<T>& a, cudaStream_t s) {
  constexpr int L = 1 << LOG2L;
  constexpr int NT = (L / 4 < 512) ? L / 4 : 512;
  const int D = a.n_sub;
  const int n_out_max = (2 * a.grid_half + 1) / D + 2;
  size_t smem = (size_t)L * sizeof(cpx<T>) +
                fft_task_extra<T>(a.n_active, n_out_max, (a.n + 127) / 128);
  cudaError_t e = cudaFuncSetAttribute(fft_taylor_kernel<T, LOG2L, NT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.series, D);
  fft_taylor_kernel<T, LOG2L, NT><<<grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <class T, int LOG2L>
cudaError_t launch_l_batch(const FftArgs<T>* items, const int4* tasks, int n_tasks, int* counter,
                           int max_n_out, int max_active, int max_hi, int n_ctas, cudaStream_t s) {
  constexpr int L = 1 << LOG2L;
  constexpr int NT = (L / 4 < 512) ? L / 4 : 512;
  size_t smem = (size_t)L * sizeof(cpx<T>) + fft_task_extra<T>(max_active, max_n_out + 2, max_hi);
  cudaError_t e = cudaFuncSetAttribute(fft_taylor_batch_kernel<T, LOG2L, NT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fft_taylor_batch_kernel<T, LOG2L, NT>,
                                                    NT, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  fft_taylor_batch_kernel<T, LOG2L, NT><<<n_ctas * per_sm, NT, smem, s>>>(items, tasks, n_tasks,
                                                                        counter);
  return cudaGetLastError();
}

}  // namespace

template <class T>
cudaError_t launch_fft_batch(const FftArgs<T>* items, const int4* tasks, int n_tasks, int* counter,
                             int log2_sub, int max_n_out, int max_active, int max_hi, int n_ctas,
                             cudaStream_t s) {
  switch (log2_sub) {
    case 10: return launch_l_batch<T, 10>(items, tasks, n_tasks, counter, max_n_out, max_active, max_hi, n_ctas, s);
    case 11: return launch_l_batch<T, 11>(items, tasks, n_tasks, counter, max_n_out, max_active, max_hi, n_ctas, s);
    case 12: return launch_l_batch<T, 12>(items, tasks, n_tasks, counter, max_n_out, max_active, max_hi, n_ctas, s);
    case 13: return launch_l_batch<T, 13>(items, tasks, n_tasks, counter, max_n_out, max_active, max_hi, n_ctas, s);
    case 14:
      if constexpr (sizeof(T) == 4)
        return launch_l_batch<T, 14>(items, tasks, n_tasks, counter, max_n_out, max_active, max_hi, n_ctas, s);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_fft_batch<float>(const FftArgs<float>*, const int4*, int, int*, int, int,
                                             int, int, int, cudaStream_t);
template cudaError_t launch_fft_batch<double>(const FftArgs<double>*, const int4*, int, int*, int,
                                              int, int, int, int, cudaStream_t);

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
