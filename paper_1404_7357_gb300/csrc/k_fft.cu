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
#include "dft_small.cuh"

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

// ---- large-radix Stockham passes (lengths 2^10 .. 2^14)
//
// One pass of radix R (R = 2, 4, 8, 16) at span p: for each butterfly i < L/R with
// k = i mod p the inputs x[i + r L/R] (r < R) are multiplied by W_{R p}^{r k} and
// transformed by an R-point DFT in registers; output s goes to
// x'[(i - k) R + k + s p].  A radix-16 DFT is two radix-4 stages with the internal
// twiddles W_16^{r0 s0}.  The shared buffer is padded by one entry every 16
// (index e -> e + e/16), which makes the strided writes of the first passes
// conflict-free.  The twiddles of a butterfly come from the two-level tables
// (W^{k stride} and W^{4 k stride}) and at most two products.
__device__ __forceinline__ int pidx(int e) { return e + (e >> 4); }

template <class T, int R>
__device__ __forceinline__ void dft_r(cpx<T>* v) {
  if constexpr (R == 2) {
    const cpx<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  } else if constexpr (R == 4) {
    dft4(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    dft8(v);
  } else {
    static_assert(R == 16, "radix");
    // r = 4 r1 + r0: radix-4 over r1, twiddle W_16^{r0 s0}, radix-4 over r0
    cpx<T> a[4][4];
#pragma unroll
    for (int r0 = 0; r0 < 4; ++r0) {
#pragma unroll
      for (int r1 = 0; r1 < 4; ++r1) a[r0][r1] = v[4 * r1 + r0];
      dft4(a[r0][0], a[r0][1], a[r0][2], a[r0][3]);
    }
    const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;
    const T h = (T)0.70710678118654752440;
    const cpx<T> w1 = mk(c1, -s1), w2 = mk(h, -h), w3 = mk(s1, -c1);
    const cpx<T> w6 = mk(-h, -h), w9 = mk(-c1, s1);
    a[1][1] = a[1][1] * w1;
    a[1][2] = a[1][2] * w2;
    a[1][3] = a[1][3] * w3;
    a[2][1] = a[2][1] * w2;
    a[2][2] = mk(a[2][2].im, -a[2][2].re);   // * W_16^4 = -i
    a[2][3] = a[2][3] * w6;
    a[3][1] = a[3][1] * w3;
    a[3][2] = a[3][2] * w6;
    a[3][3] = a[3][3] * w9;
#pragma unroll
    for (int s0 = 0; s0 < 4; ++s0) {
      dft4(a[0][s0], a[1][s0], a[2][s0], a[3][s0]);
      v[s0] = a[0][s0];
      v[s0 + 4] = a[1][s0];
      v[s0 + 8] = a[2][s0];
      v[s0 + 12] = a[3][s0];
    }
  }
}

// the span P of a pass is a compile-time constant, so the padded indices of a
// butterfly's inputs and outputs are one base plus constant offsets
template <class T, int R, int LOG2L, int NT, int P>
__device__ __forceinline__ void stockham_pass(cpx<T>* buf, const cpx<T>* thi, const cpx<T>* tlo) {
  constexpr int L = 1 << LOG2L;
  constexpr int NB = L / R;
  constexpr int BPT = NB / NT;
  static_assert(BPT >= 1 && NB % NT == 0, "butterflies per thread");
  static_assert(NB % 16 == 0, "input groups start on a padding boundary");
  constexpr int p = P;
  const int tid = threadIdx.x;
  constexpr int stride = L / (R * P);
  cpx<T> v[BPT][R];
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int i = tid + NT * b;
    const int pi = pidx(i);
#pragma unroll
    for (int r = 0; r < R; ++r) v[b][r] = buf[pi + r * (NB + NB / 16)];
  }
  __syncthreads();
  if constexpr (BPT > 1 && R >= 4 && P > 1 && NT % P == 0) {
    // every butterfly of this thread has the same k = tid mod P: its twiddles are formed
    // once and applied to all of them as they are formed
    const int k = tid & (p - 1);
    if (k != 0) {
      const int e = k * stride;
      const cpx<T> t1 = tw2(thi, tlo, e), t2 = t1 * t1, t3 = t2 * t1;
#pragma unroll
      for (int b = 0; b < BPT; ++b) {
        v[b][1] = v[b][1] * t1;
        v[b][2] = v[b][2] * t2;
        v[b][3] = v[b][3] * t3;
      }
      if constexpr (R >= 8) {
        cpx<T> q = tw2(thi, tlo, 4 * e);
#pragma unroll
        for (int g = 1; g < R / 4; ++g) {
          const cpx<T> q1 = q * t1, q2 = q * t2, q3 = q * t3;
#pragma unroll
          for (int b = 0; b < BPT; ++b) {
            v[b][4 * g] = v[b][4 * g] * q;
            v[b][4 * g + 1] = v[b][4 * g + 1] * q1;
            v[b][4 * g + 2] = v[b][4 * g + 2] * q2;
            v[b][4 * g + 3] = v[b][4 * g + 3] * q3;
          }
          if (g + 1 < R / 4) q = tw2(thi, tlo, 4 * (g + 1) * e);
        }
      }
    }
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
      const int i = tid + NT * b;
      dft_r<T, R>(v[b]);
      const int j = (i - k) * R + k;
      if constexpr (P % 16 == 0) {
        const int pj = pidx(j);
        constexpr int step = P + P / 16;
#pragma unroll
        for (int s = 0; s < R; ++s) buf[pj + s * step] = v[b][s];
      } else {
#pragma unroll
        for (int s = 0; s < R; ++s) buf[pidx(j + s * p)] = v[b][s];
      }
    }
    __syncthreads();
    return;
  }
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int i = tid + NT * b;
    const int k = i & (p - 1);
    if (p > 1 && k != 0) {
      const int e = k * stride;
      const cpx<T> t1 = tw2(thi, tlo, e);
      if constexpr (R == 2) {
        v[b][1] = v[b][1] * t1;
      } else {
        const cpx<T> t2 = t1 * t1, t3 = t2 * t1;
        v[b][1] = v[b][1] * t1;
        v[b][2] = v[b][2] * t2;
        v[b][3] = v[b][3] * t3;
        if constexpr (R >= 8) {
          const cpx<T> t4 = tw2(thi, tlo, 4 * e);
          cpx<T> q = t4;
#pragma unroll
          for (int g = 1; g < R / 4; ++g) {
            v[b][4 * g] = v[b][4 * g] * q;
            v[b][4 * g + 1] = v[b][4 * g + 1] * (q * t1);
            v[b][4 * g + 2] = v[b][4 * g + 2] * (q * t2);
            v[b][4 * g + 3] = v[b][4 * g + 3] * (q * t3);
            if (g + 1 < R / 4) q = tw2(thi, tlo, 4 * (g + 1) * e);
          }
        }
      }
    }
    dft_r<T, R>(v[b]);
    const int j = (i - k) * R + k;
    if constexpr (P == 1 || P % 16 == 0) {
      // pidx(j + s P) = pidx(j) + s (P + P / 16) (P = 1: j = i R and s < R <= 16)
      const int pj = pidx(j);
      constexpr int step = P == 1 ? 1 : P + P / 16;
#pragma unroll
      for (int s = 0; s < R; ++s) buf[pj + s * step] = v[b][s];
    } else {
#pragma unroll
      for (int s = 0; s < R; ++s) buf[pidx(j + s * p)] = v[b][s];
    }
  }
  __syncthreads();
}

template <class T, int LOG2L, int NT, int P, int REMAIN>
__device__ __forceinline__ void radix16_passes(cpx<T>* buf, const cpx<T>* thi, const cpx<T>* tlo) {
  if constexpr (REMAIN > 0) {
    stockham_pass<T, 16, LOG2L, NT, P>(buf, thi, tlo);
    radix16_passes<T, LOG2L, NT, P * 16, REMAIN - 1>(buf, thi, tlo);
  }
}

// W_{R P}^{r k} twiddles of one butterfly (k = butterfly index mod P, stride = L / (R P))
template <class T, int R>
__device__ __forceinline__ void twiddle_inputs(cpx<T>* v, int e, const cpx<T>* thi, const cpx<T>* tlo) {
  const cpx<T> t1 = tw2(thi, tlo, e);
  if constexpr (R == 2) {
    v[1] = v[1] * t1;
  } else {
    const cpx<T> t2 = t1 * t1, t3 = t2 * t1;
    v[1] = v[1] * t1;
    v[2] = v[2] * t2;
    v[3] = v[3] * t3;
    if constexpr (R >= 8) {
      cpx<T> q = tw2(thi, tlo, 4 * e);
#pragma unroll
      for (int g = 1; g < R / 4; ++g) {
        v[4 * g] = v[4 * g] * q;
        v[4 * g + 1] = v[4 * g + 1] * (q * t1);
        v[4 * g + 2] = v[4 * g + 2] * (q * t2);
        v[4 * g + 3] = v[4 * g + 3] * (q * t3);
        if (g + 1 < R / 4) q = tw2(thi, tlo, 4 * (g + 1) * e);
      }
    }
  }
}

// first pass (span 1, radix R) with its inputs produced by `input(jp)` instead of
// being read back from the buffer: the fold of the transform's input feeds the
// butterflies directly
template <class T, int R, int LOG2L, int NT, class In>
__device__ __forceinline__ void first_pass_fused(cpx<T>* buf, In input) {
  constexpr int L = 1 << LOG2L;
  constexpr int NB = L / R;
  constexpr int BPT = NB / NT;
  static_assert(BPT >= 1 && NB % NT == 0, "butterflies per thread");
  const int tid = threadIdx.x;
#pragma unroll 1
  for (int b = 0; b < BPT; ++b) {
    const int i = tid + NT * b;
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = input(i + r * NB);
    dft_r<T, R>(v);
    const int pj = pidx(i * R);   // span 1: outputs i R + s, one base plus s
#pragma unroll
    for (int s2 = 0; s2 < R; ++s2) buf[pj + s2] = v[s2];
  }
  __syncthreads();
}

// last pass (radix 16, span L/16): each butterfly's outputs t = i + s L/16 that the
// task needs go straight into the Taylor accumulation `use(t, value)`
template <class T, int LOG2L, int NT, class Use>
__device__ __forceinline__ void last_pass_fused(const cpx<T>* buf, const cpx<T>* thi, const cpx<T>* tlo,
                                                Use use) {
  constexpr int L = 1 << LOG2L;
  constexpr int P = L / 16;
  constexpr int NB = P;
  constexpr int BPT = NB / NT;
  static_assert(BPT >= 1 && NB % NT == 0 && NB % 16 == 0, "butterflies per thread");
  const int tid = threadIdx.x;
#pragma unroll 1
  for (int b = 0; b < BPT; ++b) {
    const int i = tid + NT * b;   // = k (i < P), stride 1
    const int pi = pidx(i);
    cpx<T> v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = buf[pi + r * (NB + NB / 16)];
    if (i != 0) twiddle_inputs<T, 16>(v, i, thi, tlo);
    dft_r<T, 16>(v);
#pragma unroll
    for (int s2 = 0; s2 < 16; ++s2) use(i + s2 * P, v[s2]);
  }
  __syncthreads();
}

// the last pass when only the outputs s = 0 and s = 15 of each butterfly are needed
// (t_hi < L/16 and t_lo > -L/16: the needed t = i and t = i - L/16 (mod L)).  With the
// butterfly's inputs v_r and twiddles W_L^(r i), both outputs are polynomials in one
// root of unity, evaluated by Horner's rule:
//   X_0  = sum_r v_r z^r,   X_15 = sum_r v_r (z W16^-1)^r,   z = W_L^i
// (W16^(15 r) = W16^(-r)), so no per-input twiddle is formed
template <class T, int LOG2L, int NT, class Use>
__device__ __forceinline__ void last_pass_pruned(const cpx<T>* buf, const cpx<T>* thi, const cpx<T>* tlo,
                                                 int t_lo, int t_hi, Use use) {
  constexpr int L = 1 << LOG2L;
  constexpr int P = L / 16;
  constexpr int NB = P;
  constexpr int BPT = NB / NT;
  static_assert(BPT >= 1 && NB % NT == 0 && NB % 16 == 0, "butterflies per thread");
  const int tid = threadIdx.x;
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;
#pragma unroll 1
  for (int b = 0; b < BPT; ++b) {
    const int i = tid + NT * b;
    const bool need0 = i <= t_hi, need15 = i >= P + t_lo;
    if (need0 || need15) {
      const int pi = pidx(i);
      cpx<T> v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = buf[pi + r * (NB + NB / 16)];
      const cpx<T> z = tw2(thi, tlo, i);
      const cpx<T> w = z * mk(c1, s1);   // z W16^-1
      cpx<T> x0 = v[15], x15 = v[15];
#pragma unroll
      for (int r = 14; r >= 0; --r) {
        x0 = x0 * z + v[r];
        x15 = x15 * w + v[r];
      }
      if (need0) use(i, x0);
      if (need15) use(i + 15 * P, x15);
    }
  }
  __syncthreads();
}

// radix-16 passes with spans P, 16 P, ... leaving the last (span L/16) to the caller
template <class T, int LOG2L, int NT, int P>
__device__ __forceinline__ void middle_passes(cpx<T>* buf, const cpx<T>* thi, const cpx<T>* tlo) {
  if constexpr (P < (1 << LOG2L) / 16) {
    stockham_pass<T, 16, LOG2L, NT, P>(buf, thi, tlo);
    middle_passes<T, LOG2L, NT, P * 16>(buf, thi, tlo);
  }
}

// in-place (Stockham, autosorting) length-2^LOG2L FFT over the padded buffer:
// one pass of radix 2^(LOG2L mod 4) when that is not 1, then radix-16 passes
template <class T, int LOG2L, int NT>
__device__ __forceinline__ void fft16_inplace(cpx<T>* buf, const cpx<T>* thi, const cpx<T>* tlo) {
  constexpr int REM = LOG2L & 3;
  if constexpr (REM == 1) stockham_pass<T, 2, LOG2L, NT, 1>(buf, thi, tlo);
  if constexpr (REM == 2) stockham_pass<T, 4, LOG2L, NT, 1>(buf, thi, tlo);
  if constexpr (REM == 3) stockham_pass<T, 8, LOG2L, NT, 1>(buf, thi, tlo);
  radix16_passes<T, LOG2L, NT, (1 << REM), LOG2L / 4>(buf, thi, tlo);
}

__device__ __forceinline__ int floor_div(int a, int b) {  // b > 0
  int q = a / b;
  return (a % b != 0 && a < 0) ? q - 1 : q;
}


// threads of a transform task and shared-buffer padding, by length
template <int LOG2L>
struct FftShape {
  static constexpr int L = 1 << LOG2L;
  static constexpr bool R16 = LOG2L >= 10;                       // large-radix passes
  static constexpr int NT = R16 ? (L / 16 < 512 ? L / 16 : 512) : (L / 4 < 512 ? L / 4 : 512);
  static constexpr int BUF = R16 ? L + L / 16 : L;               // padded buffer entries
};

// Chebyshev polynomial T_m(z) by its three-term recurrence (|z| <= 1: stable)
template <class T>
__device__ __forceinline__ T cheb_t(int m, T z) {
  if (m == 0) return (T)1;
  T t0 = (T)1, t1 = z;
  for (int i = 1; i < m; ++i) {
    const T t2 = (T)2 * z * t1 - t0;
    t0 = t1;
    t1 = t2;
  }
  return t1;
}

// a / b for a small positive integer b: in float32 by the reciprocal-based quotient
// (two units in the last place), in float64 exactly
template <class T>
__device__ __forceinline__ T div_int(T a, int b) {
  if constexpr (sizeof(T) == 4) return __fdividef(a, (float)b);
  else return a / (double)b;
}

// I_m(a) / ((a/2)^m / m!) = sum_i q^i m! / (i! (i+m)!), q = (a/2)^2: the power series of
// the modified Bessel function I_m without its leading factor
template <class T>
__device__ __forceinline__ T bessel_i_tail(int m, T q) {
  T t = (T)1, sum = (T)1;
  const T eps = sizeof(T) == 4 ? (T)1e-8 : (T)1e-17;
  for (int i = 1; i < 48; ++i) {
    t = div_int<T>(t * q, i * (i + m));
    sum += t;
    if (t <= eps * sum) break;
  }
  return sum;
}

// one (series, k2) task: all terms of the contour-factor expansion of one residue class of
// the outputs.  The real exponential exp(beta_I s) = exp(H s b), b = beta_I / H in [0, 1]
// on the active prefix of the contour (0 beyond it), is expanded in one of two series:
//  * series 0, the Taylor series of Eq. 22: term 0 = all nodes with weight 1, term n >= 1
//    = the active nodes with weight b^n, output coefficient (H s)^n / n!;
//  * series 1, the Chebyshev series of the same factor about the middle of b's range:
//    exp(H s b) = exp(a) exp(a z), a = H s / 2, z = 2 b - 1 in [-1, 1], and
//    exp(a z) = I_0(a) + 2 sum_m I_m(a) T_m(z); term 0 = the nodes beyond the active
//    prefix (b = 0: weight 1, exactly), term m + 1 = the active nodes with weight T_m(z),
//    output coefficient exp(a) (2 - [m = 0]) I_m(a).  Its coefficients fall like
//    (a / 2)^m / m! instead of (2 a)^n / n!, so fewer transforms reach a tolerance.
// use_zt: the pre-twiddled active inputs times the current weight are kept in shared
// memory (two arrays for the Chebyshev recurrence) and advanced by the weight recurrence
// instead of being re-read
template <class T, int LOG2L, int NT>
__device__ __forceinline__ void fft_taylor_task(const FftArgs<T>& a, int series, int k2,
                                                unsigned char* smem_raw, int use_zt) {
  constexpr int L = 1 << LOG2L;
  constexpr bool R16 = FftShape<LOG2L>::R16;
  constexpr int BUF = FftShape<LOG2L>::BUF;
  auto bidx = [](int e) { return R16 ? pidx(e) : e; };
  const int D = a.n_sub;
  const int K = a.grid_half;
  const int t_lo = -floor_div(K + k2, D);     // ceil((-K - k2) / D)
  const int t_hi = floor_div(K - k2, D);
  const int n_out = t_hi - t_lo + 1;
  const int n = a.n;
  const int na = a.n_active;
  const bool cheb = a.expansion == 1;
  const int n_terms = a.taylor + (cheb ? 2 : 1);
  const int n_hi = (n + 127) >> 7;
  const int tid = threadIdx.x;
  const int64_t P = a.fft_len;
  // shared layout: FFT buffer | pre-twiddle lo, hi | FFT twiddle hi, lo | acc | coefficient |
  // stored active inputs (one array, two for the Chebyshev recurrence)
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* plo = buf + BUF;          // exp(-2 pi i r k2 / P), r < 128
  cpx<T>* phi = plo + 128;          // exp(-2 pi i 128 m k2 / P), m < n_hi
  cpx<T>* thi = phi + n_hi;         // exp(-2 pi i 128 m / L), m < L / 128
  cpx<T>* tlo = thi + 128;          // exp(-2 pi i r / L), r < 128
  cpx<T>* acc = tlo + 128;
  T* fac = reinterpret_cast<T*>(acc + n_out);
  cpx<T>* zt = reinterpret_cast<cpx<T>*>((reinterpret_cast<uintptr_t>(fac + n_out) + 15) & ~(uintptr_t)15);
  cpx<T>* zt2 = zt + na;
  const cpx<T>* y = a.y + (size_t)series * n;
  auto brel = [&](int j) -> T {
    if constexpr (sizeof(T) == 4) return a.bi_rel_f[j];
    else return a.bi_rel[j];
  };

  // ---- per-task tables (exact integer argument reduction; the sine and cosine in the
  // precision of T: the angles are (integer < P) / P).  In float32 the quotient is formed
  // in float32 too (P < 2^24 is exact there): float64 arithmetic runs at 1/64 rate
  auto angle = [&](int64_t num) -> T {   // -2 num / P, num in [0, P)
    if constexpr (sizeof(T) == 4) return -2.0f * (float)num / (float)P;
    else return -2.0 * (double)num / (double)P;
  };
  for (int r = tid; r < 128; r += NT) {
    T sv, cv;
    int64_t rk = (int64_t)r * k2;     // < 128 D <= 2 P
    if (rk >= P) rk %= P;
    sincospi_(angle(rk), &sv, &cv);
    plo[r] = mk(cv, sv);
    sincospi_((T)-2 * (T)r / (T)L, &sv, &cv);
    tlo[r] = mk(cv, sv);
    if (r < ((L >> 7) > 0 ? (L >> 7) : 1)) {
      sincospi_((T)-2 * (T)(128 * r) / (T)L, &sv, &cv);
      thi[r] = mk(cv, sv);
    }
  }
  for (int m = tid; m < n_hi; m += NT) {
    T sv, cv;
    sincospi_(angle(((int64_t)m * 128 * k2) % P), &sv, &cv);
    phi[m] = mk(cv, sv);
  }
  // fac[o]: the running factor of output o's coefficient, (H s)^n / n! for the Taylor
  // series, exp(a) (a/2)^m / m! for the Chebyshev series (a = H s / 2)
  const T dsh = (T)a.ds_height;
  for (int o = tid; o < n_out; o += NT) {
    acc[o] = mk((T)0, (T)0);
    fac[o] = cheb ? exp((T)0.5 * dsh * (T)(k2 + D * (t_lo + o))) : (T)1;
  }
  __syncthreads();
  for (int nt = 0; nt < n_terms; ++nt) {
    // input nodes [j_lo, lim) of this term
    const int j_lo = (cheb && nt == 0) ? na : 0;
    const int lim = nt == 0 ? n : na;
    // coefficient of output o in this term; advances its running factor to the next term
    // (each needed output is used once per term, by one thread)
    const T inv_next = (T)1 / (T)(cheb ? (nt > 0 ? nt : 1) : nt + 1);
    auto coef = [&](int o) -> T {
      const T x = dsh * (T)(k2 + D * (t_lo + o));   // H s_k
      const T f = fac[o];
      if (!cheb) {
        fac[o] = f * x * inv_next;
        return f;
      }
      if (nt == 0) return (T)1;
      const int m = nt - 1;
      const T h = (T)0.25 * x;   // a / 2
      fac[o] = f * h * inv_next;
      return (m == 0 ? (T)1 : (T)2) * f * bessel_i_tail<T>(m, h * h);
    };
    const bool stored = use_zt && (cheb ? nt > 1 : nt > 0);
    // fold + pre-twiddle W_P^{j k2} + the term's weight, for the residue jp of the nodes
    auto fold = [&](int jp) -> cpx<T> {
      cpx<T> v = mk((T)0, (T)0);
      if (stored) {
        for (int j = jp; j < lim; j += L) {
          const cpx<T> c = zt[j];
          v = v + c;
          if (!cheb) {
            zt[j] = brel(j) * c;   // next Taylor term
          } else {
            const T z2 = (T)4 * brel(j) - (T)2;   // 2 z
            const cpx<T> pv = zt2[j];
            zt[j] = z2 * c - pv;   // next Chebyshev term
            zt2[j] = c;
          }
        }
        return v;
      }
      int j = jp;
      if (j < j_lo) j += ((j_lo - j + L - 1) / L) * L;   // first node of the class in range
      for (; j < lim; j += L) {
        cpx<T> x = y[j];
        if (a.prec) x = x * a.prec[j];
        if (k2 != 0) x = x * (phi[j >> 7] * plo[j & 127]);
        if (!cheb) {
          T b = (T)1;
          if (nt > 0 || use_zt) b = brel(j);
          if (nt > 0) x = powi_scale<T>(b, nt).re * x;
          else if (use_zt && j < na) zt[j] = b * x;   // first Taylor term for nt = 1
        } else if (nt >= 1) {
          const T z = (T)2 * brel(j) - (T)1;
          if (nt == 1) {
            if (use_zt) {
              zt[j] = z * x;   // T_1 x, the next term's input
              zt2[j] = x;      // T_0 x
            }
          } else {
            x = cheb_t<T>(nt - 1, z) * x;
          }
        }
        v = v + x;
      }
      return v;
    };
    if constexpr (R16) {
      constexpr int REM = LOG2L & 3;
      constexpr int R0 = REM == 0 ? 16 : (1 << REM);
      first_pass_fused<T, R0, LOG2L, NT>(buf, fold);
      middle_passes<T, LOG2L, NT, R0>(buf, thi, tlo);
      // the needed outputs k = k2 + D t, |k| <= K, accumulate the term's coefficient times it
      auto use = [&](int t, cpx<T> v) {
        const int tt = t <= t_hi ? t : t - L;
        if (tt >= t_lo && tt <= t_hi) {
          const int o = tt - t_lo;
          acc[o] = acc[o] + coef(o) * v;
        }
      };
      if (t_hi < L / 16 && t_lo > -(L / 16)) last_pass_pruned<T, LOG2L, NT>(buf, thi, tlo, t_lo, t_hi, use);
      else last_pass_fused<T, LOG2L, NT>(buf, thi, tlo, use);
      continue;
    }
    for (int jp = tid; jp < L; jp += NT) buf[bidx(jp)] = fold(jp);
    __syncthreads();
    fft_inplace<T, LOG2L, NT>(buf, thi, tlo);
    // ---- accumulate the needed outputs: k = k2 + D t, |k| <= K
    for (int o = tid; o < n_out; o += NT) {
      int t = t_lo + o;
      int idx = t & (L - 1);  // t mod L (two's complement)
      acc[o] = acc[o] + coef(o) * buf[bidx(idx)];
    }
    __syncthreads();
  }
  // ---- half-sample phase exp(-i pi k / P) and demodulation exp(+i pi k / sigma)
  cpx<T>* out = a.grid + (size_t)series * (2 * K + 1);
  const int64_t two_p = 2 * P;
  for (int o = tid; o < n_out; o += NT) {
    int k = k2 + D * (t_lo + o);
    cpx<T> ph;
    if constexpr (sizeof(T) == 4) {
      // exp(i pi k / sigma) exp(-i pi k / P): sigma is a power of two, so k mod 2 sigma is
      // exact in integers, and |k| <= K < P / 2 keeps the second angle below pi / 2
      float s1, c1, s2, c2;
      sincospif((float)(k & (2 * a.sigma - 1)) / (float)a.sigma, &s1, &c1);
      sincospif(-(float)k / (float)P, &s2, &c2);
      ph = mk(c1 * c2 - s1 * s2, s1 * c2 + c1 * s2);
    } else {
      // pi k (1/sigma - 1/P) = pi k (n - 1) / P, reduced exactly modulo 2 pi
      int64_t e = ((int64_t)k * (int64_t)(n - 1)) % two_p;
      if (e < 0) e += two_p;
      ph = expipi<T>((double)e / (double)P);
    }
    out[k + K] = acc[o] * ph;
  }
}

// at most 128 registers per thread whatever the block size
template <int NT>
constexpr int fft_min_blocks() { return NT >= 512 ? 1 : 512 / NT; }

template <class T, int LOG2L, int NT>
__global__ void __launch_bounds__(NT, fft_min_blocks<NT>()) fft_taylor_kernel(FftArgs<T> a, int use_zt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fft_taylor_task<T, LOG2L, NT>(a, blockIdx.x, blockIdx.y, smem_raw, use_zt);
}

// persistent form: CTAs pull (item, series, k2) tasks from a counter until none is left
template <class T, int LOG2L, int NT>
__global__ void __launch_bounds__(NT, fft_min_blocks<NT>()) fft_taylor_batch_kernel(const FftArgs<T>* items,
                                                              const int4* tasks, int n_tasks,
                                                              int* counter, int use_zt) {
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
    fft_taylor_task<T, LOG2L, NT>(a, tk.y, tk.z, smem_raw, use_zt);
    __syncthreads();
  }
}

// shared bytes of a transform task with zt_arrays stores of the active inputs (0: none)
template <class T, int LOG2L>
size_t fft_task_smem(int n_active, int n_out_max, int hi_max, int zt_arrays) {
  return (size_t)FftShape<LOG2L>::BUF * sizeof(cpx<T>) + fft_task_extra<T>(n_active, n_out_max, hi_max) +
         (zt_arrays > 0 ? (size_t)zt_arrays * n_active * sizeof(cpx<T>) + 16 : 0);
}

// the opt-in maximum of dynamic shared memory per block (227 KB) less the static words
constexpr size_t kFftSmemCap = 227 * 1024 - 64;

template <class T, int LOG2L>
cudaError_t launch_l(const FftArgs<T>& a, cudaStream_t s) {
  constexpr int NT = FftShape<LOG2L>::NT;
  const int D = a.n_sub;
  const int n_out_max = (2 * a.grid_half + 1) / D + 2;
  const int hi = (a.n + 127) / 128;
  // the stored active inputs pay when at least two terms after the first read them
  const int arrays = a.expansion == 1 ? 2 : 1;
  const bool zt = a.taylor > 0 && fft_task_smem<T, LOG2L>(a.n_active, n_out_max, hi, arrays) <= kFftSmemCap;
  const size_t smem = fft_task_smem<T, LOG2L>(a.n_active, n_out_max, hi, zt ? arrays : 0);
  cudaError_t e = cudaFuncSetAttribute(fft_taylor_kernel<T, LOG2L, NT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.series, D);
  fft_taylor_kernel<T, LOG2L, NT><<<grid, NT, smem, s>>>(a, zt ? 1 : 0);
  return cudaGetLastError();
}

template <class T, int LOG2L>
cudaError_t launch_l_batch(const FftArgs<T>* items, const int4* tasks, int n_tasks, int* counter,
                           int max_n_out, int max_active, int max_hi, int zt_arrays, int n_ctas,
                           cudaStream_t s) {
  constexpr int NT = FftShape<LOG2L>::NT;
  const bool zt = fft_task_smem<T, LOG2L>(max_active, max_n_out + 2, max_hi, zt_arrays) <= kFftSmemCap;
  const size_t smem = fft_task_smem<T, LOG2L>(max_active, max_n_out + 2, max_hi, zt ? zt_arrays : 0);
  cudaError_t e = cudaFuncSetAttribute(fft_taylor_batch_kernel<T, LOG2L, NT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fft_taylor_batch_kernel<T, LOG2L, NT>,
                                                    NT, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  fft_taylor_batch_kernel<T, LOG2L, NT><<<n_ctas * per_sm, NT, smem, s>>>(items, tasks, n_tasks,
                                                                        counter, zt ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace

template <class T>
cudaError_t launch_fft_batch(const FftArgs<T>* items, const int4* tasks, int n_tasks, int* counter,
                             int log2_sub, int max_n_out, int max_active, int max_hi, int zt_arrays,
                             int n_ctas, cudaStream_t s) {
  switch (log2_sub) {
    case 10: return launch_l_batch<T, 10>(items, tasks, n_tasks, counter, max_n_out, max_active, max_hi, zt_arrays, n_ctas, s);
    case 11: return launch_l_batch<T, 11>(items, tasks, n_tasks, counter, max_n_out, max_active, max_hi, zt_arrays, n_ctas, s);
    case 12: return launch_l_batch<T, 12>(items, tasks, n_tasks, counter, max_n_out, max_active, max_hi, zt_arrays, n_ctas, s);
    case 13: return launch_l_batch<T, 13>(items, tasks, n_tasks, counter, max_n_out, max_active, max_hi, zt_arrays, n_ctas, s);
    case 14:
      if constexpr (sizeof(T) == 4)
        return launch_l_batch<T, 14>(items, tasks, n_tasks, counter, max_n_out, max_active, max_hi, zt_arrays, n_ctas, s);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_fft_batch<float>(const FftArgs<float>*, const int4*, int, int*, int, int,
                                             int, int, int, int, cudaStream_t);
template cudaError_t launch_fft_batch<double>(const FftArgs<double>*, const int4*, int, int*, int,
                                              int, int, int, int, int, cudaStream_t);

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
