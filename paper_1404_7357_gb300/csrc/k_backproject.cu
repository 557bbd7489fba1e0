// Back-projection of the beta transform onto the uniform rho grid of the table.
//
// The harmonic form of Eq. 9 integrates exp(i q alpha) g_q(rho cos alpha) over
// the angle (the one-dimensional FFT in beta gives g_q on a uniform s grid):
//   Z_q(rho) = 1/(4 pi^2) int_0^{2 pi} exp(i q alpha) g_q(rho cos alpha) d alpha
//            = 1/(2 pi^2) int_0^{pi} cos(q alpha) g_q(rho cos alpha) d alpha
// evaluated with the midpoint rule on N' nodes (spectrally accurate: the
// integrand is smooth, even and 2 pi-periodic) and with g_q interpolated
// between grid samples by a TAPS-point Lagrange stencil.  The grid holds
// g_q(s) exp(i beta_max s / 2) (spectrum centred on zero), so the value at
// s = u ds is re-modulated by exp(-i pi u / sigma) after interpolation.  The
// paper instead refines its 2-D table by Whittaker-Shannon zero padding and
// interpolates at second order (Section III-B-3); here the zero padding is
// the FFT's sigma and the stencil width is chosen for the precision target.
//
// Node pairs alpha and pi - alpha share their stencil: s -> -s mirrors the
// fractional position (the node set is symmetric about 1/2, so the weights
// are reversed), conjugates the re-modulation phase and multiplies
// cos(q alpha) by (-1)^q.  N' grows with the angular content of the
// integrand, |beta| rho: the nodes of a chunk of rows are fixed by its
// largest rho, and their cosines (as a float pair hi + lo in float32 mode)
// and cos(q alpha) are staged in shared memory once per CTA.  Node positions
// u = (rho/ds) cos(alpha) reach thousands of grid steps, so in float32 they
// are formed as float pairs (products by fma) to keep the fractional position
// and the re-modulation phase exact to float32 rounding.
// Layout: one CTA = (group of series sharing the harmonic q, q, chunk of rows);
// every warp owns rows; lanes split the node pairs; the node weights are
// computed once per node pair and applied to every series of the group.
#include "cfft_common.cuh"

namespace cfft {

namespace {

constexpr int kWarps = 8;
constexpr int kGroupMax = 8;

__global__ void chunk_cosine_kernel(const int* n_nodes, const int64_t* offset, int n_chunks,
                                    double* cosv) {
  int c = blockIdx.y;
  if (c >= n_chunks) return;
  int np = n_nodes[c];
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < np; l += gridDim.x * blockDim.x)
    cosv[offset[c] + l] = cospi(((double)l + 0.5) / (double)np);
}

template <class T>
struct NodeCos;
template <>
struct NodeCos<float> {
  float hi, lo;
};
template <>
struct NodeCos<double> {
  double v, pad;
};

template <class T, int TAPS>
__global__ void __launch_bounds__(kWarps * 32)
backproject_kernel(BackprojArgs<T> a, const int* chunk_nodes, const int64_t* chunk_off,
                   const double* cosv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int HALF = TAPS / 2 - 1;  // stencil nodes at base - HALF .. base - HALF + TAPS - 1
  const int g0 = blockIdx.x * a.group;
  const int ng = min(a.group, a.series_per_q - g0);
  const int qi = blockIdx.y;
  const int chunk = blockIdx.z;
  const int r0 = chunk * a.rchunk;
  const int r1 = min(r0 + a.rchunk, a.n_rho);
  const int q = qi - a.q_max;
  const int np = chunk_nodes[chunk];
  const double rho_top = (r1 - 1) * a.d_rho;
  int kseg = (int)ceil(rho_top / a.d_s) + TAPS / 2 + 2;
  if (kseg > a.grid_half) kseg = a.grid_half;
  const int seg = 2 * kseg + 1;

  cpx<T>* sg = reinterpret_cast<cpx<T>*>(smem_raw);                     // [ng][seg]
  NodeCos<T>* scos = reinterpret_cast<NodeCos<T>*>(sg + (size_t)a.group * seg);  // [np]
  T* scq = reinterpret_cast<T*>(scos + np);                             // [np] cos(q alpha)

  const int tid = threadIdx.x;
  for (int g = 0; g < ng; ++g) {
    const cpx<T>* src = a.grid + ((size_t)(g0 + g) * a.n_harm + qi) * (2 * a.grid_half + 1) +
                        (a.grid_half - kseg);
    for (int t = tid; t < seg; t += blockDim.x) sg[(size_t)g * seg + t] = src[t];
  }
  const int four_np = 4 * np;
  for (int t = tid; t < np; t += blockDim.x) {
    const double c = cosv[chunk_off[chunk] + t];
    NodeCos<T> nc;
    if constexpr (sizeof(T) == 4) {
      nc.hi = (float)c;
      nc.lo = (float)(c - (double)nc.hi);
    } else {
      nc.v = c;
      nc.pad = 0.0;
    }
    scos[t] = nc;
    // cos(q alpha_t), alpha_t = (t + 1/2) pi / np, argument reduced exactly
    int e = (int)(((int64_t)q * (2 * t + 1)) % four_np);
    if (e < 0) e += four_np;
    scq[t] = cospi_((T)e / (T)(2 * np));
  }
  __syncthreads();

  const int warp = tid >> 5, lane = tid & 31;
  const T norm = (T)(1.0 / (2.0 * 3.14159265358979323846 * (double)np));
  const T qsign = (q & 1) ? (T)-1 : (T)1;
  const int n_pairs = (np + 1) / 2;  // node l pairs with np - 1 - l (the middle one alone)
  // Lagrange denominators 1 / prod_{j != m} (m - j) for equally spaced nodes
  T den[TAPS];
#pragma unroll
  for (int m = 0; m < TAPS; ++m) {
    long long d = 1;
#pragma unroll
    for (int j = 0; j < TAPS; ++j)
      if (j != m) d *= (long long)(m - j);
    den[m] = (T)1 / (T)d;
  }
  for (int r = r0 + warp; r < r1; r += kWarps) {
    const double arow = (double)r * a.d_rho / a.d_s;  // rho_r / ds
    float ahi = 0.f, alo = 0.f;
    if constexpr (sizeof(T) == 4) {
      ahi = (float)arow;
      alo = (float)(arow - (double)ahi);
    }
    cpx<T> acc[kGroupMax];
#pragma unroll
    for (int g = 0; g < kGroupMax; ++g) acc[g] = mk((T)0, (T)0);
    for (int l = lane; l < n_pairs; l += 32) {
      const NodeCos<T> nc = scos[l];
      int base;
      T fr;
      cpx<T> ph;
      if constexpr (sizeof(T) == 4) {
        float p = ahi * nc.hi;
        float e = fmaf(ahi, nc.hi, -p);
        e = fmaf(ahi, nc.lo, e);
        e = fmaf(alo, nc.hi, e);
        float fl = floorf(p);
        float f = (p - fl) + e;
        if (f < 0.f) { f += 1.f; fl -= 1.f; }
        if (f >= 1.f) { f -= 1.f; fl += 1.f; }
        base = (int)fl;
        fr = f;
        const float inv_sigma = 1.0f / (float)a.sigma;  // power of two: exact
        float ps = p * inv_sigma;
        float red = ps - 2.f * floorf(0.5f * ps);      // exact
        float s, c;
        sincospif(-(red + e * inv_sigma), &s, &c);
        ph = mk(c, s);
      } else {
        const double u = arow * nc.v;
        const double fl = floor(u);
        base = (int)fl;
        fr = (T)(u - fl);
        ph = expipi<T>(-u / (double)a.sigma);
      }
      // Lagrange weights at x = fr for nodes x_m = m - HALF (prefix/suffix products)
      T w[TAPS];
      {
        T pre = (T)1;
#pragma unroll
        for (int m = 0; m < TAPS; ++m) {
          w[m] = pre;
          pre *= (fr - (T)(m - HALF));
        }
        T suf = (T)1;
#pragma unroll
        for (int m = TAPS - 1; m >= 0; --m) {
          w[m] *= suf * den[m];
          suf *= (fr - (T)(m - HALF));
        }
      }
      const bool paired = (np - 1 - l) != l;
      const T cq = scq[l];
      const cpx<T> wa = cq * ph;                                   // node l
      const cpx<T> wb = paired ? (qsign * cq) * conj(ph) : mk((T)0, (T)0);  // node np-1-l
      const int ia = kseg + base - HALF;          // tap m of node l at ia + m
      const int ib = kseg - (base - HALF);        // tap m of the mirror node at ib - m
#pragma unroll
      for (int g = 0; g < kGroupMax; ++g) {
        if (g < ng) {
          const cpx<T>* sgp = sg + (size_t)g * seg;
          cpx<T> va = mk((T)0, (T)0), vb = mk((T)0, (T)0);
#pragma unroll
          for (int m = 0; m < TAPS; ++m) {
            const cpx<T> xa = sgp[ia + m];
            const cpx<T> xb = sgp[ib - m];
            va.re = fma(w[m], xa.re, va.re);
            va.im = fma(w[m], xa.im, va.im);
            vb.re = fma(w[m], xb.re, vb.re);
            vb.im = fma(w[m], xb.im, vb.im);
          }
          cmac(acc[g], wa, va);
          cmac(acc[g], wb, vb);
        }
      }
    }
#pragma unroll
    for (int g = 0; g < kGroupMax; ++g) {
      if (g < ng) {
        T re = acc[g].re, im = acc[g].im;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          re += __shfl_xor_sync(0xffffffffu, re, off);
          im += __shfl_xor_sync(0xffffffffu, im, off);
        }
        if (lane == 0)
          a.table[((size_t)(g0 + g) * a.n_harm + qi) * a.n_rho + r] = mk(re * norm, im * norm);
      }
    }
  }
}

template <class T, int TAPS>
cudaError_t launch_taps(const BackprojArgs<T>& a, const int* chunk_nodes, const int64_t* chunk_off,
                        const double* cosv, int n_chunks, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(backproject_kernel<T, TAPS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.series_per_q + a.group - 1) / a.group, a.n_harm, n_chunks);
  backproject_kernel<T, TAPS><<<grid, kWarps * 32, smem, s>>>(a, chunk_nodes, chunk_off, cosv);
  return cudaGetLastError();
}

}  // namespace

// shared memory bytes of one CTA for a group size, segment length and node count
template <class T>
size_t backproject_smem(int group, int max_seg, int max_nodes) {
  return (size_t)group * max_seg * sizeof(cpx<T>) + (size_t)max_nodes * (sizeof(NodeCos<T>) + sizeof(T)) + 64;
}

template <class T>
cudaError_t launch_backproject_impl(const BackprojArgs<T>& a, const int* chunk_nodes,
                                    const int64_t* chunk_off, const double* cosv,
                                    const double* /*unused*/, int n_chunks, int max_nodes,
                                    int max_seg, cudaStream_t s) {
  if (a.group > kGroupMax || a.group < 1) return cudaErrorInvalidValue;
  const size_t smem = backproject_smem<T>(a.group, max_seg, max_nodes);
  switch (a.taps) {
    case 4: return launch_taps<T, 4>(a, chunk_nodes, chunk_off, cosv, n_chunks, smem, s);
    case 6: return launch_taps<T, 6>(a, chunk_nodes, chunk_off, cosv, n_chunks, smem, s);
    case 8: return launch_taps<T, 8>(a, chunk_nodes, chunk_off, cosv, n_chunks, smem, s);
    case 10: return launch_taps<T, 10>(a, chunk_nodes, chunk_off, cosv, n_chunks, smem, s);
    case 12: return launch_taps<T, 12>(a, chunk_nodes, chunk_off, cosv, n_chunks, smem, s);
    case 16: return launch_taps<T, 16>(a, chunk_nodes, chunk_off, cosv, n_chunks, smem, s);
    case 20: return launch_taps<T, 20>(a, chunk_nodes, chunk_off, cosv, n_chunks, smem, s);
    case 24: return launch_taps<T, 24>(a, chunk_nodes, chunk_off, cosv, n_chunks, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_chunk_cosines(const int* n_nodes, const int64_t* offset, int n_chunks,
                                 int max_nodes, double* cosv, cudaStream_t s) {
  dim3 grid((max_nodes + 255) / 256, n_chunks);
  chunk_cosine_kernel<<<grid, 256, 0, s>>>(n_nodes, offset, n_chunks, cosv);
  return cudaGetLastError();
}

template size_t backproject_smem<float>(int, int, int);
template size_t backproject_smem<double>(int, int, int);
template cudaError_t launch_backproject_impl<float>(const BackprojArgs<float>&, const int*,
                                                    const int64_t*, const double*,
                                                    const double*, int, int, int, cudaStream_t);
template cudaError_t launch_backproject_impl<double>(const BackprojArgs<double>&, const int*,
                                                     const int64_t*, const double*,
                                                     const double*, int, int, int,
                                                     cudaStream_t);

}  // namespace cfft
