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
#include "es_weights.cuh"

namespace cfft {

namespace {

constexpr int kWarps = 16;
constexpr int kGroupMax = 8;

__global__ void chunk_cosine_kernel(const int* n_nodes, const int64_t* offset, int n_chunks,
                                    double* cosv) {
  for (int c = blockIdx.y; c < n_chunks; c += gridDim.y) {
    int np = n_nodes[c];
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < np; l += gridDim.x * blockDim.x)
      cosv[offset[c] + l] = cospi(((double)l + 0.5) / (double)np);
  }
}

__host__ __device__ __forceinline__ int padded(int i) { return i + (i >> 4); }

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

// one task: (group of series g0.., harmonic qi, chunk of rows)
template <class T, int TAPS>
__device__ __forceinline__ void backproject_task(const BackprojArgs<T>& a, int gidx, int qi,
                                                 int chunk, unsigned char* smem_raw) {
  constexpr int HALF = TAPS / 2 - 1;  // stencil nodes at base - HALF .. base - HALF + TAPS - 1
  const int* chunk_nodes = a.chunk_nodes;
  const int64_t* chunk_off = a.chunk_off;
  const double* cosv = a.cosv;
  const int g0 = gidx * a.group;
  const int ng = min(a.group, a.series_per_q - g0);
  const int r0 = chunk * a.rchunk;
  const int r1 = min(r0 + a.rchunk, a.n_rho);
  const int q = qi - a.q_max;
  const int np = chunk_nodes[chunk];
  const double rho_top = (r1 - 1) * a.d_rho;
  int kseg = (int)ceil(rho_top / a.d_s) + TAPS / 2 + 2;
  if (kseg > a.grid_half) kseg = a.grid_half;
  const int seg = 2 * kseg + 1;

  cpx<T>* sg = reinterpret_cast<cpx<T>*>(smem_raw);                     // [ng][seg]
  NodeCos<T>* scos = reinterpret_cast<NodeCos<T>*>(sg + (size_t)a.group * padded(seg));  // [np]
  T* scq = reinterpret_cast<T*>(scos + np);                             // [np] cos(q alpha)

  const int tid = threadIdx.x;
  // staged with one padding slot every 16 entries: lanes whose nodes sit a few grid
  // steps apart then fall into different shared-memory banks
  const int seg_p = padded(seg);
  for (int g = 0; g < ng; ++g) {
    const cpx<T>* src = a.grid + ((size_t)(g0 + g) * a.n_harm + qi) * (2 * a.grid_half + 1) +
                        (a.grid_half - kseg);
    for (int t = tid; t < seg; t += blockDim.x) sg[(size_t)g * seg_p + padded(t)] = src[t];
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
          const cpx<T>* sgp = sg + (size_t)g * seg_p;
          cpx<T> va = mk((T)0, (T)0), vb = mk((T)0, (T)0);
#pragma unroll
          for (int m = 0; m < TAPS; ++m) {
            const cpx<T> xa = sgp[padded(ia + m)];
            const cpx<T> xb = sgp[padded(ib - m)];
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

// ---------------------------------------------------------------------------
// Matrix form of the back-projection.  For harmonic q the table rows are a
// linear map of the transform grid that is the same for every MBF pair:
//   Z_q,g(rho_r) = sum_k W_q(r, k) g_q,g(s_k),
//   W_q(r, k) = 1/(2 pi N') sum_l cos(q alpha_l) exp(-i pi u_rl / sigma) L_m(u_rl),
// with u_rl = rho_r cos(alpha_l) / ds and L_m the Lagrange weight of grid
// point k = floor(u_rl) - HALF + m.  One CTA owns a tile of WR rows and one q:
// for each tile of WK grid points it scatters the stencils of the nodes that
// reach the tile into W (shared memory), then multiplies W by the grid tile of
// all MBF pairs of that q (a register-tiled complex product; 2 rows x up to
// 8 series per thread).  The weights of a node are computed once per q instead
// of once per series, and the grid values are read once per tile.
constexpr int kWR = 64;       // rows per tile
constexpr int kWK = 64;       // grid points per tile
constexpr int kWThreads = 256;
constexpr int kWSeriesMax = 64;

template <class T>
__host__ __device__ constexpr int wbp_series_pad(int series) { return (series + 1) & ~1; }

template <class T>
__host__ __device__ constexpr size_t wbp_smem_bytes(int n_nodes_max, int series) {
  return (size_t)kWK * (kWR + 2) * sizeof(cpx<T>) + (size_t)kWK * wbp_series_pad<T>(series) * sizeof(cpx<T>) +
         (size_t)n_nodes_max * (sizeof(NodeCos<T>) + sizeof(T)) + (size_t)(2 * kWR) * sizeof(int) + 64;
}

// two adjacent complex values from shared memory (16-byte aligned)
template <class T>
__device__ __forceinline__ void ld_pair(const cpx<T>* p, cpx<T>& x0, cpx<T>& x1) {
  if constexpr (sizeof(T) == 4) {
    const float4 f = *reinterpret_cast<const float4*>(p);
    x0 = mk(f.x, f.y);
    x1 = mk(f.z, f.w);
  } else {
    x0 = p[0];
    x1 = p[1];
  }
}

template <class T, int TAPS>
__device__ __forceinline__ void backproject_w_task(const BackprojArgs<T>& a, int tile, int qi,
                                                   unsigned char* smem_raw) {
  constexpr int HALF = TAPS / 2 - 1;
  constexpr int kSub = kWThreads / kWR;            // threads per row in the scatter
  const int S = a.series_per_q;
  const int S2 = wbp_series_pad<T>(S);
  const int r0 = tile * a.rchunk;                 // a.rchunk == kWR
  const int r1 = min(r0 + a.rchunk, a.n_rho);
  const int q = qi - a.q_max;
  const int np = a.chunk_nodes[tile];
  const int tid = threadIdx.x;
  // shared layout: W [WK][WR + 2] | G [WK][S2] | node cos | cos(q alpha) | row node ranges
  cpx<T>* W = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* G = W + kWK * (kWR + 2);
  NodeCos<T>* scos = reinterpret_cast<NodeCos<T>*>(G + kWK * S2);
  T* scq = reinterpret_cast<T*>(scos + np);
  int* l_lo = reinterpret_cast<int*>(scq + np);
  int* l_hi = l_lo + kWR;
  const int four_np = 4 * np;
  for (int t = tid; t < np; t += blockDim.x) {
    const double c = a.cosv[a.chunk_off[tile] + t];
    NodeCos<T> nc;
    if constexpr (sizeof(T) == 4) {
      nc.hi = (float)c;
      nc.lo = (float)(c - (double)nc.hi);
    } else {
      nc.v = c;
      nc.pad = 0.0;
    }
    scos[t] = nc;
    int e = (int)(((int64_t)q * (2 * t + 1)) % four_np);
    if (e < 0) e += four_np;
    scq[t] = cospi_((T)e / (T)(2 * np));
  }
  T den[TAPS];
#pragma unroll
  for (int m = 0; m < TAPS; ++m) {
    long long d = 1;
#pragma unroll
    for (int j = 0; j < TAPS; ++j)
      if (j != m) d *= (long long)(m - j);
    den[m] = (T)1 / (T)d;
  }
  // GEMM thread layout: a warp holds 8 row pairs x 4 series pairs, so each of its
  // shared-memory loads covers one 128-byte line (W) or a broadcast (G)
  const int lane = tid & 31, warp = tid >> 5;
  const int rp = (warp & 3) * 8 + (lane & 7);     // rows 2 rp, 2 rp + 1
  const int sp = (warp >> 2) * 4 + (lane >> 3);   // series 2 sp, 2 sp + 1 (+ 16 per pass)
  constexpr int NPASS = kWSeriesMax / 16;
  cpx<T> acc[NPASS][4];                           // [pass][row0 s0, row0 s1, row1 s0, row1 s1]
#pragma unroll
  for (int j = 0; j < NPASS; ++j)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[j][k] = mk((T)0, (T)0);
  const int npass = (S2 + 15) / 16;
  // scatter layout: kSub threads per row, nodes interleaved among them
  const int srow = tid % kWR, ssub = tid / kWR;
  const double arow = (double)(r0 + srow) * a.d_rho / a.d_s;
  const double rho_top = (r1 - 1) * a.d_rho;
  const int kmax = min(a.grid_half - 1, (int)ceil(rho_top / a.d_s) + TAPS);
  const int k_first = -kmax, n_tiles = (2 * kmax + kWK) / kWK;
  __syncthreads();
  for (int kt = 0; kt < n_tiles; ++kt) {
    const int k0 = k_first + kt * kWK;
    // ---- zero W, load the grid tile of every series of this q, find node ranges
    for (int t = tid; t < kWK * (kWR + 2); t += blockDim.x) W[t] = mk((T)0, (T)0);
    for (int t = tid; t < kWK * S2; t += blockDim.x) {
      const int g = t / kWK, kk = t - g * kWK;
      const int k = k0 + kk;
      G[kk * S2 + g] = (g < S && k >= -a.grid_half && k <= a.grid_half)
                           ? a.grid[((size_t)g * a.n_harm + qi) * (2 * a.grid_half + 1) + k + a.grid_half]
                           : mk((T)0, (T)0);
    }
    if (tid < kWR) {
      const int r = r0 + tid;
      int lo = 0, hi = -1;
      if (r < r1) {
        if (arow <= 0.0) {
          if (k0 <= TAPS - 1 - HALF && k0 + kWK - 1 >= -HALF) { lo = 0; hi = np - 1; }
        } else {
          // stencil bases b with [b - HALF, b - HALF + TAPS - 1] meeting [k0, k0 + WK)
          const double ulo = (double)(k0 + HALF - TAPS + 1), uhi = (double)(k0 + kWK + HALF);
          const double chi = fmin(1.0, uhi / arow), clo = fmax(-1.0, ulo / arow);
          if (chi >= clo) {
            const float scale = (float)np / 3.14159265f;
            lo = (int)floorf(acosf((float)chi) * scale - 0.5f) - 1;
            hi = (int)ceilf(acosf((float)clo) * scale - 0.5f) + 1;
            lo = max(lo, 0);
            hi = min(hi, np - 1);
          }
        }
      }
      l_lo[tid] = lo;
      l_hi[tid] = hi;
    }
    __syncthreads();
    // ---- scatter the node stencils that reach this tile into W (each thread one row:
    // the lanes of a warp add into 32 different rows)
    {
      const int lo = l_lo[srow], hi = l_hi[srow];
      float ahi = 0.f, alo = 0.f;
      if constexpr (sizeof(T) == 4) {
        ahi = (float)arow;
        alo = (float)(arow - (double)ahi);
      }
      for (int l = lo + ssub; l <= hi; l += kSub) {
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
          const float inv_sigma = 1.0f / (float)a.sigma;
          float ps = p * inv_sigma;
          float red = ps - 2.f * floorf(0.5f * ps);
          float sv, cv;
          sincospif(-(red + e * inv_sigma), &sv, &cv);
          ph = mk(cv, sv);
        } else {
          const double u = arow * nc.v;
          const double fl = floor(u);
          base = (int)fl;
          fr = (T)(u - fl);
          ph = expipi<T>(-u / (double)a.sigma);
        }
        const int kb = base - HALF - k0;   // tile column of tap 0
        if (kb + TAPS - 1 < 0 || kb >= kWK) continue;
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
        const cpx<T> wc = scq[l] * ph;
#pragma unroll
        for (int m = 0; m < TAPS; ++m) {
          const int kk = kb + m;
          if (kk >= 0 && kk < kWK) {
            T* dst = reinterpret_cast<T*>(&W[kk * (kWR + 2) + srow]);
            atomicAdd(dst, wc.re * w[m]);
            atomicAdd(dst + 1, wc.im * w[m]);
          }
        }
      }
    }
    __syncthreads();
    // ---- acc[rows 2rp, 2rp+1][series 2sp, 2sp+1 (+16 j)] += W[:, rows] x G[:, series]
#pragma unroll 4
    for (int kk = 0; kk < kWK; ++kk) {
      cpx<T> w0, w1;
      ld_pair(W + kk * (kWR + 2) + 2 * rp, w0, w1);
      const cpx<T>* gk = G + kk * S2 + 2 * sp;
#pragma unroll
      for (int j = 0; j < NPASS; ++j) {
        if (j < npass && 2 * sp + 16 * j < S2) {
          cpx<T> g0, g1;
          ld_pair(gk + 16 * j, g0, g1);
          cmac(acc[j][0], w0, g0);
          cmac(acc[j][1], w0, g1);
          cmac(acc[j][2], w1, g0);
          cmac(acc[j][3], w1, g1);
        }
      }
    }
    __syncthreads();
  }
  const T norm = (T)(1.0 / (2.0 * 3.14159265358979323846 * (double)np));
  const int ra = r0 + 2 * rp, rb = ra + 1;
#pragma unroll
  for (int j = 0; j < NPASS; ++j) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int g = 2 * sp + 16 * j + (k & 1);
      const int r = (k < 2) ? ra : rb;
      if (j < npass && g < S && r < r1)
        a.table[((size_t)g * a.n_harm + qi) * a.n_rho + r] = mk(acc[j][k].re * norm, acc[j][k].im * norm);
    }
  }
}

// ---- paired-harmonic, mirror-folded matrix form (FP32-mixed)
//
// Two symmetries of the alpha quadrature shrink the matrix form:
//  * cos(q alpha) is even in q, so one interpolation matrix serves q and -q
//    (32 series per task: 16 of q = +|q|, 16 of q = -|q|);
//  * the midpoint nodes are symmetric about alpha = pi/2: the node at pi - alpha
//    has u = rho cos / ds of the opposite sign, the weight (-1)^q cos(q alpha),
//    the mirrored Lagrange stencil and the conjugate demodulation phase.  For a
//    node with u >= 0 and its mirror the two contributions sum to
//      c sum_k L_k(u) [ Re(ph) G+(k) + i Im(ph) G-(k) ],
//      G+-(k) = G(k) +- (-1)^q G(-k),
//    so only the nodes with alpha <= pi/2 are visited (the middle node, when the
//    count is odd, with weight 1/2), the K range is k >= -(taps/2 - 1), and the
//    two matrices A = sum c L Re(ph), B = sum c L Im(ph) are real:
//      Z(r) = sum_k A(r, k) G+(k) + i B(r, k) G-(k).
// A CTA owns 256 rows (one thread per row): every thread adds the stencils of
// its row's nodes into its own column of (A, B) with plain read-modify-write.
// The product is register-tiled 4 rows x 8 series per thread; the lanes of a
// warp cover 8 row quads x 4 series octets, so each 16-byte shared-memory load
// is one wavefront.
constexpr int kPR = 256;           // rows per tile = threads
constexpr int kPK = 32;            // grid points per K-tile
constexpr int kPStride = kPR;      // W row stride (entries (A, B)): a row's column in one bank pair
constexpr int kPSeries = 16;       // series per sign per task
// G+- tiles as [series][kk] with a pitch of kPK + 2 entries: the fill writes
// consecutive kk (no bank conflicts) and the GEMM's 16-byte reads of the 4 series
// a warp needs at once (series so + 4 j, so = lane / 8) fall on distinct banks
constexpr int kGPitch = kPK + 2;

size_t pm_smem_bytes(int n_nodes_max) {
  const int n_half = (n_nodes_max + 1) / 2;
  return (size_t)kPK * kPStride * sizeof(cpx<float>) +
         (size_t)2 * 2 * kPSeries * kGPitch * sizeof(cpx<float>) +
         (size_t)n_half * (sizeof(NodeCos<float>) + sizeof(float)) + 64;
}

// KERN: the stencil weights, 0 Lagrange (grid of g itself), 1 ES (precorrected grid)
template <int TAPS, int KERN>
__device__ __forceinline__ void backproject_pm_task(const BackprojArgs<float>& a, int tile, int p, int chunk,
                                                    unsigned char* smem_raw) {
  constexpr int HALF = TAPS / 2 - 1;
  const int S = a.series_per_q;
  const int r0 = tile * kPR;
  const int r1 = min(r0 + kPR, a.n_rho);
  const int np = a.chunk_nodes[tile];
  const int nhalf = (np + 1) / 2;            // nodes with alpha <= pi / 2
  const int tid = threadIdx.x;
  cpx<float>* W = reinterpret_cast<cpx<float>*>(smem_raw);          // (A, B) [kk][row]
  cpx<float>* Gp = W + kPK * kPStride;                               // G+ [series][kk]
  cpx<float>* Gm = Gp + 2 * kPSeries * kGPitch;                      // G- [series][kk]
  NodeCos<float>* scos = reinterpret_cast<NodeCos<float>*>(Gm + 2 * kPSeries * kGPitch);
  float* scq = reinterpret_cast<float*>(scos + nhalf);
  const int four_np = 4 * np;
  for (int t = tid; t < nhalf; t += blockDim.x) {
    const double c = a.cosv[a.chunk_off[tile] + t];
    NodeCos<float> nc;
    nc.hi = (float)c;
    nc.lo = (float)(c - (double)nc.hi);
    scos[t] = nc;
    int e = (int)(((int64_t)p * (2 * t + 1)) % four_np);
    float cq = cospif((float)e / (float)(2 * np));
    if (2 * t + 1 == np) cq *= 0.5f;          // the middle node is its own mirror
    scq[t] = cq;
  }
  float den[TAPS];
#pragma unroll
  for (int m = 0; m < TAPS; ++m) {
    long long d = 1;
#pragma unroll
    for (int j = 0; j < TAPS; ++j)
      if (j != m) d *= (long long)(m - j);
    den[m] = 1.0f / (float)d;
  }
  // GEMM layout
  const int lane = tid & 31, warp = tid >> 5;
  const int rq = warp * 8 + (lane & 7);     // rows 4 rq .. 4 rq + 3
  const int so = lane >> 3;                 // series so + 4 j, j = 0 .. 7
  cpx<float> acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = mk(0.f, 0.f);
  // scatter: this thread's row
  const int r = r0 + tid;
  const bool row_ok = r < r1;
  const double arow = (double)r * a.d_rho / a.d_s;
  const float inv_arow = arow > 0.0 ? (float)(1.0 / arow) : 0.f;
  const float ahi = (float)arow, alo = (float)(arow - (double)ahi);
  const float inv_sigma = 1.0f / (float)a.sigma;
  const float scale = (float)np / 3.14159265f;
  const double rho_top = (r1 - 1) * a.d_rho;
  const int kmax = min(a.grid_half - 1, (int)ceil(rho_top / a.d_s) + TAPS);
  const int k_first = -HALF - 1, n_ktiles = (kmax - k_first + kPK) / kPK;
  const int qi_pos = a.q_max + p, qi_neg = a.q_max - p;
  const float par = (p & 1) ? -1.f : 1.f;   // (-1)^q, the same for q and -q
  __syncthreads();
  for (int kt = 0; kt < n_ktiles; ++kt) {
    const int k0 = k_first + kt * kPK;
    // ---- own column of (A, B) to zero, then the row's node stencils that reach this tile
#pragma unroll
    for (int kk = 0; kk < kPK; ++kk) W[kk * kPStride + tid] = mk(0.f, 0.f);
    if (row_ok) {
      int lo = 0, hi = -1;
      if (!(arow > 0.0)) {
        if (k0 <= TAPS - 1 - HALF && k0 + kPK - 1 >= -HALF) { lo = 0; hi = nhalf - 1; }
      } else {
        // stencil bases b with [b - HALF, b - HALF + TAPS - 1] meeting [k0, k0 + PK),
        // among the nodes with u >= 0
        const float chi = fminf(1.0f, (float)(k0 + kPK + HALF) * inv_arow);
        const float clo = fmaxf(0.0f, (float)(k0 + HALF - TAPS + 1) * inv_arow);
        if (chi >= clo) {
          lo = max((int)floorf(acosf(chi) * scale - 0.5f) - 1, 0);
          hi = min((int)ceilf(acosf(clo) * scale - 0.5f) + 1, nhalf - 1);
        }
      }
      cpx<float>* wcol = W + tid;
      for (int l = lo; l <= hi; ++l) {
        const NodeCos<float> nc = scos[l];
        float pr = ahi * nc.hi;
        float e = fmaf(ahi, nc.hi, -pr);
        e = fmaf(ahi, nc.lo, e);
        e = fmaf(alo, nc.hi, e);
        float fl = floorf(pr);
        float f = (pr - fl) + e;
        if (f < 0.f) { f += 1.f; fl -= 1.f; }
        if (f >= 1.f) { f -= 1.f; fl += 1.f; }
        const int kb = (int)fl - HALF - k0;   // tile column of tap 0
        if (kb + TAPS - 1 < 0 || kb >= kPK) continue;
        const float ps = pr * inv_sigma;
        const float red = ps - 2.f * floorf(0.5f * ps);
        float sv, cv;
        sincospif(-(red + e * inv_sigma), &sv, &cv);
        float w[TAPS];
        if constexpr (KERN == 1) {
          es_weights<TAPS>(f, w);
        } else {
          float pre = 1.f;
#pragma unroll
          for (int m = 0; m < TAPS; ++m) {
            w[m] = pre;
            pre *= (f - (float)(m - HALF));
          }
          float suf = 1.f;
#pragma unroll
          for (int m = TAPS - 1; m >= 0; --m) {
            w[m] *= suf * den[m];
            suf *= (f - (float)(m - HALF));
          }
        }
        const float cq = scq[l];
        const float wr = cq * cv, wi = cq * sv;   // A gets Re(ph), B gets Im(ph)
        if (kb >= 0 && kb + TAPS <= kPK) {
#pragma unroll
          for (int m = 0; m < TAPS; ++m) {
            cpx<float> v = wcol[(kb + m) * kPStride];
            v.re = fmaf(wr, w[m], v.re);
            v.im = fmaf(wi, w[m], v.im);
            wcol[(kb + m) * kPStride] = v;
          }
        } else {
#pragma unroll
          for (int m = 0; m < TAPS; ++m) {
            const int kk = kb + m;
            if (kk >= 0 && kk < kPK) {
              cpx<float> v = wcol[kk * kPStride];
              v.re = fmaf(wr, w[m], v.re);
              v.im = fmaf(wi, w[m], v.im);
              wcol[kk * kPStride] = v;
            }
          }
        }
      }
    }
    // ---- folded grid tiles G+-(k) = G(k) +- (-1)^q G(-k): columns 0..15 the series of
    // q = +p, 16..31 those of q = -p
    for (int t = tid; t < kPK * 2 * kPSeries; t += blockDim.x) {
      const int c = t / kPK, kk = t - c * kPK;
      const int k = k0 + kk;
      const int g = chunk * kPSeries + (c & (kPSeries - 1));
      const int qi = c < kPSeries ? qi_pos : qi_neg;
      cpx<float> gk = mk(0.f, 0.f), gn = mk(0.f, 0.f);
      if (g < S && (c < kPSeries || p > 0)) {
        const cpx<float>* src = a.grid + ((size_t)g * a.n_harm + qi) * (2 * a.grid_half + 1) + a.grid_half;
        if (k >= -a.grid_half && k <= a.grid_half) gk = src[k];
        if (-k >= -a.grid_half && -k <= a.grid_half) gn = src[-k];
      }
      Gp[c * kGPitch + kk] = mk(gk.re + par * gn.re, gk.im + par * gn.im);
      Gm[c * kGPitch + kk] = mk(gk.re - par * gn.re, gk.im - par * gn.im);
    }
    __syncthreads();
    // ---- acc[4 rows][8 series] += A G+ + i B G-, two grid points per step
#pragma unroll 1
    for (int kk = 0; kk < kPK; kk += 2) {
      const float4* wp0 = reinterpret_cast<const float4*>(W + kk * kPStride + 4 * rq);
      const float4* wp1 = reinterpret_cast<const float4*>(W + (kk + 1) * kPStride + 4 * rq);
      const float4 wa0 = wp0[0], wb0 = wp0[1], wa1 = wp1[0], wb1 = wp1[1];
      const float a0[4] = {wa0.x, wa0.z, wb0.x, wb0.z}, b0[4] = {wa0.y, wa0.w, wb0.y, wb0.w};
      const float a1[4] = {wa1.x, wa1.z, wb1.x, wb1.z}, b1[4] = {wa1.y, wa1.w, wb1.y, wb1.w};
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = so + 4 * j;
        // (G(kk), G(kk + 1)) of series c
        const float4 gpv = *reinterpret_cast<const float4*>(Gp + c * kGPitch + kk);
        const float4 gmv = *reinterpret_cast<const float4*>(Gm + c * kGPitch + kk);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          // (re, im) += A (Gp.re, Gp.im) + B (-Gm.im, Gm.re), at kk and kk + 1
          float re = fmaf(a0[i], gpv.x, fmaf(-b0[i], gmv.y, acc[i][j].re));
          float im = fmaf(a0[i], gpv.y, fmaf(b0[i], gmv.x, acc[i][j].im));
          acc[i][j].re = fmaf(a1[i], gpv.z, fmaf(-b1[i], gmv.w, re));
          acc[i][j].im = fmaf(a1[i], gpv.w, fmaf(b1[i], gmv.z, im));
        }
      }
    }
    __syncthreads();
  }
  const float norm = (float)(1.0 / (2.0 * 3.14159265358979323846 * (double)np));
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c = so + 4 * j;
    const int g = chunk * kPSeries + (c & (kPSeries - 1));
    if (g >= S || (c >= kPSeries && p == 0)) continue;
    const int qi = c < kPSeries ? qi_pos : qi_neg;
    cpx<float>* dst = a.table + ((size_t)g * a.n_harm + qi) * a.n_rho;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int rr = r0 + 4 * rq + i;
      if (rr < r1) dst[rr] = mk(acc[i][j].re * norm, acc[i][j].im * norm);
    }
  }
}

// tasks in a 1-D grid, larger rho tiles (more work) first
template <int TAPS, int KERN>
__global__ void __launch_bounds__(kPR, 2) backproject_pm_kernel(BackprojArgs<float> a, int n_tiles, int n_p,
                                                                int n_chunk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int per_tile = n_p * n_chunk;
  const int t = blockIdx.x;
  const int tile = n_tiles - 1 - t / per_tile;
  const int rem = t - (t / per_tile) * per_tile;
  backproject_pm_task<TAPS, KERN>(a, tile, rem / n_chunk, rem - (rem / n_chunk) * n_chunk, smem_raw);
}

// persistent form over (item, |q|, tile, series chunk) tasks
template <int TAPS, int KERN>
__global__ void __launch_bounds__(kPR, 2)
backproject_pm_batch_kernel(const BackprojArgs<float>* items, const int4* tasks, int n_tasks, int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_task;
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= n_tasks) break;
    const int4 tk = tasks[t];
    const BackprojArgs<float> a = items[tk.x];
    backproject_pm_task<TAPS, KERN>(a, tk.z, tk.y, tk.w, smem_raw);
    __syncthreads();
  }
}

template <class T, int TAPS>
__global__ void __launch_bounds__(kWThreads) backproject_w_kernel(BackprojArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  backproject_w_task<T, TAPS>(a, blockIdx.x, blockIdx.y, smem_raw);
}

// persistent form over (item, row tile, harmonic) tasks
template <class T, int TAPS>
__global__ void __launch_bounds__(kWThreads)
backproject_w_batch_kernel(const BackprojArgs<T>* items, const int4* tasks, int n_tasks, int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_task;
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= n_tasks) break;
    const int4 tk = tasks[t];
    const BackprojArgs<T> a = items[tk.x];
    backproject_w_task<T, TAPS>(a, tk.z, tk.y, smem_raw);
    __syncthreads();
  }
}

template <class T, int TAPS>
__global__ void __launch_bounds__(kWarps * 32) backproject_kernel(BackprojArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  backproject_task<T, TAPS>(a, blockIdx.x, blockIdx.y, blockIdx.z, smem_raw);
}

// persistent form over (item, group, harmonic, chunk) tasks
template <class T, int TAPS>
__global__ void __launch_bounds__(kWarps * 32)
backproject_batch_kernel(const BackprojArgs<T>* items, const int4* tasks, int n_tasks, int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_task;
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= n_tasks) break;
    const int4 tk = tasks[t];
    const int item = tk.x >> 12, gidx = tk.x & 4095;
    const BackprojArgs<T> a = items[item];
    backproject_task<T, TAPS>(a, gidx, tk.y, tk.z, smem_raw);
    __syncthreads();
  }
}

template <class T, int TAPS>
cudaError_t launch_taps(const BackprojArgs<T>& a, int n_chunks, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(backproject_kernel<T, TAPS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.series_per_q + a.group - 1) / a.group, a.n_harm, n_chunks);
  backproject_kernel<T, TAPS><<<grid, kWarps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <class T, int TAPS>
cudaError_t launch_taps_batch(const BackprojArgs<T>* items, const int4* tasks, int n_tasks,
                              int* counter, size_t smem, int n_ctas, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(backproject_batch_kernel<T, TAPS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, backproject_batch_kernel<T, TAPS>,
                                                    kWarps * 32, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  backproject_batch_kernel<T, TAPS><<<n_ctas * per_sm, kWarps * 32, smem, s>>>(items, tasks, n_tasks,
                                                                             counter);
  return cudaGetLastError();
}

}  // namespace

// shared memory bytes of one CTA for a group size, segment length and node count
template <class T>
size_t backproject_smem(int group, int max_seg, int max_nodes) {
  return (size_t)group * padded(max_seg) * sizeof(cpx<T>) +
         (size_t)max_nodes * (sizeof(NodeCos<T>) + sizeof(T)) + 64;
}

template <class T>
cudaError_t launch_backproject_impl(const BackprojArgs<T>& a0, const int* chunk_nodes,
                                    const int64_t* chunk_off, const double* cosv,
                                    const double* /*unused*/, int n_chunks, int max_nodes,
                                    int max_seg, cudaStream_t s) {
  if (a0.group > kGroupMax || a0.group < 1) return cudaErrorInvalidValue;
  BackprojArgs<T> a = a0;
  a.chunk_nodes = chunk_nodes;
  a.chunk_off = chunk_off;
  a.cosv = cosv;
  const size_t smem = backproject_smem<T>(a.group, max_seg, max_nodes);
  switch (a.taps) {
    case 4: return launch_taps<T, 4>(a, n_chunks, smem, s);
    case 6: return launch_taps<T, 6>(a, n_chunks, smem, s);
    case 8: return launch_taps<T, 8>(a, n_chunks, smem, s);
    case 10: return launch_taps<T, 10>(a, n_chunks, smem, s);
    case 12: return launch_taps<T, 12>(a, n_chunks, smem, s);
    case 16: return launch_taps<T, 16>(a, n_chunks, smem, s);
    case 20: return launch_taps<T, 20>(a, n_chunks, smem, s);
    case 24: return launch_taps<T, 24>(a, n_chunks, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

template <class T>
cudaError_t launch_backproject_batch(const BackprojArgs<T>* items, const int4* tasks, int n_tasks,
                                     int* counter, int taps, int group, int max_nodes, int max_seg,
                                     int n_ctas, cudaStream_t s) {
  if (group > kGroupMax || group < 1) return cudaErrorInvalidValue;
  const size_t smem = backproject_smem<T>(group, max_seg, max_nodes);
  switch (taps) {
    case 8: return launch_taps_batch<T, 8>(items, tasks, n_tasks, counter, smem, n_ctas, s);
    case 12: return launch_taps_batch<T, 12>(items, tasks, n_tasks, counter, smem, n_ctas, s);
    case 16: return launch_taps_batch<T, 16>(items, tasks, n_tasks, counter, smem, n_ctas, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_backproject_batch<float>(const BackprojArgs<float>*, const int4*, int,
                                                     int*, int, int, int, int, int, cudaStream_t);
template cudaError_t launch_backproject_batch<double>(const BackprojArgs<double>*, const int4*, int,
                                                      int*, int, int, int, int, int, cudaStream_t);

template <class T>
size_t backproject_w_smem(int max_nodes, int series) { return wbp_smem_bytes<T>(max_nodes, series); }
int backproject_w_rows() { return kWR; }

template <class T, int TAPS>
cudaError_t launch_w_taps(const BackprojArgs<T>& a, int n_tiles, int max_nodes, cudaStream_t s) {
  const size_t smem = wbp_smem_bytes<T>(max_nodes, a.series_per_q);
  cudaError_t e = cudaFuncSetAttribute(backproject_w_kernel<T, TAPS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(n_tiles, a.n_harm);
  backproject_w_kernel<T, TAPS><<<grid, kWThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_backproject_w(const BackprojArgs<T>& a, int n_tiles, int max_nodes, cudaStream_t s) {
  if (a.series_per_q > kWSeriesMax || a.rchunk != kWR) return cudaErrorInvalidValue;
  switch (a.taps) {
    case 8: return launch_w_taps<T, 8>(a, n_tiles, max_nodes, s);
    case 12: return launch_w_taps<T, 12>(a, n_tiles, max_nodes, s);
    case 16: return launch_w_taps<T, 16>(a, n_tiles, max_nodes, s);
    default: return cudaErrorInvalidValue;
  }
}

template <class T, int TAPS>
cudaError_t launch_w_batch_taps(const BackprojArgs<T>* items, const int4* tasks, int n_tasks,
                                int* counter, int max_nodes, int series, int n_ctas, cudaStream_t s) {
  const size_t smem = wbp_smem_bytes<T>(max_nodes, series);
  cudaError_t e = cudaFuncSetAttribute(backproject_w_batch_kernel<T, TAPS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, backproject_w_batch_kernel<T, TAPS>,
                                                    kWThreads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  backproject_w_batch_kernel<T, TAPS><<<n_ctas * per_sm, kWThreads, smem, s>>>(items, tasks, n_tasks,
                                                                              counter);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_backproject_w_batch(const BackprojArgs<T>* items, const int4* tasks, int n_tasks,
                                       int* counter, int taps, int max_nodes, int series, int n_ctas,
                                       cudaStream_t s) {
  if (series > kWSeriesMax) return cudaErrorInvalidValue;
  switch (taps) {
    case 8: return launch_w_batch_taps<T, 8>(items, tasks, n_tasks, counter, max_nodes, series, n_ctas, s);
    case 12: return launch_w_batch_taps<T, 12>(items, tasks, n_tasks, counter, max_nodes, series, n_ctas, s);
    case 16: return launch_w_batch_taps<T, 16>(items, tasks, n_tasks, counter, max_nodes, series, n_ctas, s);
    default: return cudaErrorInvalidValue;
  }
}

template size_t backproject_w_smem<float>(int, int);
template size_t backproject_w_smem<double>(int, int);
template cudaError_t launch_backproject_w<float>(const BackprojArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_backproject_w<double>(const BackprojArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_backproject_w_batch<float>(const BackprojArgs<float>*, const int4*, int, int*,
                                                       int, int, int, int, cudaStream_t);
template cudaError_t launch_backproject_w_batch<double>(const BackprojArgs<double>*, const int4*, int,
                                                        int*, int, int, int, int, cudaStream_t);

size_t backproject_pm_smem(int max_nodes) { return pm_smem_bytes(max_nodes); }
int backproject_pm_rows() { return kPR; }
int backproject_pm_series_chunk() { return kPSeries; }

template <int TAPS, int KERN>
cudaError_t launch_pm_taps(const BackprojArgs<float>& a, int n_tiles, int max_nodes, cudaStream_t s) {
  const size_t smem = pm_smem_bytes(max_nodes);
  cudaError_t e = cudaFuncSetAttribute(backproject_pm_kernel<TAPS, KERN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int n_p = a.q_max + 1;
  const int n_chunk = (a.series_per_q + kPSeries - 1) / kPSeries;
  backproject_pm_kernel<TAPS, KERN><<<n_tiles * n_p * n_chunk, kPR, smem, s>>>(a, n_tiles, n_p, n_chunk);
  return cudaGetLastError();
}

cudaError_t launch_backproject_pm(const BackprojArgs<float>& a, int n_tiles, int max_nodes, cudaStream_t s) {
  if (a.rchunk != kPR) return cudaErrorInvalidValue;
  if (a.kern == 1) {
    switch (a.taps) {
      case 6: return launch_pm_taps<6, 1>(a, n_tiles, max_nodes, s);
      case 8: return launch_pm_taps<8, 1>(a, n_tiles, max_nodes, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (a.taps) {
    case 8: return launch_pm_taps<8, 0>(a, n_tiles, max_nodes, s);
    case 12: return launch_pm_taps<12, 0>(a, n_tiles, max_nodes, s);
    case 16: return launch_pm_taps<16, 0>(a, n_tiles, max_nodes, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int TAPS, int KERN>
cudaError_t launch_pm_batch_taps(const BackprojArgs<float>* items, const int4* tasks, int n_tasks, int* counter,
                                 int max_nodes, int n_ctas, cudaStream_t s) {
  const size_t smem = pm_smem_bytes(max_nodes);
  cudaError_t e = cudaFuncSetAttribute(backproject_pm_batch_kernel<TAPS, KERN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, backproject_pm_batch_kernel<TAPS, KERN>, kPR, smem) !=
          cudaSuccess || per_sm < 1)
    per_sm = 1;
  backproject_pm_batch_kernel<TAPS, KERN><<<n_ctas * per_sm, kPR, smem, s>>>(items, tasks, n_tasks, counter);
  return cudaGetLastError();
}

cudaError_t launch_backproject_pm_batch(const BackprojArgs<float>* items, const int4* tasks, int n_tasks,
                                        int* counter, int taps, int kern, int max_nodes, int n_ctas,
                                        cudaStream_t s) {
  if (kern == 1) {
    switch (taps) {
      case 6: return launch_pm_batch_taps<6, 1>(items, tasks, n_tasks, counter, max_nodes, n_ctas, s);
      case 8: return launch_pm_batch_taps<8, 1>(items, tasks, n_tasks, counter, max_nodes, n_ctas, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (taps) {
    case 8: return launch_pm_batch_taps<8, 0>(items, tasks, n_tasks, counter, max_nodes, n_ctas, s);
    case 12: return launch_pm_batch_taps<12, 0>(items, tasks, n_tasks, counter, max_nodes, n_ctas, s);
    case 16: return launch_pm_batch_taps<16, 0>(items, tasks, n_tasks, counter, max_nodes, n_ctas, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_chunk_cosines(const int* n_nodes, const int64_t* offset, int n_chunks,
                                 int max_nodes, double* cosv, cudaStream_t s) {
  dim3 grid((max_nodes + 255) / 256, n_chunks < 65535 ? n_chunks : 65535);
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
