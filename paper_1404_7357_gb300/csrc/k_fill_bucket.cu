// Bucketed reduced-matrix fill (Section III-B-3, Eq. 3 per block, Eq. 9 per
// entry): the same interpolation as the per-row fill, organised so that the
// table is read from shared memory with warp-wide broadcasts.
//
// Every element pair (m, n) needs, for each harmonic q and MBF pair (a, b),
// the taps-point Lagrange interpolation of Z^{cls}_ab,q at rho_mn; its stencil
// starts at table row i0(rho_mn).  The pairs of a group of test elements
// ("row block") are counting-sorted by (rotation class, i0) in global memory.
// A CTA then owns one (row block, class, window of `win` consecutive i0): it
// copies the table rows the window's stencils touch, for all harmonics and
// MBF pairs, into shared memory as [q][row][ab], and each thread takes one
// pair after another.  Consecutive pairs of the sorted list share i0, so the
// 32 lanes of a warp read the same shared-memory words (one broadcast
// wavefront per load) and each load brings the M consecutive b-entries of a
// row: per (q, a) and tap one or two 16-byte loads feed 2M FMAs.
//
// For M = 4 with 8 taps in FP32 the same buckets feed the tensor cores instead
// (fill_tc_kernel, adjoint_tc_kernel below): one CTA per stencil cell, whose
// pairs all use the same 8 table rows, so the harmonic sum of all of them is
// one product with that slice of the table; the adjoint of the fill (gradient
// with respect to the positions and, through derivative tables, the substrate)
// runs over the same buckets in either form.
//
// Geometry in the FP32-mixed mode runs in float-float arithmetic (positions
// split into a float head and tail; rho from a corrected float square root)
// instead of float64, whose throughput is a small fraction of float32 on this
// part; rho and the stencil coordinate keep about 44 significant bits, the
// same decisions as float64 except at exact cell-boundary ties, where either
// stencil is a valid one.
#include <algorithm>
#include <type_traits>

#include "cfft_common.cuh"
#include "spectra_tc.cuh"
#include "tc_sm100.cuh"

namespace cfft {

namespace {

constexpr int kBThreads = 256;

struct BucketArgs {
  int m0;           // first test element of this wave
  int rows;         // test elements in this wave
  int br;           // test elements per row block
  int nb_bits;      // bits of n in a pair code (code = m_local << nb_bits | n)
  int n_ck;         // rotation classes (1 or 4)
  int n_cells;      // stencil starts i0 in [-half, n_rho - taps]
  int win;          // stencil starts per window
  int vec_out;      // output rows 16-byte aligned: vector stores
  float ih, il;     // 1 / d_rho as float head + tail
  const float4* ps; // positions as (x head, x tail, y head, y tail)
  unsigned* cursor; // [n_keys] counts, then scatter cursors
  unsigned* off;    // [n_keys + 1] exclusive offsets
  unsigned* list;   // sorted pair codes
  unsigned* seg;    // [<= 1024] segment sums / offsets of the key scan
};

// renormalised float-float difference (a_hi + a_lo) - (b_hi + b_lo)
__device__ __forceinline__ void df_sub(float ah, float al, float bh, float bl, float& h, float& l) {
  const float s = __fsub_rn(ah, bh);
  const float bb = __fsub_rn(s, ah);
  float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(-bh, bb));
  e = __fadd_rn(e, __fsub_rn(al, bl));
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}

template <class T>
struct BGeom {
  int i0;       // first stencil row (negative: parity rows)
  T x;          // stencil coordinate of rho, u - i0
  T ex, ey;     // exp(i phi)
  T rho;        // the pair distance (for the adjoint's d phi / d Delta)
  bool bad;     // rho beyond the table
};

// stencil of pair (m, n), FP32-mixed: float-float geometry from the split positions
template <int TAPS>
__device__ __forceinline__ BGeom<float> bucket_geom_ps(const FillArgs<float, float>& a, const BucketArgs& b,
                                                       float4 pm, float4 pn) {
  constexpr int HALF = TAPS / 2 - 1;
  float dxh, dxl, dyh, dyl;
  df_sub(pm.x, pm.y, pn.x, pn.y, dxh, dxl);
  df_sub(pm.z, pm.w, pn.z, pn.w, dyh, dyl);
  // rho^2 as float-float
  const float px = __fmul_rn(dxh, dxh), py = __fmul_rn(dyh, dyh);
  const float ex = __fadd_rn(fmaf(dxh, dxh, -px), __fmul_rn(2.f * dxh, dxl));
  const float ey = __fadd_rn(fmaf(dyh, dyh, -py), __fmul_rn(2.f * dyh, dyl));
  const float s = __fadd_rn(px, py);
  const float bb = __fsub_rn(s, px);
  float e = __fadd_rn(__fsub_rn(px, __fsub_rn(s, bb)), __fsub_rn(py, bb));
  e = __fadd_rn(e, __fadd_rn(ex, ey));
  const float r2h = __fadd_rn(s, e), r2l = __fsub_rn(e, __fsub_rn(r2h, s));
  // rho = r + rl with r the rounded square root and rl its first correction
  const float r = sqrtf(r2h);
  const float rl = r > 0.f ? __fmul_rn(__fadd_rn(fmaf(-r, r, r2h), r2l), __fdiv_rn(0.5f, r)) : 0.f;
  // u = rho / d_rho
  const float p = __fmul_rn(r, b.ih);
  const float pe = __fadd_rn(fmaf(r, b.ih, -p), __fadd_rn(__fmul_rn(r, b.il), __fmul_rn(rl, b.ih)));
  float fl = floorf(p);
  float f = __fadd_rn(__fsub_rn(p, fl), pe);
  if (f < 0.f) { f = __fadd_rn(f, 1.f); fl = __fsub_rn(fl, 1.f); }
  if (f >= 1.f) { f = __fsub_rn(f, 1.f); fl = __fadd_rn(fl, 1.f); }
  BGeom<float> g;
  const float top = (float)(a.n_rho - 1);
  g.bad = fl > top || (fl == top && f > 1e-6f) || !(r == r);
  const int fi = (int)fl;
  int i0 = fi - HALF;
  if (i0 + TAPS > a.n_rho) i0 = a.n_rho - TAPS;
  g.i0 = i0;
  g.x = (float)(fi - i0) + f;
  g.rho = __fadd_rn(r, rl);
  if (r > 0.f) {
    g.ex = __fdiv_rn(dxh, r);
    g.ey = __fdiv_rn(dyh, r);
  } else {
    g.ex = 1.f;
    g.ey = 0.f;
  }
  return g;
}

template <class T, int TAPS>
__device__ __forceinline__ typename std::enable_if<sizeof(T) == 4, BGeom<T>>::type
bucket_geom(const FillArgs<T, T>& a, const BucketArgs& b, int m, int n) {
  return bucket_geom_ps<TAPS>(a, b, b.ps[m], b.ps[n]);
}

// stencil of pair (m, n), FP64 mode: float64 geometry
template <class T, int TAPS>
__device__ __forceinline__ typename std::enable_if<sizeof(T) == 8, BGeom<T>>::type
bucket_geom(const FillArgs<T, T>& a, const BucketArgs&, int m, int n) {
  constexpr int HALF = TAPS / 2 - 1;
  // rounded operations only (no contraction), so every kernel takes the same decisions
  const double dx = __dsub_rn(a.pos[2 * m], a.pos[2 * n]);
  const double dy = __dsub_rn(a.pos[2 * m + 1], a.pos[2 * n + 1]);
  const double rho = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
  const double u = __dmul_rn(rho, a.inv_d_rho);
  BGeom<T> g;
  g.bad = !(rho <= a.rho_max * (1.0 + 1e-12));
  const double fl = floor(u);
  int i0 = (int)fl - HALF;
  if (i0 + TAPS > a.n_rho) i0 = a.n_rho - TAPS;
  g.i0 = i0;
  g.x = __dsub_rn(u, (double)i0);
  g.rho = rho;
  g.ex = rho > 0.0 ? dx / rho : 1.0;
  g.ey = rho > 0.0 ? dy / rho : 0.0;
  return g;
}

__device__ __forceinline__ int bucket_class(const int* rot, int n_ck, int m, int n) {
  return (n_ck == 1 || rot == nullptr) ? 0 : 2 * (rot[m] != 0) + (rot[n] != 0);
}

__global__ void split_positions_kernel(const double* pos, int n_el, float4* ps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_el) return;
  const double x = pos[2 * i], y = pos[2 * i + 1];
  const float xh = (float)x, yh = (float)y;
  ps[i] = make_float4(xh, (float)(x - (double)xh), yh, (float)(y - (double)yh));
}

// pass 1 (count) and pass 2 (scatter) of the counting sort of this wave's pairs
template <class T, int TAPS, bool SCATTER>
__global__ void __launch_bounds__(kBThreads) bucket_sort_kernel(FillArgs<T, T> a, BucketArgs b) {
  constexpr int HALF = TAPS / 2 - 1;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.n_el) return;
  for (int ml = blockIdx.y; ml < b.rows; ml += gridDim.y) {
    const int m = b.m0 + ml;
    const BGeom<T> g = bucket_geom<T, TAPS>(a, b, m, n);
    if (g.bad) {
      if (!SCATTER) {
        atomicOr(a.err, 1);
        if (a.z == nullptr) continue;   // the adjoint: no matrix
        const int M = a.n_mbf;
        for (int ia = 0; ia < M; ++ia)
          for (int ib = 0; ib < M; ++ib)
            a.z[(size_t)(m * M + ia) * a.ld + (size_t)n * M + ib] = mk((T)0, (T)0);
      }
      continue;
    }
    const int blk = ml / b.br;
    const int cls = bucket_class(a.rot, b.n_ck, m, n);
    const size_t key = ((size_t)blk * b.n_ck + cls) * b.n_cells + (g.i0 + HALF);
    if (!SCATTER) {
      atomicAdd(&b.cursor[key], 1u);
    } else {
      const unsigned slot = atomicAdd(&b.cursor[key], 1u);
      b.list[slot] = ((unsigned)(ml - blk * b.br) << b.nb_bits) | (unsigned)n;
    }
  }
}

// exclusive scan of the key counts, off[k] = sum_{j<k} count[j], off[n] = total, with the
// counts replaced by the scatter cursors (= off): three passes over segments of
// kScanSeg keys (segment sums; a scan of the sums; the segments rescanned in tiles of
// 1024 with warp-shuffle scans), every load and store coalesced
constexpr int kScanSeg = 16 * 1024;

__device__ __forceinline__ unsigned block_incl_scan(unsigned v, unsigned* warp_tot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) warp_tot[w] = v;
  __syncthreads();
  if (w == 0) {
    unsigned t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    warp_tot[lane] = t;   // inclusive over warps
  }
  __syncthreads();
  return v + (w > 0 ? warp_tot[w - 1] : 0u);
}

__global__ void __launch_bounds__(1024) scan_segment_sums(const unsigned* cnt, size_t n_keys, unsigned* seg_sum) {
  __shared__ unsigned red[32];
  const size_t base = (size_t)blockIdx.x * kScanSeg;
  unsigned v = 0;
  for (int i = threadIdx.x; i < kScanSeg; i += blockDim.x)
    if (base + i < n_keys) v += cnt[base + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) seg_sum[blockIdx.x] = t;
  }
}

// exclusive scan of the segment sums (at most 1024 segments) and the grand total
__global__ void __launch_bounds__(1024) scan_segment_offsets(unsigned* seg_sum, int n_seg, unsigned* off,
                                                             size_t n_keys) {
  __shared__ unsigned wt[32];
  const unsigned v = threadIdx.x < n_seg ? seg_sum[threadIdx.x] : 0u;
  const unsigned incl = block_incl_scan(v, wt);
  if (threadIdx.x < n_seg) seg_sum[threadIdx.x] = incl - v;
  if (threadIdx.x == blockDim.x - 1) off[n_keys] = incl;
}

__global__ void __launch_bounds__(1024) scan_apply(unsigned* cnt, unsigned* off, size_t n_keys,
                                                   const unsigned* seg_off) {
  __shared__ unsigned wt[32];
  __shared__ unsigned s_run;
  const size_t base = (size_t)blockIdx.x * kScanSeg;
  if (threadIdx.x == 0) s_run = seg_off[blockIdx.x];
  __syncthreads();
  for (int t0 = 0; t0 < kScanSeg; t0 += blockDim.x) {
    const size_t k = base + t0 + threadIdx.x;
    const unsigned c = k < n_keys ? cnt[k] : 0u;
    const unsigned incl = block_incl_scan(c, wt);
    const unsigned run = s_run;
    if (k < n_keys) {
      off[k] = run + incl - c;
      cnt[k] = run + incl - c;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_run = run + incl;
    __syncthreads();
  }
}

// M consecutive complex entries from shared memory, in 16-byte loads when they allow
template <class T, int M>
__device__ __forceinline__ void load_row(const cpx<T>* p, cpx<T>* v) {
  if constexpr (sizeof(T) == 4 && (M % 2) == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int i = 0; i < M / 2; ++i) {
      const float4 f = q[i];
      v[2 * i] = mk(f.x, f.y);
      v[2 * i + 1] = mk(f.z, f.w);
    }
  } else if constexpr (sizeof(T) == 8) {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const double2 d = q[i];
      v[i] = mk(d.x, d.y);
    }
  } else {
#pragma unroll
    for (int i = 0; i < M; ++i) v[i] = p[i];
  }
}

// M consecutive complex entries to global memory; vec: the destination is 16-byte aligned
// M consecutive complex entries from global memory; vec: the source is 16-byte aligned
template <class T, int M>
__device__ __forceinline__ void load_grad_row(const cpx<T>* src, cpx<T>* v, bool vec) {
  if constexpr (sizeof(T) == 4 && (M % 2) == 0) {
    if (vec) {
      const float4* q = reinterpret_cast<const float4*>(src);
#pragma unroll
      for (int i = 0; i < M / 2; ++i) {
        const float4 f = __ldg(q + i);
        v[2 * i] = mk(f.x, f.y);
        v[2 * i + 1] = mk(f.z, f.w);
      }
      return;
    }
  }
#pragma unroll
  for (int i = 0; i < M; ++i) v[i] = src[i];
}

template <class T, int M>
__device__ __forceinline__ void store_row(cpx<T>* dst, const cpx<T>* v, bool vec) {
  if constexpr (sizeof(T) == 4 && (M % 2) == 0) {
    if (vec) {
      float4* q = reinterpret_cast<float4*>(dst);
#pragma unroll
      for (int i = 0; i < M / 2; ++i) q[i] = make_float4(v[2 * i].re, v[2 * i].im, v[2 * i + 1].re, v[2 * i + 1].im);
      return;
    }
#pragma unroll
    for (int i = 0; i < M; ++i) dst[i] = v[i];
  } else if constexpr (sizeof(T) == 8) {
    double2* q = reinterpret_cast<double2*>(dst);
#pragma unroll
    for (int i = 0; i < M; ++i) q[i] = make_double2(v[i].re, v[i].im);
  } else {
#pragma unroll
    for (int i = 0; i < M; ++i) dst[i] = v[i];
  }
}

// The table rows of one window, [q][row][ab] with row = r_first .. r_first + R - 1,
// into shared memory; rows below 0 by the parity Z_q(-rho) = (-1)^q Z_q(rho),
// rows past the table as zeros (never inside a stencil).
template <class T, int M>
__device__ __forceinline__ void load_window(const FillArgs<T, T>& a, const cpx<T>* tab_cls, int r_first,
                                            int R, cpx<T>* S) {
  constexpr int P2 = M * M;
  const int total = a.n_harm * R * P2;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int ab = e % P2;
    const int rest = e / P2;
    const int qi = rest / R;
    const int lr = rest - qi * R;
    int r = r_first + lr;
    cpx<T> v = mk((T)0, (T)0);
    if (r < a.n_rho) {
      const bool neg = r < 0;
      if (neg) r = -r;
      v = tab_cls[((size_t)ab * a.n_harm + qi) * a.n_rho + r];
      if (neg && ((qi - a.q_max) & 1)) v = mk(-v.re, -v.im);
    }
    S[e] = v;
  }
}

// Lagrange weights at x on the nodes 0..TAPS-1 (Eq. 9's interpolation), and with
// SLOPE their derivatives d/dx, from prefix and suffix products of (x - j)
template <class T, int TAPS, bool SLOPE>
__device__ __forceinline__ void stencil_weights(T x, T* wt, T* dwt) {
  T den[TAPS];
#pragma unroll
  for (int t = 0; t < TAPS; ++t) {
    long long d = 1;
#pragma unroll
    for (int j = 0; j < TAPS; ++j)
      if (j != t) d *= (long long)(t - j);
    den[t] = (T)1 / (T)d;
  }
  T pre = (T)1, dpre = (T)0;
#pragma unroll
  for (int t = 0; t < TAPS; ++t) {
    wt[t] = pre;
    if (SLOPE) {
      dwt[t] = dpre;
      dpre = dpre * (x - (T)t) + pre;
    }
    pre *= (x - (T)t);
  }
  T suf = (T)1, dsuf = (T)0;
#pragma unroll
  for (int t = TAPS - 1; t >= 0; --t) {
    if (SLOPE) {
      dwt[t] = (dwt[t] * suf + wt[t] * dsuf) * den[t];
      dsuf = dsuf * (x - (T)t) + suf;
    }
    wt[t] *= suf * den[t];
    suf *= (x - (T)t);
  }
}

template <class T, int M, int TAPS>
__global__ void __launch_bounds__(kBThreads, 2) bucket_fill_kernel(FillArgs<T, T> a, BucketArgs b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int HALF = TAPS / 2 - 1;
  constexpr int P2 = M * M;
  const int w = blockIdx.x, cls = blockIdx.y, blk = blockIdx.z;
  const int cell0 = w * b.win;
  if (cell0 >= b.n_cells) return;
  const int cell1 = min(cell0 + b.win, b.n_cells);
  const size_t kbase = ((size_t)blk * b.n_ck + cls) * b.n_cells;
  const unsigned p0 = b.off[kbase + cell0], p1 = b.off[kbase + cell1];
  if (p0 == p1) return;
  const int R = b.win + TAPS - 1;       // table rows of the window
  const int r_first = cell0 - HALF;     // table row of window row 0
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smem_raw);
  load_window<T, M>(a, a.table + (size_t)cls * P2 * a.n_harm * a.n_rho, r_first, R, S);
  __syncthreads();
  const unsigned nmask = (1u << b.nb_bits) - 1u;
  for (unsigned p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const unsigned code = b.list[p];
    const int n = (int)(code & nmask);
    const int m = b.m0 + blk * b.br + (int)(code >> b.nb_bits);
    const BGeom<T> g = bucket_geom<T, TAPS>(a, b, m, n);
    const int lr0 = g.i0 - r_first;
    if (lr0 < 0 || lr0 >= b.win) {  // a stencil outside its bucket's window: never expected
      atomicOr(a.err, 2);
      continue;
    }
    T wt[TAPS];
    stencil_weights<T, TAPS, false>(g.x, wt, nullptr);
    const cpx<T> e1 = mk(g.ex, g.ey);
    cpx<T> zq = mk((T)1, (T)0);  // exp(-i q_max phi)
    for (int k = 0; k < a.q_max; ++k) zq = zq * conj(e1);
    cpx<T>* zrow = a.z + (size_t)m * M * a.ld + (size_t)n * M;
#pragma unroll 1
    for (int ia = 0; ia < M; ++ia) {
      cpx<T> acc[M];
#pragma unroll
      for (int ib = 0; ib < M; ++ib) acc[ib] = mk((T)0, (T)0);
      cpx<T> ph = zq;
      const cpx<T>* sp = S + (size_t)lr0 * P2 + ia * M;
#pragma unroll 1
      for (int qi = 0; qi < a.n_harm; ++qi) {
        // all stencil rows of this (q, a) first (independent loads in flight), then the FMAs
        cpx<T> row[TAPS][M];
#pragma unroll
        for (int t = 0; t < TAPS; ++t) load_row<T, M>(sp + t * P2, row[t]);
        cpx<T> v[M];
#pragma unroll
        for (int ib = 0; ib < M; ++ib) v[ib] = mk((T)0, (T)0);
#pragma unroll
        for (int t = 0; t < TAPS; ++t) {
#pragma unroll
          for (int ib = 0; ib < M; ++ib) {
            v[ib].re = fma(wt[t], row[t][ib].re, v[ib].re);
            v[ib].im = fma(wt[t], row[t][ib].im, v[ib].im);
          }
        }
#pragma unroll
        for (int ib = 0; ib < M; ++ib) cmac(acc[ib], ph, v[ib]);
        ph = ph * e1;
        sp += (size_t)R * P2;
      }
      store_row<T, M>(zrow + (size_t)ia * a.ld, acc, b.vec_out != 0);
    }
  }
}

// Adjoint of the fill over the same buckets.  With dL = Re sum conj(G) dZ and
//   Z_ab(m, n) = sum_q e^{i q phi} sum_t w_t(x) Z^{cls}_ab,q(i0 + t),
// POS = true takes, per pair, D = dZ/dx (weights w') and Q = sum_q q e^{i q phi} (...)
// (dZ/dphi = i Q), and from s_rho = Re sum conj(G) D / d_rho and
// s_phi = -Im sum conj(G) Q the gradient with respect to Delta = r_m - r_n through
// rho and phi; it is added to element m and subtracted from element n.  POS =
// false contracts conj(G) with the fill of a derivative table (table = dZ/d theta,
// contour held fixed) into one scalar, d L / d theta.
template <class T>
struct AdjArgs {
  const cpx<T>* grad;    // dL/dZ, entry (m*M + a, n*M + b) at (m*M + a) * ld_g + n*M + b
  int64_t ld_g;
  int vec_g;             // grad rows 16-byte aligned: vector loads
  double* grad_pos;      // [2 * n_el], accumulated (POS)
  double* grad_theta;    // one scalar, accumulated (!POS)
};

template <class T, int M, int TAPS, bool POS>
__global__ void __launch_bounds__(kBThreads, sizeof(T) == 4 ? 2 : 1) bucket_adjoint_kernel(FillArgs<T, T> a, BucketArgs b,
                                                                      AdjArgs<T> g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int HALF = TAPS / 2 - 1;
  constexpr int P2 = M * M;
  const int w = blockIdx.x, cls = blockIdx.y, blk = blockIdx.z;
  const int cell0 = w * b.win;
  if (cell0 >= b.n_cells) return;
  const int cell1 = min(cell0 + b.win, b.n_cells);
  const size_t kbase = ((size_t)blk * b.n_ck + cls) * b.n_cells;
  const unsigned p0 = b.off[kbase + cell0], p1 = b.off[kbase + cell1];
  if (p0 == p1) return;
  const int R = b.win + TAPS - 1;
  const int r_first = cell0 - HALF;
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smem_raw);
  load_window<T, M>(a, a.table + (size_t)cls * P2 * a.n_harm * a.n_rho, r_first, R, S);
  __syncthreads();
  const unsigned nmask = (1u << b.nb_bits) - 1u;
  double theta_sum = 0.0;
  for (unsigned p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const unsigned code = b.list[p];
    const int n = (int)(code & nmask);
    const int m = b.m0 + blk * b.br + (int)(code >> b.nb_bits);
    if (POS && m == n) continue;   // Z(m, m) does not depend on the positions
    const BGeom<T> geo = bucket_geom<T, TAPS>(a, b, m, n);
    const int lr0 = geo.i0 - r_first;
    if (lr0 < 0 || lr0 >= b.win) {
      atomicOr(a.err, 2);
      continue;
    }
    T wt[TAPS], dwt[TAPS];
    stencil_weights<T, TAPS, POS>(geo.x, wt, dwt);
    const cpx<T> e1 = mk(geo.ex, geo.ey);
    cpx<T> zq = mk((T)1, (T)0);
    for (int k = 0; k < a.q_max; ++k) zq = zq * conj(e1);
    const cpx<T>* grow = g.grad + (size_t)m * M * g.ld_g + (size_t)n * M;
    T s_a = (T)0, s_b = (T)0;
#pragma unroll 1
    for (int ia = 0; ia < M; ++ia) {
      cpx<T> accA[M], accB[M];
#pragma unroll
      for (int ib = 0; ib < M; ++ib) accA[ib] = accB[ib] = mk((T)0, (T)0);
      cpx<T> ph = zq;
      T qf = (T)(-a.q_max);
      const cpx<T>* sp = S + (size_t)lr0 * P2 + ia * M;
#pragma unroll 1
      for (int qi = 0; qi < a.n_harm; ++qi) {
        cpx<T> v[M], dv[M];
#pragma unroll
        for (int ib = 0; ib < M; ++ib) v[ib] = dv[ib] = mk((T)0, (T)0);
#pragma unroll
        for (int t = 0; t < TAPS; ++t) {
          cpx<T> row[M];
          load_row<T, M>(sp + t * P2, row);
#pragma unroll
          for (int ib = 0; ib < M; ++ib) {
            v[ib].re = fma(wt[t], row[ib].re, v[ib].re);
            v[ib].im = fma(wt[t], row[ib].im, v[ib].im);
            if (POS) {
              dv[ib].re = fma(dwt[t], row[ib].re, dv[ib].re);
              dv[ib].im = fma(dwt[t], row[ib].im, dv[ib].im);
            }
          }
        }
#pragma unroll
        for (int ib = 0; ib < M; ++ib) {
          if (POS) {
            cmac(accA[ib], ph, dv[ib]);
            const cpx<T> pv = ph * v[ib];
            accB[ib].re = fma(qf, pv.re, accB[ib].re);
            accB[ib].im = fma(qf, pv.im, accB[ib].im);
          } else {
            cmac(accA[ib], ph, v[ib]);
          }
        }
        ph = ph * e1;
        qf += (T)1;
        sp += (size_t)R * P2;
      }
      cpx<T> gv[M];
      load_grad_row<T, M>(grow + (size_t)ia * g.ld_g, gv, g.vec_g != 0);
#pragma unroll
      for (int ib = 0; ib < M; ++ib) {
        // Re(conj(G) A) and Im(conj(G) B)
        s_a += gv[ib].re * accA[ib].re + gv[ib].im * accA[ib].im;
        if (POS) s_b += gv[ib].re * accB[ib].im - gv[ib].im * accB[ib].re;
      }
    }
    if (POS) {
      const double s_rho = (double)s_a * a.inv_d_rho;   // d/d rho = (1 / d_rho) d/dx
      const double s_phi = -(double)s_b;
      const double c = (double)geo.ex, sn = (double)geo.ey, rho = (double)geo.rho;
      const double gx = s_rho * c - s_phi * sn / rho;
      const double gy = s_rho * sn + s_phi * c / rho;
      atomicAdd(&g.grad_pos[2 * m], gx);
      atomicAdd(&g.grad_pos[2 * m + 1], gy);
      atomicAdd(&g.grad_pos[2 * n], -gx);
      atomicAdd(&g.grad_pos[2 * n + 1], -gy);
    } else {
      theta_sum += (double)s_a;
    }
  }
  if (!POS) {
    __shared__ double red[kBThreads / 32];
    double v = theta_sum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0; i < kBThreads / 32; ++i) t += red[i];
      atomicAdd(g.grad_theta, t);
    }
  }
}


// ---- the fill of M = 4 on the tensor cores (FP32-mixed, 8 taps)
//
// For the pairs of one stencil cell (table rows i0 .. i0 + 7 of one class) the
// harmonic sum is a product with the cell's table slice, and the tap sum follows:
//   D_p[t][ab] = sum_q e^{iq phi_p} T[q][i0+t][ab],   Z_p[ab] = sum_t w_t(x_p) D_p[t][ab].
// The first is a real GEMM D (pairs x 256) = A (pairs x K) B (K x 256), K = 2 per
// harmonic (padded to a multiple of 8), n = 2 (16 t + ab) + re/im:
//   A(p, 2 qi) = Re e^{iq phi},  A(p, 2 qi + 1) = Im e^{iq phi},
//   B(2 qi, 2 j) = Re T,  B(2 qi + 1, 2 j) = -Im T,  B(2 qi, 2 j + 1) = Im T,  B(2 qi + 1, 2 j + 1) = Re T.
// A CTA owns one (cell, class, row block): B (TF32 head and tail) stays in shared
// memory; the pairs go through in M-tiles of 128: the A tile (both halves of the
// CTA form one row's harmonics each), three TF32 products of width 256 into one of
// two tensor-memory accumulators (27 accumulation steps per tile: the truncating
// accumulation stays near 1e-7), and while the tensor core runs tile j each thread
// reads one MBF-row pair (a = 2h, 2h+1) of its pair's D of tile j-1 and applies the
// Lagrange weights.
constexpr int kFcTaps = 8;
constexpr int kFcN = 256;            // 8 taps x 16 MBF pairs x (re, im)

__host__ __device__ constexpr int fc_kpad(int n_harm) { return (2 * n_harm + 7) & ~7; }

size_t fc_smem_bytes(int n_harm) {
  return (size_t)2 * kFcN * fc_kpad(n_harm) * 4 +      // B head, tail
         (size_t)2 * 128 * fc_kpad(n_harm) * 4 + 1024; // A head, tail + alignment
}

// staged table slice: [ab][qi][t] with 9 entries per (ab, qi), so that the reads of
// consecutive ab (as consecutive threads make them) fall on distinct banks
constexpr int kStgPitch = kFcTaps + 1;

// The B operand of one stencil cell (table rows i0 .. i0 + 7 of one class table):
// [ab][qi][t] staged in stg with coalesced loads (parity below row 0, zero past the
// end), then written as TF32 head and tail in the K-major layout, column n = 2 (16 t +
// ab) + re/im, K = 2 qi + re/im of the A operand.  Ends with a CTA barrier.
__device__ __forceinline__ void fc_build_b(const cpx<float>* tab_cls, int n_rho, int q_max, int nh, int kpad,
                                           int i0, float* Bh, float* Bl, cpx<float>* stg) {
  const int tid = threadIdx.x;
  {
    // the cell's table rows, staged as [ab][qi][t] in the (still unused) A buffer with
    // coalesced loads (8 consecutive rows per (ab, qi)); parity below row 0, zero past the end
    const cpx<float>* tab = tab_cls;
    const int n_st = 16 * nh * kFcTaps;
    const bool inside = i0 >= 0 && i0 + kFcTaps <= n_rho;
#pragma unroll 4
    for (int e = tid; e < n_st; e += blockDim.x) {
      const int t = e & 7, rest = e >> 3;
      const int qi = rest % nh, ab = rest / nh;
      int r = i0 + t;
      cpx<float> v = mk(0.f, 0.f);
      if (inside) {
        v = tab[((size_t)ab * nh + qi) * n_rho + r];
      } else if (r < n_rho) {
        const bool neg = r < 0;
        if (neg) r = -r;
        v = tab[((size_t)ab * nh + qi) * n_rho + r];
        if (neg && ((qi - q_max) & 1)) v = mk(-v.re, -v.im);
      }
      stg[(size_t)rest * kStgPitch + t] = v;
    }
    __syncthreads();
    // one 16-byte group per (column n, harmonics qi, qi + 1): consecutive threads take
    // consecutive n, so the eight rows of a core matrix are written in one wavefront
    const int total = kFcN * (kpad / 4);
    for (int e = tid; e < total; e += blockDim.x) {
      const int n = e & (kFcN - 1), k4 = e / kFcN;
      const int j = n >> 1, c = n & 1, t = j >> 4, ab = j & 15;
      float f[4];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int qi = 2 * k4 + u;
        const cpx<float> v = qi < nh ? stg[((size_t)ab * nh + qi) * kStgPitch + t] : mk(0.f, 0.f);
        // column 2j (real part of D): (Re T, -Im T); column 2j + 1: (Im T, Re T)
        f[2 * u] = c ? v.im : v.re;
        f[2 * u + 1] = c ? v.re : -v.im;
      }
      float4 h, l;
      tf32_split(f[0], h.x, l.x);
      tf32_split(f[1], h.y, l.y);
      tf32_split(f[2], h.z, l.z);
      tf32_split(f[3], h.w, l.w);
      const uint32_t off = tc::kmajor_offset(n, 4 * k4, kpad) / 4;
      *reinterpret_cast<float4*>(Bh + off) = h;
      *reinterpret_cast<float4*>(Bl + off) = l;
    }
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
}

// Row r of an A tile: e^{iq phi} (qweight: q e^{iq phi}) for the harmonic pairs
// (qi, qi + 1), qi = 4 u + 2 half, one 16-byte group each, TF32 head and tail; zero when !ok
__device__ __forceinline__ void fc_write_a(int r, int half, bool ok, cpx<float> e1, int q_max, int nh, int kpad,
                                           bool qweight, float* Ah, float* Al) {
  const cpx<float> e2 = e1 * e1, e4 = e2 * e2;
  cpx<float> ph = mk(ok ? 1.f : 0.f, 0.f);
  for (int k = 0; k < q_max; ++k) ph = ph * conj(e1);   // q = -q_max
  if (half) ph = ph * e2;                                 // q = -q_max + 2
  for (int qi = 2 * half; 2 * qi < kpad; qi += 4) {
    cpx<float> v0 = qi < nh ? ph : mk(0.f, 0.f);
    const cpx<float> p1v = ph * e1;
    cpx<float> v1 = qi + 1 < nh ? p1v : mk(0.f, 0.f);
    if (qweight) {
      const float q0 = (float)(qi - q_max), q1 = q0 + 1.f;
      v0 = mk(q0 * v0.re, q0 * v0.im);
      v1 = mk(q1 * v1.re, q1 * v1.im);
    }
    float4 h, l;
    tf32_split(v0.re, h.x, l.x);
    tf32_split(v0.im, h.y, l.y);
    tf32_split(v1.re, h.z, l.z);
    tf32_split(v1.im, h.w, l.w);
    const uint32_t off = tc::kmajor_offset(r, 2 * qi, kpad) / 4;
    *reinterpret_cast<float4*>(Ah + off) = h;
    *reinterpret_cast<float4*>(Al + off) = l;
    ph = ph * e4;
  }
}

// D (128 x 256, fp32 in tensor memory at d) = A B as three TF32 products (one thread)
__device__ __forceinline__ void fc_mma(uint32_t d, const float* Ah, const float* Al, const float* Bh,
                                       const float* Bl, int kpad, uint32_t sbo, uint32_t idesc) {
  const uint32_t a_hi = tc::smem_u32(Ah), a_lo = tc::smem_u32(Al);
  const uint32_t b_hi = tc::smem_u32(Bh), b_lo = tc::smem_u32(Bl);
  for (int ks = 0; ks < kpad / 8; ++ks) {
    const uint32_t ko = ks * 256;
    const uint64_t dah = tc::sdesc(a_hi + ko, 128, sbo), dal = tc::sdesc(a_lo + ko, 128, sbo);
    const uint64_t dbh = tc::sdesc(b_hi + ko, 128, sbo), dbl = tc::sdesc(b_lo + ko, 128, sbo);
    tc::mma_tf32(d, dah, dbl, idesc, ks > 0 ? 1u : 0u);
    tc::mma_tf32(d, dal, dbh, idesc, 1u);
    tc::mma_tf32(d, dah, dbh, idesc, 1u);
  }
}

__global__ void __launch_bounds__(kBThreads, 1) fill_tc_kernel(FillArgs<float, float> a, BucketArgs b) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int HALF = kFcTaps / 2 - 1;
  __shared__ uint64_t mbar;
  __shared__ uint32_t taddr_s;
  __shared__ int s_fail;
  const int cell = blockIdx.x, cls = blockIdx.y, blk = blockIdx.z;
  const size_t key = ((size_t)blk * b.n_ck + cls) * b.n_cells + cell;
  const unsigned p0 = b.off[key], p1 = b.off[key + 1];
  if (p0 == p1) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nh = a.n_harm;
  const int kpad = fc_kpad(nh);
  const uint32_t sbo = (uint32_t)(kpad / 4) * 128u;
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  float* Bh = reinterpret_cast<float*>(base);
  float* Bl = Bh + (size_t)kFcN * kpad;
  float* Ah = Bl + (size_t)kFcN * kpad;
  float* Al = Ah + (size_t)128 * kpad;
  if (tid == 0) {
    s_fail = 0;
    tc::mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tc::tmem_alloc(&taddr_s, 512);
    tc::tmem_relinquish();
  }
  // ---- B: the cell's table rows i0 .. i0 + 7 (parity below row 0, zero past the end;
  // K rows past 2 n_harm are zero)
  const int i0 = cell - HALF;
  const cpx<float>* tab_cls = a.table + (size_t)cls * 16 * nh * a.n_rho;
  fc_build_b(tab_cls, a.n_rho, a.q_max, nh, kpad, i0, Bh, Bl, reinterpret_cast<cpx<float>*>(Ah));
  const uint32_t tmem = taddr_s;
  const uint32_t idesc = tc::idesc_tf32(128, kFcN);
  const int r = tid & 127, half = tid >> 7;
  const unsigned nmask = (1u << b.nb_bits) - 1u;
  uint32_t n_commit = 0;
  uint32_t n_issued = 0;   // products committed (thread 0)
  // Z of a tile from accumulator set `set`: this thread's pair (row r; MBF rows
  // a = 2 half, 2 half + 1) with stencil coordinate x, if ok
  auto epilogue = [&](uint32_t set, bool ok, int mm, int nn, float x) {
    float wt[kFcTaps];
    stencil_weights<float, kFcTaps, false>(x, wt, nullptr);
    float z[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) z[u] = 0.f;
    const uint32_t tl = tmem + set * kFcN + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(16 * half);
#pragma unroll
    for (int t = 0; t < kFcTaps; t += 2) {
      float v[16], w[16];
      tc::tmem_ld16x2(tl + 32 * t, tl + 32 * (t + 1), v, w);
#pragma unroll
      for (int u = 0; u < 16; ++u) z[u] = fmaf(wt[t + 1], w[u], fmaf(wt[t], v[u], z[u]));
    }
    if (ok) {
#pragma unroll
      for (int u2 = 0; u2 < 2; ++u2) {
        cpx<float> zz[4];
#pragma unroll
        for (int ib = 0; ib < 4; ++ib) zz[ib] = mk(z[8 * u2 + 2 * ib], z[8 * u2 + 2 * ib + 1]);
        store_row<float, 4>(a.z + ((size_t)mm * 4 + 2 * half + u2) * a.ld + (size_t)nn * 4, zz, b.vec_out != 0);
      }
    }
  };
  // this thread's pair of the next tile: code and split positions, loaded ahead
  auto fetch = [&](unsigned t0, bool& ok, int& m, int& n, float4& pm, float4& pn) {
    const unsigned pidx = t0 + (unsigned)r;
    ok = pidx < p1;
    m = n = 0;
    if (ok) {
      const unsigned code = b.list[pidx];
      n = (int)(code & nmask);
      m = b.m0 + blk * b.br + (int)(code >> b.nb_bits);
      pm = b.ps[m];
      pn = b.ps[n];
    }
  };
  bool nx_ok;
  int nx_m, nx_n;
  float4 nx_pm = make_float4(0.f, 0.f, 0.f, 0.f), nx_pn = nx_pm;
  fetch(p0, nx_ok, nx_m, nx_n, nx_pm, nx_pn);
  bool pv_ok = false, have_prev = false;
  int pv_m = 0, pv_n = 0;
  float pv_x = 0.f;
  for (unsigned t0 = p0; t0 < p1; t0 += 128) {
    const bool ok0 = nx_ok;
    const int m0 = nx_m, n0 = nx_n;
    float x0 = 0.f;
    bool ok = ok0;
    // ---- A row r: e^{iq phi} of this thread's pair; harmonic pairs (qi, qi + 1) with
    // qi = 4 u + 2 half, one 16-byte group each
    {
      cpx<float> e1 = mk(1.f, 0.f);
      if (ok) {
        const BGeom<float> g = bucket_geom_ps<kFcTaps>(a, b, nx_pm, nx_pn);
        if (g.i0 != i0) {   // a pair outside its bucket's cell: never expected
          atomicOr(a.err, 2);
          ok = false;
        }
        e1 = mk(g.ex, g.ey);
        x0 = g.x;
      }
      fc_write_a(r, half, ok, e1, a.q_max, nh, kpad, false, Ah, Al);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    const uint32_t set = n_commit & 1u;
    if (tid == 0 && !s_fail) {
      tc::fence_after_sync();
      fc_mma(tmem + set * kFcN, Ah, Al, Bh, Bl, kpad, sbo, idesc);
      tc::mma_commit(&mbar);
      ++n_issued;
    }
    // while the tensor core runs this tile: the next tile's pairs, the previous tile's Z
    if (t0 + 128 < p1) fetch(t0 + 128, nx_ok, nx_m, nx_n, nx_pm, nx_pn);
    if (have_prev && !__shfl_sync(0xffffffffu, *reinterpret_cast<volatile int*>(&s_fail), 0))
      epilogue(set ^ 1u, pv_ok, pv_m, pv_n, pv_x);
    // this tile's products done: the A buffer is free, its accumulator readable
    if (lane == 0 && !s_fail && !tc::mbar_wait(&mbar, n_commit & 1u, kTcPolls)) atomicOr(&s_fail, 1);
    __syncwarp();
    ++n_commit;
    tc::fence_after_sync();
    tc::fence_before_sync();
    __syncthreads();
    if (s_fail) break;
    pv_ok = ok;
    pv_m = m0;
    pv_n = n0;
    pv_x = x0;
    have_prev = true;
  }
  if (have_prev && !s_fail) epilogue((n_commit - 1) & 1u, pv_ok, pv_m, pv_n, pv_x);
  if (s_fail && tid == 0) {
    atomicOr(a.err, 16);
    // the products whose wait ran out may still be writing tensor memory: wait for them
    // once more (bounded) before it is released
    if (n_issued > 0) tc::mbar_wait(&mbar, (n_issued - 1) & 1u, kTcPolls);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}


// Adjoint of the fill on the tensor cores, over the same per-cell buckets
// (dL = Re sum conj(G) dZ', G = dL/dZ').  POS: two products with the cell's table
// slice, D (A = e^{iq phi}) and Dq (A = q e^{iq phi}), in the two accumulators; per pair
//   s_rho = Re sum_ab conj(G_ab) sum_t w'_t D[t][ab] / d_rho   (d Z'/d rho, the slope weights)
//   s_phi = -Im sum_ab conj(G_ab) sum_t w_t Dq[t][ab]          (d Z'/d phi = i sum_q q ...)
// give dL/d(r_m - r_n) through rho and phi (added to m, subtracted from n).  !POS: the
// table is a derivative table; sum_ab Re conj(G_ab) sum_t w_t D[t][ab] goes into one scalar.
template <bool POS>
__global__ void __launch_bounds__(kBThreads, 1) adjoint_tc_kernel(FillArgs<float, float> a, BucketArgs b,
                                                                  AdjArgs<float> g) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int HALF = kFcTaps / 2 - 1;
  __shared__ uint64_t mbar;
  __shared__ uint32_t taddr_s;
  __shared__ int s_fail;
  __shared__ float part[2][128];
  __shared__ double red[kBThreads / 32];
  const int cell = blockIdx.x, cls = blockIdx.y, blk = blockIdx.z;
  const size_t key = ((size_t)blk * b.n_ck + cls) * b.n_cells + cell;
  const unsigned p0 = b.off[key], p1 = b.off[key + 1];
  if (p0 == p1) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nh = a.n_harm;
  const int kpad = fc_kpad(nh);
  const uint32_t sbo = (uint32_t)(kpad / 4) * 128u;
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  float* Bh = reinterpret_cast<float*>(base);
  float* Bl = Bh + (size_t)kFcN * kpad;
  float* Ah = Bl + (size_t)kFcN * kpad;
  float* Al = Ah + (size_t)128 * kpad;
  if (tid == 0) {
    s_fail = 0;
    tc::mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tc::tmem_alloc(&taddr_s, 512);
    tc::tmem_relinquish();
  }
  const int i0 = cell - HALF;
  fc_build_b(a.table + (size_t)cls * 16 * nh * a.n_rho, a.n_rho, a.q_max, nh, kpad, i0, Bh, Bl,
             reinterpret_cast<cpx<float>*>(Ah));
  const uint32_t tmem = taddr_s;
  const uint32_t idesc = tc::idesc_tf32(128, kFcN);
  const int r = tid & 127, half = tid >> 7;
  const unsigned nmask = (1u << b.nb_bits) - 1u;
  uint32_t n_commit = 0;
  uint32_t n_issued = 0;   // products committed (thread 0)
  double theta_sum = 0.0;
  bool failed = false;
  for (unsigned t0 = p0; t0 < p1 && !failed; t0 += 128) {
    const unsigned pidx = t0 + (unsigned)r;
    bool ok = pidx < p1;
    int m = 0, n = 0;
    BGeom<float> geo{};
    if (ok) {
      const unsigned code = b.list[pidx];
      n = (int)(code & nmask);
      m = b.m0 + blk * b.br + (int)(code >> b.nb_bits);
      geo = bucket_geom<float, kFcTaps>(a, b, m, n);
      if (geo.i0 != i0) {   // a pair outside its bucket's cell: never expected
        atomicOr(a.err, 2);
        ok = false;
      }
      if (POS && m == n) ok = false;   // Z'(m, m) does not depend on the positions
    }
    const cpx<float> e1 = ok ? mk(geo.ex, geo.ey) : mk(1.f, 0.f);
#pragma unroll 1
    for (int pass = 0; pass < (POS ? 2 : 1); ++pass) {
      fc_write_a(r, half, ok, e1, a.q_max, nh, kpad, pass == 1, Ah, Al);
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();
      if (tid == 0 && !s_fail) {
        tc::fence_after_sync();
        fc_mma(tmem + (uint32_t)pass * kFcN, Ah, Al, Bh, Bl, kpad, sbo, idesc);
        tc::mma_commit(&mbar);
        ++n_issued;
      }
      // the products are done before any warp rewrites the A tile or reads the result
      if (lane == 0 && !s_fail && !tc::mbar_wait(&mbar, n_commit & 1u, kTcPolls)) atomicOr(&s_fail, 1);
      __syncwarp();
      ++n_commit;
    }
    tc::fence_before_sync();
    __syncthreads();
    failed = s_fail != 0;          // uniform: every wait of this tile precedes the barrier
    tc::fence_after_sync();
    if (!failed) {
      float wt[kFcTaps], dwt[kFcTaps];
      stencil_weights<float, kFcTaps, POS>(ok ? geo.x : 0.f, wt, dwt);
      cpx<float> gv[8];
      if (ok) {
#pragma unroll
        for (int u2 = 0; u2 < 2; ++u2)
          load_grad_row<float, 4>(g.grad + ((size_t)m * 4 + 2 * half + u2) * g.ld_g + (size_t)n * 4, gv + 4 * u2,
                                  g.vec_g != 0);
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) gv[j] = mk(0.f, 0.f);
      }
      const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(16 * half);
      float sa = 0.f, sb = 0.f;
      {
        float d[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) d[u] = 0.f;
#pragma unroll
        for (int t = 0; t < kFcTaps; t += 2) {
          float v[16], w[16];
          tc::tmem_ld16x2(tl + 32 * t, tl + 32 * (t + 1), v, w);
          const float c0 = POS ? dwt[t] : wt[t], c1 = POS ? dwt[t + 1] : wt[t + 1];
#pragma unroll
          for (int u = 0; u < 16; ++u) d[u] = fmaf(c1, w[u], fmaf(c0, v[u], d[u]));
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) sa += gv[j].re * d[2 * j] + gv[j].im * d[2 * j + 1];   // Re conj(G) D
      }
      if (POS) {
        float d[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) d[u] = 0.f;
#pragma unroll
        for (int t = 0; t < kFcTaps; t += 2) {
          float v[16], w[16];
          tc::tmem_ld16x2(tl + kFcN + 32 * t, tl + kFcN + 32 * (t + 1), v, w);
#pragma unroll
          for (int u = 0; u < 16; ++u) d[u] = fmaf(wt[t + 1], w[u], fmaf(wt[t], v[u], d[u]));
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) sb += gv[j].re * d[2 * j + 1] - gv[j].im * d[2 * j];   // Im conj(G) Q
        // the two halves of a pair's MBF rows meet in shared memory
        if (half) {
          part[0][r] = sa;
          part[1][r] = sb;
        }
        __syncthreads();
        if (!half && ok) {
          sa += part[0][r];
          sb += part[1][r];
          const double s_rho = (double)sa * a.inv_d_rho;   // d/d rho = (1 / d_rho) d/dx
          const double s_phi = -(double)sb;
          const double c = (double)geo.ex, sn = (double)geo.ey, rho = (double)geo.rho;
          const double gx = s_rho * c - s_phi * sn / rho;
          const double gy = s_rho * sn + s_phi * c / rho;
          atomicAdd(&g.grad_pos[2 * m], gx);
          atomicAdd(&g.grad_pos[2 * m + 1], gy);
          atomicAdd(&g.grad_pos[2 * n], -gx);
          atomicAdd(&g.grad_pos[2 * n + 1], -gy);
        }
      } else if (ok) {
        theta_sum += (double)sa;
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  if (!POS) {
    double v = theta_sum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (tid == 0 && !failed) {
      double t = 0.0;
      for (int i = 0; i < kBThreads / 32; ++i) t += red[i];
      atomicAdd(g.grad_theta, t);
    }
  }
  if (s_fail && tid == 0) {
    atomicOr(a.err, 16);
    // the products whose wait ran out may still be writing tensor memory: wait for them
    // once more (bounded) before it is released
    if (n_issued > 0) tc::mbar_wait(&mbar, (n_issued - 1) & 1u, kTcPolls);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// The scratch layout of a plan and the sort state shared by the fill and its adjoint
template <class T>
BucketArgs bucket_args(const FillArgs<T, T>& a, const FillBucketPlan& pl, void* scratch) {
  BucketArgs b{};
  unsigned char* sp = reinterpret_cast<unsigned char*>(scratch);
  b.ps = reinterpret_cast<const float4*>(sp);
  sp += ((size_t)a.n_el * sizeof(float4) + 255) / 256 * 256;
  b.cursor = reinterpret_cast<unsigned*>(sp);
  sp += (pl.n_keys_max * sizeof(unsigned) + 255) / 256 * 256;
  b.off = reinterpret_cast<unsigned*>(sp);
  sp += ((pl.n_keys_max + 1) * sizeof(unsigned) + 255) / 256 * 256;
  b.seg = reinterpret_cast<unsigned*>(sp);
  sp += 1024 * sizeof(unsigned);
  b.list = reinterpret_cast<unsigned*>(sp);
  b.br = pl.block_rows;
  b.nb_bits = pl.nb_bits;
  b.n_ck = a.n_cls;
  b.n_cells = pl.n_cells;
  b.win = pl.win;
  const double inv = a.inv_d_rho;
  b.ih = (float)inv;
  b.il = (float)(inv - (double)b.ih);
  b.vec_out = (a.z != nullptr && (reinterpret_cast<uintptr_t>(a.z) & 15) == 0 &&
               ((size_t)a.ld * sizeof(cpx<T>)) % 16 == 0) ? 1 : 0;
  return b;
}

// Waves of whole row blocks: per wave the counting sort (count, scan, scatter) of its
// pairs, then `consume(b, grid)` launches the kernels that walk the buckets.
template <class T, int TAPS, class Consume>
cudaError_t run_waves(const FillArgs<T, T>& a, const FillBucketPlan& pl, BucketArgs b, cudaStream_t s,
                      Consume consume) {
  if (sizeof(T) == 4) {
    split_positions_kernel<<<(a.n_el + 255) / 256, 256, 0, s>>>(a.pos, a.n_el,
                                                              const_cast<float4*>(b.ps));
  }
  const int n_windows = (pl.n_cells + pl.win - 1) / pl.win;
  for (int m0 = 0; m0 < a.n_el; m0 += pl.rows_per_wave) {
    b.m0 = m0;
    b.rows = min(pl.rows_per_wave, a.n_el - m0);
    const int n_blocks = (b.rows + b.br - 1) / b.br;
    const size_t n_keys = (size_t)n_blocks * b.n_ck * b.n_cells;
    cudaError_t e = cudaMemsetAsync(b.cursor, 0, n_keys * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    dim3 sg((a.n_el + kBThreads - 1) / kBThreads, min(b.rows, 65535));
    bucket_sort_kernel<T, TAPS, false><<<sg, kBThreads, 0, s>>>(a, b);
    const int n_seg = (int)((n_keys + kScanSeg - 1) / kScanSeg);
    if (n_seg > 1024) return cudaErrorInvalidValue;
    scan_segment_sums<<<n_seg, 1024, 0, s>>>(b.cursor, n_keys, b.seg);
    scan_segment_offsets<<<1, 1024, 0, s>>>(b.seg, n_seg, b.off, n_keys);
    scan_apply<<<n_seg, 1024, 0, s>>>(b.cursor, b.off, n_keys, b.seg);
    bucket_sort_kernel<T, TAPS, true><<<sg, kBThreads, 0, s>>>(a, b);
    e = consume(b, dim3(n_windows, b.n_ck, n_blocks));
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <class T, int M, int TAPS>
cudaError_t run_bucketed(const FillArgs<T, T>& a, const FillBucketPlan& pl, void* scratch, cudaStream_t s) {
  const size_t smem = pl.smem;
  cudaError_t e = cudaFuncSetAttribute(bucket_fill_kernel<T, M, TAPS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return run_waves<T, TAPS>(a, pl, bucket_args(a, pl, scratch), s, [&](const BucketArgs& b, dim3 fg) {
    bucket_fill_kernel<T, M, TAPS><<<fg, kBThreads, smem, s>>>(a, b);
    return cudaSuccess;
  });
}

template <class T, int M, int TAPS>
cudaError_t run_adjoint(const FillArgs<T, T>& a, const FillAdjointArgs<T>& ad, const FillBucketPlan& pl,
                        void* scratch, cudaStream_t s) {
  const size_t smem = pl.smem;
  cudaError_t e = cudaFuncSetAttribute(bucket_adjoint_kernel<T, M, TAPS, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(bucket_adjoint_kernel<T, M, TAPS, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  AdjArgs<T> g{};
  g.grad = ad.grad;
  g.ld_g = ad.ld_g;
  g.vec_g = ((reinterpret_cast<uintptr_t>(ad.grad) & 15) == 0 &&
             ((size_t)ad.ld_g * sizeof(cpx<T>)) % 16 == 0) ? 1 : 0;
  return run_waves<T, TAPS>(a, pl, bucket_args(a, pl, scratch), s, [&](const BucketArgs& b, dim3 fg) {
    if (ad.grad_pos) {
      AdjArgs<T> gp = g;
      gp.grad_pos = ad.grad_pos;
      bucket_adjoint_kernel<T, M, TAPS, true><<<fg, kBThreads, smem, s>>>(a, b, gp);
    }
    if (ad.grad_theta && ad.dtab_eps && ad.dtab_h) {
      const cpx<T>* dt[2] = {ad.dtab_eps, ad.dtab_h};
      for (int c = 0; c < 2; ++c) {
        FillArgs<T, T> ac = a;
        ac.table = dt[c];
        AdjArgs<T> gt = g;
        gt.grad_theta = ad.grad_theta + c;
        bucket_adjoint_kernel<T, M, TAPS, false><<<fg, kBThreads, smem, s>>>(ac, b, gt);
      }
    }
    return cudaSuccess;
  });
}

cudaError_t run_adjoint_tc(const FillArgs<float, float>& a, const FillAdjointArgs<float>& ad,
                           const FillBucketPlan& pl, void* scratch, cudaStream_t s) {
  const size_t smem = pl.smem;
  cudaError_t e = cudaFuncSetAttribute(adjoint_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(adjoint_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  AdjArgs<float> g{};
  g.grad = ad.grad;
  g.ld_g = ad.ld_g;
  g.vec_g = ((reinterpret_cast<uintptr_t>(ad.grad) & 15) == 0 && ((size_t)ad.ld_g * sizeof(cpx<float>)) % 16 == 0)
                ? 1 : 0;
  return run_waves<float, kFcTaps>(a, pl, bucket_args(a, pl, scratch), s, [&](const BucketArgs& b, dim3 fg) {
    if (ad.grad_pos) {
      AdjArgs<float> gp = g;
      gp.grad_pos = ad.grad_pos;
      adjoint_tc_kernel<true><<<fg, kBThreads, smem, s>>>(a, b, gp);
    }
    if (ad.grad_theta && ad.dtab_eps && ad.dtab_h) {
      const cpx<float>* dt[2] = {ad.dtab_eps, ad.dtab_h};
      for (int c = 0; c < 2; ++c) {
        FillArgs<float, float> ac = a;
        ac.table = dt[c];
        AdjArgs<float> gt = g;
        gt.grad_theta = ad.grad_theta + c;
        adjoint_tc_kernel<false><<<fg, kBThreads, smem, s>>>(ac, b, gt);
      }
    }
    return cudaSuccess;
  });
}

cudaError_t run_fill_tc(const FillArgs<float, float>& a, const FillBucketPlan& pl, void* scratch, cudaStream_t s) {
  const size_t smem = pl.smem;
  cudaError_t e = cudaFuncSetAttribute(fill_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return run_waves<float, kFcTaps>(a, pl, bucket_args(a, pl, scratch), s, [&](const BucketArgs& b, dim3 fg) {
    fill_tc_kernel<<<fg, kBThreads, smem, s>>>(a, b);
    return cudaSuccess;
  });
}

template <class T, int M>
cudaError_t run_taps(const FillArgs<T, T>& a, const FillBucketPlan& pl, void* scratch, cudaStream_t s) {
  switch (a.taps) {
    case 8: return run_bucketed<T, M, 8>(a, pl, scratch, s);
    case 12: return run_bucketed<T, M, 12>(a, pl, scratch, s);
    case 16: return run_bucketed<T, M, 16>(a, pl, scratch, s);
    default: return cudaErrorInvalidValue;
  }
}

template <class T, int M>
cudaError_t adjoint_taps(const FillArgs<T, T>& a, const FillAdjointArgs<T>& ad, const FillBucketPlan& pl,
                         void* scratch, cudaStream_t s) {
  switch (a.taps) {
    case 8: return run_adjoint<T, M, 8>(a, ad, pl, scratch, s);
    case 12: return run_adjoint<T, M, 12>(a, ad, pl, scratch, s);
    case 16: return run_adjoint<T, M, 16>(a, ad, pl, scratch, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// Plan of the bucketed fill, or plan.ok = false when it does not apply (the
// per-row fill runs instead): M in {1, 2, 4}, taps in {8, 12, 16}, and a
// window of at least 4 stencil starts fitting in shared memory.
template <class T>
FillBucketPlan plan_fill_bucketed(int n_el, int n_mbf, int n_harm, int n_rho, int taps, int n_cls,
                                  int block_rows, bool tc) {
  FillBucketPlan pl{};
  pl.ok = false;
  if (!(n_mbf == 1 || n_mbf == 2 || n_mbf == 4)) return pl;
  if (!(taps == 8 || taps == 12 || taps == 16)) return pl;
  if (n_el < 1 || n_rho < 2 * taps) return pl;
  int nb = 1;
  while ((1 << nb) < n_el) ++nb;
  if (nb > 24) return pl;
  // the tensor-core form: FP32, M = 4, 8 taps, one stencil cell per CTA
  pl.tc = tc && sizeof(T) == 4 && n_mbf == 4 && taps == 8 && fc_smem_bytes(n_harm) <= 227 * 1024;
  if (pl.tc) {
    pl.win = 1;
    pl.smem = fc_smem_bytes(n_harm);
  } else {
    const size_t row_bytes = (size_t)n_harm * n_mbf * n_mbf * sizeof(cpx<T>);
    // two CTAs per SM when the window stays useful, else one
    int win = (int)((110 * 1024) / row_bytes) - (taps - 1);
    if (win < 8) win = (int)((220 * 1024) / row_bytes) - (taps - 1);
    if (win < 4) return pl;
    win = std::min(win, 64);
    pl.win = win;
    pl.smem = (size_t)(win + taps - 1) * row_bytes;
  }
  pl.n_cells = n_rho - taps + (taps / 2 - 1) + 1;
  pl.nb_bits = nb;
  // waves of whole row blocks with at most 2^27 pairs (512 MB of codes); the
  // tensor-core form takes whole-wave blocks (more pairs per stencil cell)
  const size_t pair_cap = (size_t)1 << 27;
  int br = block_rows > 0 ? block_rows : (pl.tc ? n_el : 1024);
  br = std::min(br, n_el);
  br = std::min(br, 1 << std::min(30, 32 - nb));
  br = std::max(1, std::min<int>(br, (int)std::max<size_t>(1, pair_cap / (size_t)n_el)));
  pl.block_rows = br;
  int blocks_per_wave = (int)std::max<size_t>(1, pair_cap / ((size_t)br * n_el));
  int rows = std::min(n_el, blocks_per_wave * br);
  pl.rows_per_wave = rows;
  const int n_blocks = (rows + br - 1) / br;
  pl.n_keys_max = (size_t)n_blocks * n_cls * pl.n_cells;
  if (pl.n_keys_max > (size_t)1024 * kScanSeg) return pl;   // the key scan handles 16.7 M keys
  pl.scratch = ((size_t)n_el * sizeof(float4) + 255) / 256 * 256 +
               (pl.n_keys_max * sizeof(unsigned) + 255) / 256 * 256 +
               ((pl.n_keys_max + 1) * sizeof(unsigned) + 255) / 256 * 256 + 1024 * sizeof(unsigned) +
               (size_t)rows * n_el * sizeof(unsigned) + 256;
  pl.ok = true;
  return pl;
}

template <class T>
cudaError_t launch_fill_bucketed(const FillArgs<T, T>& a, const FillBucketPlan& pl, void* scratch,
                                 cudaStream_t s) {
  if (!pl.ok) return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == 4) {
    if (pl.tc) return run_fill_tc(a, pl, scratch, s);
  }
  switch (a.n_mbf) {
    case 1: return run_taps<T, 1>(a, pl, scratch, s);
    case 2: return run_taps<T, 2>(a, pl, scratch, s);
    case 4: return run_taps<T, 4>(a, pl, scratch, s);
    default: return cudaErrorInvalidValue;
  }
}

template <class T>
cudaError_t launch_fill_adjoint_bucketed(const FillArgs<T, T>& a, const FillAdjointArgs<T>& ad,
                                         const FillBucketPlan& pl, void* scratch, cudaStream_t s) {
  if (!pl.ok) return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == 4) {
    if (pl.tc) return run_adjoint_tc(a, ad, pl, scratch, s);
  }
  switch (a.n_mbf) {
    case 1: return adjoint_taps<T, 1>(a, ad, pl, scratch, s);
    case 2: return adjoint_taps<T, 2>(a, ad, pl, scratch, s);
    case 4: return adjoint_taps<T, 4>(a, ad, pl, scratch, s);
    default: return cudaErrorInvalidValue;
  }
}

template FillBucketPlan plan_fill_bucketed<float>(int, int, int, int, int, int, int, bool);
template FillBucketPlan plan_fill_bucketed<double>(int, int, int, int, int, int, int, bool);
template cudaError_t launch_fill_bucketed<float>(const FillArgs<float, float>&, const FillBucketPlan&, void*,
                                                 cudaStream_t);
template cudaError_t launch_fill_bucketed<double>(const FillArgs<double, double>&, const FillBucketPlan&,
                                                  void*, cudaStream_t);

template cudaError_t launch_fill_adjoint_bucketed<float>(const FillArgs<float, float>&,
                                                         const FillAdjointArgs<float>&, const FillBucketPlan&,
                                                         void*, cudaStream_t);
template cudaError_t launch_fill_adjoint_bucketed<double>(const FillArgs<double, double>&,
                                                          const FillAdjointArgs<double>&,
                                                          const FillBucketPlan&, void*, cudaStream_t);

}  // namespace cfft
