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
// Geometry in the FP32-mixed mode runs in float-float arithmetic (positions
// split into a float head and tail; rho from a corrected float square root)
// instead of float64, whose throughput is a small fraction of float32 on this
// part; rho and the stencil coordinate keep about 44 significant bits, the
// same decisions as float64 except at exact cell-boundary ties, where either
// stencil is a valid one.
#include <algorithm>
#include <type_traits>

#include "cfft_common.cuh"

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
  bool bad;     // rho beyond the table
};

// stencil of pair (m, n), FP32-mixed: float-float geometry
template <class T, int TAPS>
__device__ __forceinline__ typename std::enable_if<sizeof(T) == 4, BGeom<T>>::type
bucket_geom(const FillArgs<T, T>& a, const BucketArgs& b, int m, int n) {
  constexpr int HALF = TAPS / 2 - 1;
  const float4 pm = b.ps[m], pn = b.ps[n];
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
  BGeom<T> g;
  const float top = (float)(a.n_rho - 1);
  g.bad = fl > top || (fl == top && f > 1e-6f) || !(r == r);
  const int fi = (int)fl;
  int i0 = fi - HALF;
  if (i0 + TAPS > a.n_rho) i0 = a.n_rho - TAPS;
  g.i0 = i0;
  g.x = (float)(fi - i0) + f;
  if (r > 0.f) {
    g.ex = __fdiv_rn(dxh, r);
    g.ey = __fdiv_rn(dyh, r);
  } else {
    g.ex = 1.f;
    g.ey = 0.f;
  }
  return g;
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

// exclusive scan of the key counts: off[k] = sum_{j<k} count[j], off[n] = total,
// and the counts are replaced by the scatter cursors (= off)
__global__ void __launch_bounds__(1024) bucket_scan_kernel(unsigned* cursor, unsigned* off, size_t n_keys) {
  __shared__ unsigned part[1024];
  const int tid = threadIdx.x;
  const size_t per = (n_keys + 1023) / 1024;
  const size_t k0 = (size_t)tid * per, k1 = min(k0 + per, n_keys);
  unsigned sum = 0;
  for (size_t k = k0; k < k1; ++k) sum += cursor[k];
  part[tid] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const unsigned v = tid >= o ? part[tid - o] : 0u;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  unsigned run = part[tid] - sum;
  for (size_t k = k0; k < k1; ++k) {
    const unsigned c = cursor[k];
    off[k] = run;
    cursor[k] = run;
    run += c;
  }
  if (tid == 1023) off[n_keys] = part[1023];
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
  {
    const cpx<T>* tab = a.table + (size_t)cls * P2 * a.n_harm * a.n_rho;
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
        v = tab[((size_t)ab * a.n_harm + qi) * a.n_rho + r];
        // Z_q(-rho) = (-1)^q Z_q(rho)
        if (neg && ((qi - a.q_max) & 1)) v = mk(-v.re, -v.im);
      }
      S[e] = v;
    }
  }
  __syncthreads();
  T den[TAPS];
#pragma unroll
  for (int t = 0; t < TAPS; ++t) {
    long long d = 1;
#pragma unroll
    for (int j = 0; j < TAPS; ++j)
      if (j != t) d *= (long long)(t - j);
    den[t] = (T)1 / (T)d;
  }
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
    // Lagrange weights at x on the nodes 0..TAPS-1
    T wt[TAPS];
    {
      T pre = (T)1;
#pragma unroll
      for (int t = 0; t < TAPS; ++t) {
        wt[t] = pre;
        pre *= (g.x - (T)t);
      }
      T suf = (T)1;
#pragma unroll
      for (int t = TAPS - 1; t >= 0; --t) {
        wt[t] *= suf * den[t];
        suf *= (g.x - (T)t);
      }
    }
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

template <class T, int M, int TAPS>
cudaError_t run_bucketed(const FillArgs<T, T>& a, const FillBucketPlan& pl, void* scratch, cudaStream_t s) {
  BucketArgs b{};
  unsigned char* sp = reinterpret_cast<unsigned char*>(scratch);
  b.ps = reinterpret_cast<const float4*>(sp);
  sp += ((size_t)a.n_el * sizeof(float4) + 255) / 256 * 256;
  b.cursor = reinterpret_cast<unsigned*>(sp);
  sp += (pl.n_keys_max * sizeof(unsigned) + 255) / 256 * 256;
  b.off = reinterpret_cast<unsigned*>(sp);
  sp += ((pl.n_keys_max + 1) * sizeof(unsigned) + 255) / 256 * 256;
  b.list = reinterpret_cast<unsigned*>(sp);
  b.br = pl.block_rows;
  b.nb_bits = pl.nb_bits;
  b.n_ck = a.n_cls;
  b.n_cells = pl.n_cells;
  b.win = pl.win;
  const double inv = a.inv_d_rho;
  b.ih = (float)inv;
  b.il = (float)(inv - (double)b.ih);
  b.vec_out = ((reinterpret_cast<uintptr_t>(a.z) & 15) == 0 &&
               ((size_t)a.ld * sizeof(cpx<T>)) % 16 == 0) ? 1 : 0;
  if (sizeof(T) == 4) {
    split_positions_kernel<<<(a.n_el + 255) / 256, 256, 0, s>>>(a.pos, a.n_el,
                                                              const_cast<float4*>(b.ps));
  }
  const size_t smem = pl.smem;
  cudaError_t e = cudaFuncSetAttribute(bucket_fill_kernel<T, M, TAPS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int n_windows = (pl.n_cells + pl.win - 1) / pl.win;
  for (int m0 = 0; m0 < a.n_el; m0 += pl.rows_per_wave) {
    b.m0 = m0;
    b.rows = min(pl.rows_per_wave, a.n_el - m0);
    const int n_blocks = (b.rows + b.br - 1) / b.br;
    const size_t n_keys = (size_t)n_blocks * b.n_ck * b.n_cells;
    e = cudaMemsetAsync(b.cursor, 0, n_keys * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    dim3 sg((a.n_el + kBThreads - 1) / kBThreads, min(b.rows, 65535));
    bucket_sort_kernel<T, TAPS, false><<<sg, kBThreads, 0, s>>>(a, b);
    bucket_scan_kernel<<<1, 1024, 0, s>>>(b.cursor, b.off, n_keys);
    bucket_sort_kernel<T, TAPS, true><<<sg, kBThreads, 0, s>>>(a, b);
    dim3 fg(n_windows, b.n_ck, n_blocks);
    bucket_fill_kernel<T, M, TAPS><<<fg, kBThreads, smem, s>>>(a, b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
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

}  // namespace

// Plan of the bucketed fill, or plan.ok = false when it does not apply (the
// per-row fill runs instead): M in {1, 2, 4}, taps in {8, 12, 16}, and a
// window of at least 4 stencil starts fitting in shared memory.
template <class T>
FillBucketPlan plan_fill_bucketed(int n_el, int n_mbf, int n_harm, int n_rho, int taps, int n_cls,
                                  int block_rows) {
  FillBucketPlan pl{};
  pl.ok = false;
  if (!(n_mbf == 1 || n_mbf == 2 || n_mbf == 4)) return pl;
  if (!(taps == 8 || taps == 12 || taps == 16)) return pl;
  if (n_el < 1 || n_rho < 2 * taps) return pl;
  int nb = 1;
  while ((1 << nb) < n_el) ++nb;
  if (nb > 24) return pl;
  const size_t row_bytes = (size_t)n_harm * n_mbf * n_mbf * sizeof(cpx<T>);
  // two CTAs per SM when the window stays useful, else one
  int win = (int)((110 * 1024) / row_bytes) - (taps - 1);
  if (win < 8) win = (int)((220 * 1024) / row_bytes) - (taps - 1);
  if (win < 4) return pl;
  win = std::min(win, 64);
  pl.win = win;
  pl.smem = (size_t)(win + taps - 1) * row_bytes;
  pl.n_cells = n_rho - taps + (taps / 2 - 1) + 1;
  pl.nb_bits = nb;
  // waves of whole row blocks with at most 2^27 pairs (512 MB of codes)
  const size_t pair_cap = (size_t)1 << 27;
  int br = block_rows > 0 ? block_rows : 1024;
  br = std::min(br, n_el);
  br = std::min(br, 1 << std::min(30, 32 - nb));
  br = std::max(1, std::min<int>(br, (int)std::max<size_t>(1, pair_cap / (size_t)n_el)));
  pl.block_rows = br;
  int blocks_per_wave = (int)std::max<size_t>(1, pair_cap / ((size_t)br * n_el));
  int rows = std::min(n_el, blocks_per_wave * br);
  pl.rows_per_wave = rows;
  const int n_blocks = (rows + br - 1) / br;
  pl.n_keys_max = (size_t)n_blocks * n_cls * pl.n_cells;
  pl.scratch = ((size_t)n_el * sizeof(float4) + 255) / 256 * 256 +
               (pl.n_keys_max * sizeof(unsigned) + 255) / 256 * 256 +
               ((pl.n_keys_max + 1) * sizeof(unsigned) + 255) / 256 * 256 +
               (size_t)rows * n_el * sizeof(unsigned) + 256;
  pl.ok = true;
  return pl;
}

template <class T>
cudaError_t launch_fill_bucketed(const FillArgs<T, T>& a, const FillBucketPlan& pl, void* scratch,
                                 cudaStream_t s) {
  if (!pl.ok) return cudaErrorInvalidValue;
  switch (a.n_mbf) {
    case 1: return run_taps<T, 1>(a, pl, scratch, s);
    case 2: return run_taps<T, 2>(a, pl, scratch, s);
    case 4: return run_taps<T, 4>(a, pl, scratch, s);
    default: return cudaErrorInvalidValue;
  }
}

template FillBucketPlan plan_fill_bucketed<float>(int, int, int, int, int, int, int);
template FillBucketPlan plan_fill_bucketed<double>(int, int, int, int, int, int, int);
template cudaError_t launch_fill_bucketed<float>(const FillArgs<float, float>&, const FillBucketPlan&, void*,
                                                 cudaStream_t);
template cudaError_t launch_fill_bucketed<double>(const FillArgs<double, double>&, const FillBucketPlan&,
                                                  void*, cudaStream_t);

}  // namespace cfft
