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
//
// One CTA per test element m (4 rows of the matrix): it counting-sorts the
// basis elements n of its row by (class, rho bin) in shared memory, then its
// threads take the pairs in that order.  The 32 lanes of a warp therefore hold
// nearly equal rho: their table stencils overlap, so each table load of the
// warp touches one or two cache lines instead of 32, while every store stays
// inside the CTA's 4 rows of the matrix (one page range, not the whole
// matrix).  Each thread writes its M x M block as M runs of M entries.
#include <algorithm>
#include <type_traits>

#include "cfft_common.cuh"

namespace cfft {

namespace {

constexpr int kMaxM = 8;
constexpr int kMaxTaps = 16;
constexpr int kRowThreads = 256;
constexpr int kRowsPerBin = 2;

struct RowSort {
  unsigned* hist;     // [n_bins] counts, then cursors
  unsigned short* list;  // [n_el] basis elements in (class, rho) order
  int n_bins;
};

// class of (test m, basis n) with rotations in {0, 1}
__device__ __forceinline__ int pair_class(const int* rot, int n_cls, int m, int n) {
  return (n_cls == 1 || rot == nullptr) ? 0 : 2 * (rot[m] != 0) + (rot[n] != 0);
}

// sort the basis elements of row m by (class, rho bin); result in rs.list
__device__ void sort_row(const double* pos, const int* rot, int n_el, int n_cls, int m,
                         float inv_bin, int bins_per_class, RowSort rs) {
  const int tid = threadIdx.x;
  for (int b = tid; b < rs.n_bins; b += blockDim.x) rs.hist[b] = 0;
  __syncthreads();
  const float xm = (float)pos[2 * m], ym = (float)pos[2 * m + 1];
  auto key_of = [&](int n) {
    float dx = xm - (float)pos[2 * n], dy = ym - (float)pos[2 * n + 1];
    int bin = (int)(sqrtf(dx * dx + dy * dy) * inv_bin);
    bin = min(max(bin, 0), bins_per_class - 1);
    int c = (n_cls == 4 && rot) ? (rot[n] != 0) : 0;
    return c * bins_per_class + bin;
  };
  for (int n = tid; n < n_el; n += blockDim.x) atomicAdd(&rs.hist[key_of(n)], 1u);
  __syncthreads();
  // exclusive scan of the histogram: each thread a contiguous run, then across threads
  __shared__ unsigned part[kRowThreads];
  const int per = (rs.n_bins + blockDim.x - 1) / blockDim.x;
  const int b0 = tid * per, b1 = min(b0 + per, rs.n_bins);
  unsigned sum = 0;
  for (int b = b0; b < b1; ++b) sum += rs.hist[b];
  part[tid] = sum;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    unsigned v = tid >= off ? part[tid - off] : 0u;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  unsigned run = part[tid] - sum;
  for (int b = b0; b < b1; ++b) {
    unsigned c = rs.hist[b];
    rs.hist[b] = run;
    run += c;
  }
  __syncthreads();
  for (int n = tid; n < n_el; n += blockDim.x) {
    unsigned slot = atomicAdd(&rs.hist[key_of(n)], 1u);
    rs.list[slot] = (unsigned short)n;
  }
  __syncthreads();
}

// Lagrange weights (and optionally their x-derivatives) at x, nodes 0..taps-1
template <class T, bool SLOPE>
__device__ __forceinline__ void lagrange(T x, int taps, T* w, T* dw) {
  T pre[kMaxTaps], dpre[kMaxTaps];
  T p = (T)1, dp = (T)0;
#pragma unroll
  for (int t = 0; t < kMaxTaps; ++t)
    if (t < taps) {
      pre[t] = p;
      if (SLOPE) {
        dpre[t] = dp;
        dp = dp * (x - (T)t) + p;
      }
      p *= (x - (T)t);
    }
  T sf = (T)1, dsf = (T)0;
#pragma unroll
  for (int t = kMaxTaps - 1; t >= 0; --t)
    if (t < taps) {
      // 1 / prod_{s != t} (t - s) = (-1)^(taps-1-t) / (t! (taps-1-t)!)
      T den = (T)1;
      for (int s2 = 1; s2 <= t; ++s2) den *= (T)s2;
      for (int s2 = 1; s2 <= taps - 1 - t; ++s2) den *= (T)s2;
      if ((taps - 1 - t) & 1) den = -den;
      w[t] = pre[t] * sf / den;
      if (SLOPE) {
        dw[t] = (dpre[t] * sf + pre[t] * dsf) / den;
        dsf = dsf * (x - (T)t) + sf;
      }
      sf *= (x - (T)t);
    }
}

struct PairGeom {
  double dx, dy, rho;
  int i0;     // first stencil row (may be negative: parity rows)
  double x;   // stencil coordinate of rho, u - i0
};

__device__ __forceinline__ PairGeom pair_geom(const double* pos, int m, int n, double inv_d_rho,
                                              int taps, int n_rho) {
  PairGeom g;
  g.dx = pos[2 * m] - pos[2 * n];
  g.dy = pos[2 * m + 1] - pos[2 * n + 1];
  g.rho = sqrt(g.dx * g.dx + g.dy * g.dy);
  const double u = g.rho * inv_d_rho;
  int i0 = (int)floor(u) - (taps / 2 - 1);
  if (i0 + taps > n_rho) i0 = n_rho - taps;
  g.i0 = i0;
  g.x = u - (double)i0;
  return g;
}

template <class T, class TO>
__global__ void __launch_bounds__(kRowThreads, 2) fill_row_kernel(FillArgs<T, TO> a, float inv_bin,
                                                               int bins_per_class) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = blockIdx.x;
  RowSort rs;
  rs.n_bins = bins_per_class * (a.n_cls == 4 ? 2 : 1);
  rs.hist = reinterpret_cast<unsigned*>(smem_raw);
  rs.list = reinterpret_cast<unsigned short*>(rs.hist + rs.n_bins);
  sort_row(a.pos, a.rot, a.n_el, a.n_cls, m, inv_bin, bins_per_class, rs);
  const int M = a.n_mbf;
  const int pairs = M * M;
  for (int idx = threadIdx.x; idx < a.n_el; idx += blockDim.x) {
    const int n = rs.list[idx];
    const PairGeom g = pair_geom(a.pos, m, n, a.inv_d_rho, a.taps, a.n_rho);
    cpx<TO>* zrow = a.z + (size_t)m * M * a.ld + (size_t)n * M;
    if (!(g.rho <= a.rho_max * (1.0 + 1e-12))) {
      atomicOr(a.err, 1);
      for (int ia = 0; ia < M; ++ia)
        for (int ib = 0; ib < M; ++ib) zrow[(size_t)ia * a.ld + ib] = mk((TO)0, (TO)0);
      continue;
    }
    const cpx<T> e1 = g.rho > 0.0 ? mk((T)(g.dx / g.rho), (T)(g.dy / g.rho)) : mk((T)1, (T)0);
    const int cls = pair_class(a.rot, a.n_cls, m, n);
    T w[kMaxTaps];
    lagrange<T, false>((T)g.x, a.taps, w, nullptr);
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
        const bool odd = ((qi - a.q_max) & 1) != 0;
#pragma unroll
        for (int ib = 0; ib < kMaxM; ++ib) {
          if (ib < M) {
            const cpx<T>* row = tab + ((size_t)(ia * M + ib) * a.n_harm + qi) * a.n_rho;
            cpx<T> v = mk((T)0, (T)0);
#pragma unroll
            for (int t = 0; t < kMaxTaps; ++t) {
              if (t < a.taps) {
                int r = g.i0 + t;
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
}

// Adjoint of the fill: for dL = Re sum conj(G) dZ, accumulate dL/d(positions)
// through d rho and d phi of every element pair, and dL/d(eps_r, h) through
// the derivative tables (same interpolation, contour held fixed).
template <class T, class TG>
__global__ void __launch_bounds__(kRowThreads) fill_backward_row_kernel(FillBackArgs<T, TG> b,
                                                                        float inv_bin,
                                                                        int bins_per_class) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FillArgs<T, float>& a = b.f;
  const int m = blockIdx.x;
  RowSort rs;
  rs.n_bins = bins_per_class * (a.n_cls == 4 ? 2 : 1);
  rs.hist = reinterpret_cast<unsigned*>(smem_raw);
  rs.list = reinterpret_cast<unsigned short*>(rs.hist + rs.n_bins);
  sort_row(a.pos, a.rot, a.n_el, a.n_cls, m, inv_bin, bins_per_class, rs);
  const int M = a.n_mbf;
  const int pairs = M * M;
  double gm_x = 0.0, gm_y = 0.0, g_eps = 0.0, g_h = 0.0;
  for (int idx = threadIdx.x; idx < a.n_el; idx += blockDim.x) {
    const int n = rs.list[idx];
    const PairGeom g = pair_geom(a.pos, m, n, a.inv_d_rho, a.taps, a.n_rho);
    if (!(g.rho <= a.rho_max * (1.0 + 1e-12))) {
      atomicOr(a.err, 1);
      continue;
    }
    const double cph = g.rho > 0.0 ? g.dx / g.rho : 1.0, sph = g.rho > 0.0 ? g.dy / g.rho : 0.0;
    const cpx<T> e1 = mk((T)cph, (T)sph);
    const int cls = pair_class(a.rot, a.n_cls, m, n);
    T w[kMaxTaps], dw[kMaxTaps];
    lagrange<T, true>((T)g.x, a.taps, w, dw);
    const size_t cls_off = (size_t)cls * pairs * a.n_harm * a.n_rho;
    const cpx<T>* tab = a.table + cls_off;
    const cpx<T>* te = b.dtab_eps ? b.dtab_eps + cls_off : nullptr;
    const cpx<T>* th = b.dtab_h ? b.dtab_h + cls_off : nullptr;
    cpx<T> zq = mk((T)1, (T)0);
    for (int k = 0; k < a.q_max; ++k) zq = zq * conj(e1);
    double s_rho = 0.0, s_phi = 0.0;
    for (int ia = 0; ia < M; ++ia) {
      cpx<T> gz[kMaxM];
#pragma unroll
      for (int ib = 0; ib < kMaxM; ++ib)
        if (ib < M) {
          cpx<TG> gv = b.grad[(size_t)(m * M + ia) * b.ld_g + (size_t)n * M + ib];
          gz[ib] = mk((T)gv.re, (T)gv.im);
        }
      T acc_rho = (T)0, acc_phi = (T)0, acc_e = (T)0, acc_h = (T)0;
      cpx<T> ph = zq;
      for (int qi = 0; qi < a.n_harm; ++qi) {
        const int q = qi - a.q_max;
        const bool odd = (q & 1) != 0;
#pragma unroll
        for (int ib = 0; ib < kMaxM; ++ib) {
          if (ib < M) {
            const size_t roff = ((size_t)(ia * M + ib) * a.n_harm + qi) * a.n_rho;
            cpx<T> v = mk((T)0, (T)0), dv = mk((T)0, (T)0), ve = mk((T)0, (T)0),
                   vh = mk((T)0, (T)0);
#pragma unroll
            for (int t = 0; t < kMaxTaps; ++t) {
              if (t < a.taps) {
                int r = g.i0 + t;
                T wt = w[t], dwt = dw[t];
                if (r < 0) {
                  r = -r;
                  if (odd) {
                    wt = -wt;
                    dwt = -dwt;
                  }
                }
                const cpx<T> z = tab[roff + r];
                v = v + wt * z;
                dv = dv + dwt * z;
                if (te) {
                  ve = ve + wt * te[roff + r];
                  vh = vh + wt * th[roff + r];
                }
              }
            }
            // Re(conj(g) ph X) for the four derivatives
            const cpx<T> cg = conj(gz[ib]) * ph;
            acc_rho += cg.re * dv.re - cg.im * dv.im;
            // d/dphi of ph v is i q ph v: Re(cg i q v) = -q Im(cg v)
            acc_phi -= (T)q * (cg.re * v.im + cg.im * v.re);
            acc_e += cg.re * ve.re - cg.im * ve.im;
            acc_h += cg.re * vh.re - cg.im * vh.im;
          }
        }
        ph = ph * e1;
      }
      s_rho += (double)acc_rho * a.inv_d_rho;  // d/d rho = (1 / d_rho) d/dx
      s_phi += (double)acc_phi;
      g_eps += (double)acc_e;
      g_h += (double)acc_h;
    }
    if (m != n && b.grad_pos) {
      // rho and phi as functions of Delta = r_m - r_n
      const double gx = s_rho * cph - s_phi * sph / g.rho;
      const double gy = s_rho * sph + s_phi * cph / g.rho;
      gm_x += gx;
      gm_y += gy;
      atomicAdd(&b.grad_pos[2 * n], -gx);
      atomicAdd(&b.grad_pos[2 * n + 1], -gy);
    }
  }
  // block reduction of the row's own position gradient and the substrate terms
  __shared__ double red[4][kRowThreads / 32];
  double vals[4] = {gm_x, gm_y, g_eps, g_h};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double v = vals[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double v = 0.0;
    for (int w2 = 0; w2 < (int)blockDim.x / 32; ++w2) v += red[threadIdx.x][w2];
    if (threadIdx.x < 2) {
      if (b.grad_pos) atomicAdd(&b.grad_pos[2 * m + threadIdx.x], v);
    } else if (b.grad_theta && b.dtab_eps) {
      atomicAdd(&b.grad_theta[threadIdx.x - 2], v);
    }
  }
}

size_t row_smem(int n_el, int n_bins) {
  return (size_t)n_bins * sizeof(unsigned) + (size_t)n_el * sizeof(unsigned short) + 16;
}

// rho bins of the per-row sort: kRowsPerBin table rows each, at most 8192 per class
void row_bins(int n_rho, double inv_d_rho, float* inv_bin, int* bins_per_class) {
  int rows = kRowsPerBin;
  while ((n_rho + rows - 1) / rows > 8192) rows *= 2;
  *bins_per_class = (n_rho + rows - 1) / rows;
  *inv_bin = (float)(inv_d_rho / rows);
}

}  // namespace

template <class T, class TO>
cudaError_t launch_fill(const FillArgs<T, TO>& a, const FillBucketPlan& plan, void* scratch, cudaStream_t s) {
  if constexpr (std::is_same<T, TO>::value) {
    if (plan.ok) return launch_fill_bucketed<T>(a, plan, scratch, s);
  }
  if (a.n_mbf > kMaxM || a.taps > kMaxTaps || a.taps < 2) return cudaErrorInvalidValue;
  float inv_bin;
  int bpc;
  row_bins(a.n_rho, a.inv_d_rho, &inv_bin, &bpc);
  const size_t smem = row_smem(a.n_el, bpc * (a.n_cls == 4 ? 2 : 1));
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fill_row_kernel<T, TO>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fill_row_kernel<T, TO><<<a.n_el, kRowThreads, smem, s>>>(a, inv_bin, bpc);
  return cudaGetLastError();
}

template <class T, class TG>
cudaError_t launch_fill_backward(const FillBackArgs<T, TG>& b, cudaStream_t s) {
  const FillArgs<T, float>& a = b.f;
  if (a.n_mbf > kMaxM || a.taps > kMaxTaps || a.taps < 2) return cudaErrorInvalidValue;
  float inv_bin;
  int bpc;
  row_bins(a.n_rho, a.inv_d_rho, &inv_bin, &bpc);
  const size_t smem = row_smem(a.n_el, bpc * (a.n_cls == 4 ? 2 : 1));
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fill_backward_row_kernel<T, TG>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fill_backward_row_kernel<T, TG><<<a.n_el, kRowThreads, smem, s>>>(b, inv_bin, bpc);
  return cudaGetLastError();
}

namespace {

// dL/dZ' of the array objective L = sum_i |r_i|^2, r = Z' v - t: with
// dL = 2 Re sum_i conj(r_i) sum_j dZ'_ij v_j = Re sum_ij conj(G_ij) dZ'_ij,
// G_ij = 2 r_i conj(v_j) (row-major n x n, one grid-stride pass, coalesced stores)
template <class T>
__global__ void residual_outer_kernel(const cpx<T>* r, const cpx<T>* v, int n, cpx<T>* g) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n);
    const int j = (int)(e - (int64_t)i * n);
    const cpx<T> ri = r[i], vj = v[j];
    g[e] = mk((T)2 * (ri.re * vj.re + ri.im * vj.im), (T)2 * (ri.im * vj.re - ri.re * vj.im));
  }
}

}  // namespace

template <class T>
cudaError_t launch_residual_outer(const void* r, const void* v, int n, void* g, cudaStream_t s) {
  if (n < 1 || !r || !v || !g) return cudaErrorInvalidValue;
  const int64_t total = (int64_t)n * n;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((total + threads - 1) / threads, (int64_t)current_sm_count() * 16);
  residual_outer_kernel<T><<<(unsigned)blocks, threads, 0, s>>>(
      reinterpret_cast<const cpx<T>*>(r), reinterpret_cast<const cpx<T>*>(v), n, reinterpret_cast<cpx<T>*>(g));
  return cudaGetLastError();
}

namespace {

// A posteriori estimate of the fill's interpolation error on a table's rho grid.
// The Lagrange stencil of p taps at step d leaves the remainder
//   f(u) - L(u) = f^(p)(xi) / p! * prod_t (u - t) d^p,
// and the p-th difference of p + 1 consecutive table rows is d^p f^(p) at a
// point of their span, so for every window of p + 1 rows the error of the
// stencils there is about |nabla^p Z| * pi_max / p!, with pi_max the largest
// |prod_t (x - t)| over the stencil coordinates x that those stencils use
// (fac_c: the central interval of an interior stencil; fac_e: the last stencil,
// shifted inward at rho_max).  Rows below rho = 0 follow the parity
// Z_q(-rho) = (-1)^q Z_q(rho), as in the fill.  One block per table series
// (channel, class, pair, harmonic); out[series] = (max |Z|, max estimate of the
// interior stencils, estimate of the last stencil, 0).
template <class T>
__global__ void fill_estimate_kernel(const cpx<T>* table, int n_rho, int q_max, int n_harm,
                                     int taps, double fac_c, double fac_e, double4* out) {
  // arithmetic in the table's precision; squared magnitudes until the end
  const int64_t series = blockIdx.x;
  const cpx<T>* z = table + series * (int64_t)n_rho;
  const int q = (int)(series % n_harm) - q_max;
  const T par = (q & 1) ? (T)-1 : (T)1;
  T coef[kMaxTaps + 1];
  {
    // (-1)^(p-k) C(p, k)
    double c = 1.0;
#pragma unroll
    for (int k = 0; k <= kMaxTaps; ++k) {
      if (k <= taps) coef[k] = (T)(((taps - k) & 1) ? -c : c);
      c = c * (double)(taps - k) / (double)(k + 1);
    }
  }
  T zmax = 0, emax = 0, eedge = 0;
  for (int r = threadIdx.x; r < n_rho; r += blockDim.x) {
    const cpx<T> v = z[r];
    zmax = fmax(zmax, v.re * v.re + v.im * v.im);
  }
  const int j_lo = -(taps / 2 - 1), j_hi = n_rho - taps - 1;
  for (int j = j_lo + (int)threadIdx.x; j <= j_hi; j += blockDim.x) {
    T dr = 0, di = 0;
#pragma unroll
    for (int k = 0; k <= kMaxTaps; ++k) {
      if (k <= taps) {
        const int i = j + k;
        const cpx<T> v = z[i < 0 ? -i : i];
        const T s = (i < 0 ? par : (T)1) * coef[k];
        dr = fma(s, v.re, dr);
        di = fma(s, v.im, di);
      }
    }
    const T d2 = dr * dr + di * di;
    if (j == j_hi)
      eedge = d2;
    else
      emax = fmax(emax, d2);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    zmax = fmax(zmax, __shfl_xor_sync(0xffffffffu, zmax, off));
    emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, off));
    eedge = fmax(eedge, __shfl_xor_sync(0xffffffffu, eedge, off));
  }
  __shared__ double4 red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_double4(zmax, emax, eedge, 0.0);
  __syncthreads();
  if (threadIdx.x == 0) {
    double4 acc = make_double4(0.0, 0.0, 0.0, 0.0);
    for (int w = 0; w < (int)blockDim.x / 32; ++w) {
      acc.x = fmax(acc.x, red[w].x);
      acc.y = fmax(acc.y, red[w].y);
      acc.z = fmax(acc.z, red[w].z);
    }
    out[series] = make_double4(sqrt(acc.x), sqrt(acc.y) * fac_c, sqrt(acc.z) * fac_e, 0.0);
  }
}

}  // namespace

template <class T>
cudaError_t launch_fill_estimate(const void* table, int64_t n_series, int n_rho, int q_max, int taps,
                                 double fac_c, double fac_e, double4* out, cudaStream_t s) {
  if (n_series < 1 || n_series > 0x7fffffff || taps < 2 || taps > kMaxTaps || n_rho < taps + 1)
    return cudaErrorInvalidValue;
  fill_estimate_kernel<T><<<(unsigned)n_series, 256, 0, s>>>(
      reinterpret_cast<const cpx<T>*>(table), n_rho, q_max, 2 * q_max + 1, taps, fac_c, fac_e, out);
  return cudaGetLastError();
}

template cudaError_t launch_fill_estimate<float>(const void*, int64_t, int, int, int, double, double,
                                                 double4*, cudaStream_t);
template cudaError_t launch_fill_estimate<double>(const void*, int64_t, int, int, int, double, double,
                                                  double4*, cudaStream_t);

template cudaError_t launch_residual_outer<float>(const void*, const void*, int, void*, cudaStream_t);
template cudaError_t launch_residual_outer<double>(const void*, const void*, int, void*, cudaStream_t);

template cudaError_t launch_fill<float, float>(const FillArgs<float, float>&, const FillBucketPlan&, void*, cudaStream_t);
template cudaError_t launch_fill<float, double>(const FillArgs<float, double>&, const FillBucketPlan&, void*, cudaStream_t);
template cudaError_t launch_fill<double, double>(const FillArgs<double, double>&, const FillBucketPlan&, void*, cudaStream_t);
template cudaError_t launch_fill<double, float>(const FillArgs<double, float>&, const FillBucketPlan&, void*, cudaStream_t);
template cudaError_t launch_fill_backward<float, float>(const FillBackArgs<float, float>&, cudaStream_t);
template cudaError_t launch_fill_backward<float, double>(const FillBackArgs<float, double>&, cudaStream_t);
template cudaError_t launch_fill_backward<double, double>(const FillBackArgs<double, double>&, cudaStream_t);
template cudaError_t launch_fill_backward<double, float>(const FillBackArgs<double, float>&, cudaStream_t);

}  // namespace cfft
