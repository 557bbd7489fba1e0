// Fused contour integrand: MBF spectra (Eq. 11), the MBF kernel (Eq. 10) and
// its azimuthal harmonics, times the contour measure beta_c w_j (Eq. 8, 9).
//
// For node j of the contour and angle alpha_l = 2 pi l / N_alpha the
// wavevector is k = beta_c,j (cos alpha_l, sin alpha_l) (complex beta with real
// alpha is the analytic extension of Eq. 18).  Each element basis function is
// F_i(k) = exp(-i k.r_i) S_c(k) with S_c the closed-form transform of its
// shape class c (rooftop: a sinc^2(k_u a/2) sinc(k_v w/2); cosine strip:
// 2 pi L cos(k_x L/2)/(pi^2 - k_x^2 L^2) sinc(k_y W/2)); every supported shape
// is centro-symmetric, S_c(-k) = S_c(k).  The MBF spectra of Eq. 11 and the
// analytic continuation of the conjugated basis spectrum in Eq. 10 are
//   Mt_a(k) = sum_c S_c(k) d_c sum_{i in c} conj(Q_ia) exp(-i k.r_i)
//   Mb_b(k) = sum_c S_c(k) d_c sum_{i in c} Q_ib exp(+i k.r_i)
// (one sincos and one exp per basis: exp(+i k.r) = 1 / exp(-i k.r)).
// With G = P I - R k k^T (see k_contour.cu; R arrives premultiplied by beta_c^2)
// the kernel of Eq. 10 is
//   H_ab = P (Mt_a . Mb_b) - R beta_c^2 (u.Mt_a)(u.Mb_b),  u = (cos, sin)(alpha)
// and its harmonics H_ab,q(beta_j) = 1/N_alpha sum_l H_ab(j, l) exp(-i q alpha_l).
// An element rotated by 90 degrees has M^rot(alpha_l) = R90 M(alpha_{l - N/4}),
// an index shift on the same angular grid.  Output:
//   Y[cls][pair][q][j] = H_ab,q(beta_j) beta_c,j w_j
// which is the contour integrand of the one-dimensional transform in beta.
#include "cfft_common.cuh"
#include "shape_factor.cuh"

namespace cfft {

namespace {

constexpr int kThreads = 256;

// M is the MBF count padded to a compiled size (padding columns of Q are zero);
// a.n_mbf is the real count.  Pairs are processed pc at a time through hbuf.
template <class T, int M>
__device__ __forceinline__ void integrand_tile(const IntegrandArgs<T>& a, const int j0, int jt,
                                               int pc, unsigned char* smem_raw) {
  const int na = a.n_alpha;
  const int pts = jt * na;
  const int nh = 2 * a.q_max + 1;
  const int mr = a.n_mbf;
  const int n_pairs = mr * mr;
  // shared layout
  cpx<T>* spec = reinterpret_cast<cpx<T>*>(smem_raw);        // [pts][2 sides][M][2 comps]
  cpx<T>* hbuf = spec + (size_t)pts * 4 * M;                 // [pc][pts]
  cpx<T>* tw = hbuf + (size_t)pc * pts;                      // [na]
  cpx<T>* sq = tw + na;                                       // [n_basis][M]
  T* sx = reinterpret_cast<T*>(sq + (size_t)a.n_basis * M);   // [n_basis]
  T* sy = sx + a.n_basis;

  const int tid = threadIdx.x;
  for (int t = tid; t < na; t += kThreads) {
    T s, c;
    sincospi_((T)(-2.0 * (double)t / (double)na), &s, &c);
    tw[t] = mk(c, s);
  }
  for (int t = tid; t < a.n_basis * M; t += kThreads) sq[t] = a.q[t];
  for (int t = tid; t < a.n_basis; t += kThreads) {
    sx[t] = a.bx[t];
    sy[t] = a.by[t];
  }
  __syncthreads();

  // ---- phase 1: MBF spectra at every (j, l) of this block
  for (int p = tid; p < pts; p += kThreads) {
    int jj = p / na, l = p - jj * na;
    int j = j0 + jj;
    cpx<T> mt[2][M], mb[2][M];
#pragma unroll
    for (int d = 0; d < 2; ++d)
#pragma unroll
      for (int m = 0; m < M; ++m) {
        mt[d][m] = mk((T)0, (T)0);
        mb[d][m] = mk((T)0, (T)0);
      }
    if (j < a.n) {
      double2 b = a.beta_c[j];
      double sa, ca;
      sincospi(2.0 * (double)l / (double)na, &sa, &ca);
      cpx<T> kx = mk((T)(b.x * ca), (T)(b.y * ca));
      cpx<T> ky = mk((T)(b.x * sa), (T)(b.y * sa));
      for (int c = 0; c < a.n_shape; ++c) {
        const ShapeClass sc = a.shapes[c];
        cpx<T> accT[M], accB[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          accT[m] = mk((T)0, (T)0);
          accB[m] = mk((T)0, (T)0);
        }
        for (int i = sc.begin; i < sc.end; ++i) {
          T xi = sx[i], yi = sy[i];
          T theta = kx.re * xi + ky.re * yi;   // Re k.r
          T psi = kx.im * xi + ky.im * yi;     // Im k.r
          T sn, cs;
          sincos_(theta, &sn, &cs);
          T e = exp_(psi), ie = (T)1 / e;
          cpx<T> ph = mk(cs * e, -sn * e);     // exp(-i k.r)
          cpx<T> pb = mk(cs * ie, sn * ie);    // exp(+i k.r)
#pragma unroll
          for (int m = 0; m < M; ++m) {
            cpx<T> qv = sq[i * M + m];
            cmac_conj(accT[m], qv, ph);
            cmac(accB[m], qv, pb);
          }
        }
        cpx<T> sf = shape_factor<T>(sc, kx, ky);
        if (sc.dir == 0) {
#pragma unroll
          for (int m = 0; m < M; ++m) {
            cmac(mt[0][m], sf, accT[m]);
            cmac(mb[0][m], sf, accB[m]);
          }
        } else {
#pragma unroll
          for (int m = 0; m < M; ++m) {
            cmac(mt[1][m], sf, accT[m]);
            cmac(mb[1][m], sf, accB[m]);
          }
        }
      }
    }
    cpx<T>* o = spec + (size_t)p * 4 * M;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      o[m * 2 + 0] = mt[0][m];
      o[m * 2 + 1] = mt[1][m];
      o[2 * M + m * 2 + 0] = mb[0][m];
      o[2 * M + m * 2 + 1] = mb[1][m];
    }
  }
  __syncthreads();

  const int quarter = na / 4;
  for (int cls = 0; cls < a.n_cls; ++cls)
  for (int pair0 = 0; pair0 < n_pairs; pair0 += pc) {
    const int npc = min(pc, n_pairs - pair0);
    const bool rot_t = (cls == 2), rot_b = (cls == 1);
    // ---- phase 2: H_ab(j, l) for this rotation class and pair chunk
    for (int idx = tid; idx < npc * pts; idx += kThreads) {
      int pl = idx / pts, p = idx - pl * pts;
      int pair = pair0 + pl;
      int ia = pair / mr, ib = pair - ia * mr;
      int jj = p / na, l = p - jj * na;
      int j = j0 + jj;
      cpx<T> h = mk((T)0, (T)0);
      if (j < a.n) {
        int lt = rot_t ? (l - quarter + na) % na : l;
        int lb = rot_b ? (l - quarter + na) % na : l;
        const cpx<T>* st = spec + (size_t)(jj * na + lt) * 4 * M;
        const cpx<T>* sb = spec + (size_t)(jj * na + lb) * 4 * M + 2 * M;
        cpx<T> tx = st[ia * 2], ty = st[ia * 2 + 1];
        cpx<T> bx = sb[ib * 2], by = sb[ib * 2 + 1];
        if (rot_t) { cpx<T> t = tx; tx = mk(-ty.re, -ty.im); ty = t; }  // R90 (x,y) = (-y, x)
        if (rot_b) { cpx<T> t = bx; bx = mk(-by.re, -by.im); by = t; }
        T ua = tw[l].re;    // cos(alpha_l)
        T ub = -tw[l].im;   // sin(alpha_l)
        cpx<T> dot = tx * bx + ty * by;
        cpx<T> et = ua * tx + ub * ty;
        cpx<T> eb = ua * bx + ub * by;
        double2 gp = a.green_p[j], gr = a.green_r[j];   // P and R beta_c^2
        h = mk((T)gp.x, (T)gp.y) * dot - mk((T)gr.x, (T)gr.y) * (et * eb);
      }
      hbuf[(size_t)pl * pts + p] = h;
    }
    __syncthreads();
    // ---- phase 3: harmonics and contour measure
    const T inv_na = (T)1 / (T)na;
    for (int idx = tid; idx < npc * nh * jt; idx += kThreads) {
      int jj = idx % jt;
      int rest = idx / jt;
      int qi = rest % nh;
      int pl = rest / nh;
      int pair = pair0 + pl;
      int j = j0 + jj;
      if (j >= a.n) continue;
      int q = qi - a.q_max;
      int qm = ((q % na) + na) % na;
      const cpx<T>* hp = hbuf + (size_t)pl * pts + jj * na;
      cpx<T> acc = mk((T)0, (T)0);
      int e = 0;
      for (int l = 0; l < na; ++l) {
        cmac(acc, hp[l], tw[e]);
        e += qm;
        if (e >= na) e -= na;
      }
      double2 bw = a.bw[j];
      cpx<T> out = mk((T)bw.x, (T)bw.y) * (inv_na * acc);
      size_t series = ((size_t)cls * n_pairs + pair) * nh + qi;
      a.y[series * a.n + j] = out;
    }
    __syncthreads();
  }
}

template <class T, int M>
__global__ void __launch_bounds__(kThreads) integrand_kernel(IntegrandArgs<T> a, int jt, int pc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  integrand_tile<T, M>(a, blockIdx.x * jt, jt, pc, smem_raw);
}

// batched form: block b processes node tile map[b].y of item map[b].x
template <class T, int M>
__global__ void __launch_bounds__(kThreads) integrand_batch_kernel(const IntegrandArgs<T>* items,
                                                                   const int2* map, int jt, int pc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 bm = map[blockIdx.x];
  const IntegrandArgs<T> a = items[bm.x];
  integrand_tile<T, M>(a, bm.y, jt, pc, smem_raw);
}

// points per block: all n_alpha angles of jt contour nodes; pairs through hbuf in chunks
template <class T, int M>
bool integrand_shape(const IntegrandArgs<T>& a, int* jt_out, int* pc_out, size_t* smem_out) {
  const int n_pairs = a.n_mbf * a.n_mbf;
  const int fixed = a.n_alpha * (int)sizeof(cpx<T>) +
                    a.n_basis * (M * (int)sizeof(cpx<T>) + 2 * (int)sizeof(T)) + 64;
  const int budget = 200 * 1024;
  int pc = n_pairs < 16 ? n_pairs : 16;
  int jt = 0;
  for (;;) {
    int per_point = (4 * M + pc) * (int)sizeof(cpx<T>);
    jt = (budget - fixed) / (per_point * a.n_alpha);
    if (jt >= 1 || pc == 1) break;
    pc = (pc + 1) / 2;
  }
  if (jt < 1) return false;
  if (jt > 8) jt = 8;
  while (jt > 1 && jt * a.n_alpha > 4 * kThreads) --jt;
  *jt_out = jt;
  *pc_out = pc;
  *smem_out = (size_t)fixed + (size_t)(4 * M + pc) * sizeof(cpx<T>) * jt * a.n_alpha;
  return true;
}

template <class T, int M>
cudaError_t launch_m_batch(const IntegrandArgs<T>& shape_args, const IntegrandArgs<T>* items,
                           const int2* map, int n_blocks, int jt, cudaStream_t s) {
  int jt0, pc;
  size_t smem;
  if (!integrand_shape<T, M>(shape_args, &jt0, &pc, &smem)) return cudaErrorInvalidConfiguration;
  if (jt != jt0) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(integrand_batch_kernel<T, M>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  integrand_batch_kernel<T, M><<<n_blocks, kThreads, smem, s>>>(items, map, jt, pc);
  return cudaGetLastError();
}

template <class T, int M>
cudaError_t launch_m(const IntegrandArgs<T>& a, cudaStream_t s) {
  const int n_pairs = a.n_mbf * a.n_mbf;
  const int fixed = a.n_alpha * (int)sizeof(cpx<T>) +
                    a.n_basis * (M * (int)sizeof(cpx<T>) + 2 * (int)sizeof(T)) + 64;
  const int budget = 200 * 1024;
  // points per block: all n_alpha angles of jt contour nodes; pairs through hbuf in chunks
  int pc = n_pairs < 16 ? n_pairs : 16;
  int jt = 0;
  for (;;) {
    int per_point = (4 * M + pc) * (int)sizeof(cpx<T>);
    jt = (budget - fixed) / (per_point * a.n_alpha);
    if (jt >= 1 || pc == 1) break;
    pc = (pc + 1) / 2;
  }
  if (jt < 1) return cudaErrorInvalidConfiguration;
  if (jt > 8) jt = 8;
  while (jt > 1 && jt * a.n_alpha > 4 * kThreads) --jt;
  size_t smem = (size_t)fixed + (size_t)(4 * M + pc) * sizeof(cpx<T>) * jt * a.n_alpha;
  cudaError_t e = cudaFuncSetAttribute(integrand_kernel<T, M>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int blocks = (a.n + jt - 1) / jt;
  integrand_kernel<T, M><<<blocks, kThreads, smem, s>>>(a, jt, pc);
  return cudaGetLastError();
}

}  // namespace

// node-tile height used by the batched launch for this element and angle count
template <class T>
int integrand_tile_nodes(const IntegrandArgs<T>& a, int n_mbf_padded) {
  int jt = 0, pc = 0;
  size_t smem = 0;
  bool ok = false;
  switch (n_mbf_padded) {
    case 1: ok = integrand_shape<T, 1>(a, &jt, &pc, &smem); break;
    case 2: ok = integrand_shape<T, 2>(a, &jt, &pc, &smem); break;
    case 4: ok = integrand_shape<T, 4>(a, &jt, &pc, &smem); break;
    case 8: ok = integrand_shape<T, 8>(a, &jt, &pc, &smem); break;
    default: ok = false;
  }
  return ok ? jt : 0;
}

template <class T>
cudaError_t launch_integrand_batch(const IntegrandArgs<T>& shape_args, const IntegrandArgs<T>* items,
                                   const int2* map, int n_blocks, int jt, int n_mbf_padded,
                                   cudaStream_t s) {
  switch (n_mbf_padded) {
    case 1: return launch_m_batch<T, 1>(shape_args, items, map, n_blocks, jt, s);
    case 2: return launch_m_batch<T, 2>(shape_args, items, map, n_blocks, jt, s);
    case 4: return launch_m_batch<T, 4>(shape_args, items, map, n_blocks, jt, s);
    case 8: return launch_m_batch<T, 8>(shape_args, items, map, n_blocks, jt, s);
    default: return cudaErrorInvalidValue;
  }
}

template int integrand_tile_nodes<float>(const IntegrandArgs<float>&, int);
template int integrand_tile_nodes<double>(const IntegrandArgs<double>&, int);
template cudaError_t launch_integrand_batch<float>(const IntegrandArgs<float>&, const IntegrandArgs<float>*,
                                                   const int2*, int, int, int, cudaStream_t);
template cudaError_t launch_integrand_batch<double>(const IntegrandArgs<double>&,
                                                    const IntegrandArgs<double>*, const int2*, int,
                                                    int, int, cudaStream_t);

template <class T>
cudaError_t launch_integrand(const IntegrandArgs<T>& a, int n_mbf_padded, cudaStream_t s) {
  // n_mbf_padded is the column count of a.q (the real count is a.n_mbf)
  switch (n_mbf_padded) {
    case 1: return launch_m<T, 1>(a, s);
    case 2: return launch_m<T, 2>(a, s);
    case 4: return launch_m<T, 4>(a, s);
    case 8: return launch_m<T, 8>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_integrand<float>(const IntegrandArgs<float>&, int, cudaStream_t);
template cudaError_t launch_integrand<double>(const IntegrandArgs<double>&, int, cudaStream_t);

}  // namespace cfft
