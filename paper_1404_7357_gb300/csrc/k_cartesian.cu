// The paper's own 2-D Cartesian C-FFT (Section III-B-2 and III-B-3, Eq. 21-24,
// Appendix I), as a second tabulation beside the harmonic one.
//
// On the real grid kx, ky = -k_m + n dk (n < N, dk = 2 k_m / N; Appendix I) the
// contour of Eq. 8 enters through the extension k (1 + i gamma), gamma =
// beta_I(beta_R) / beta_R (Eq. 20): per sample the kernel of Eq. 10 at that
// complex wavevector times the Jacobian (1 + i d beta_I / d beta_R)(1 + i gamma)
// gives I_M (Eq. 21); samples outside |k| <= k_m (the polar integral's limit)
// are zero.  The contour factor exp(gamma k.Delta) is expanded in Taylor
// monomials (Eq. 22): Z' = sum_{a, b} dx^a dy^b / (a! b!) F_ab with F_ab the 2-D
// Fourier sum of (gamma kx)^a (gamma ky)^b I_M (Eq. 23-24).  Each F_ab is one
// FFT2: the N x N samples, times (-1)^(n1 + n2) (Appendix I), sit in the middle
// of a 2N x 2N zero grid (the Whittaker-Shannon refinement that halves the
// table's step), and the output is multiplied by (-1)^(k1 + k2) dk^2 / (4 pi^2)
// on the lattice dx = -x_m + k1 pi / (2 k_m).
//
// Kernels: the spectrum (Green's function in float64; MBF spectra at the complex
// wavevector), per monomial the padded input, a length-2N Stockham FFT per row
// in shared memory, a tiled transpose, the same FFT again, and a tiled
// accumulation into the table (which also undoes the transpose).  The fill
// interpolates the table with three-point Lagrange stencils in x and y.
#include <algorithm>
#include <cmath>

#include "cfft_common.cuh"
#include "green_ext.cuh"
#include "shape_factor.cuh"

namespace cfft {

namespace {

constexpr double kEta0c = 376.730313668;   // free-space wave impedance, ohm
constexpr int kCartMaxM = 8;

// grounded-slab Green's function G = P I - R k k^T at the complex radial wavenumber
// beta_c (the TE/TM denominators and branches as in the contour kernel); returns P and
// R beta_c^2
__device__ void slab_green(cpx<double> bc, double eps_r, double hs, double k0, cpx<double>* p,
                           cpx<double>* rb2) {
  const cpx<double> b2 = bc * bc;
  const double k02 = k0 * k0;
  const cpx<double> k1 = csqrt_(mk(eps_r * k02 - b2.re, -b2.im));
  cpx<double> arg2 = mk(b2.re - k02, b2.im);
  if (arg2.im == 0.0) arg2.im = 0.0;   // +0: real beta < k0 gives k2 > 0 (outgoing)
  const cpx<double> r2 = csqrt_(arg2);
  const cpx<double> k2 = mk(r2.im, -r2.re);   // -j sqrt(.): Im k2 <= 0
  cpx<double> sn, cs;
  csincos(mk(k1.re * hs, k1.im * hs), &sn, &cs);
  const cpx<double> j1 = mk(0.0, 1.0);
  const cpx<double> te = k1 * cs + j1 * (k2 * sn);
  const cpx<double> tm = eps_r * (k2 * cs) + j1 * (k1 * sn);
  const cpx<double> cfac = cdiv(mk(0.0, -kEta0c / k0) * sn, te * tm);
  *p = cfac * ((eps_r * k02) * (k2 * cs) + j1 * (k02 * (k1 * sn)));
  *rb2 = cfac * (k2 * cs + j1 * (k1 * sn)) * b2;
}

// I_M (times the Appendix I sign) of every MBF pair at every sample, and gamma kx, gamma ky
template <class T>
__global__ void cart_spectrum_kernel(CartArgs<T> a, cpx<T>* im, T* gx, T* gy) {
  const int64_t nn = (int64_t)a.n * a.n;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nn) return;
  const int n1 = (int)(e / a.n), n2 = (int)(e % a.n);
  const int pairs = a.n_mbf * a.n_mbf;
  const double kx = -a.k_max + n1 * a.dk, ky = -a.k_max + n2 * a.dk;
  const double br = hypot(kx, ky);
  if (br > a.k_max) {
    for (int pr = 0; pr < pairs; ++pr) im[pr * nn + e] = mk((T)0, (T)0);
    gx[e] = (T)0;
    gy[e] = (T)0;
    return;
  }
  double bi = 0.0, slope = 0.0;
  if (br < a.beta_p) {
    const double ip2 = 1.0 / (a.beta_p * a.beta_p);
    bi = 4.0 * a.height * br * (a.beta_p - br) * ip2;
    slope = 4.0 * a.height * (a.beta_p - 2.0 * br) * ip2;
  }
  const double gamma = br > 0.0 ? bi / br : 4.0 * a.height / a.beta_p;
  // gamma k / H: at most beta_I / H <= 1 (H moves to the spatial factor, as (H dx)^a)
  const double ih = a.height > 0.0 ? 1.0 / a.height : 0.0;
  gx[e] = (T)(gamma * kx * ih);
  gy[e] = (T)(gamma * ky * ih);
  cpx<double> p, rb2;
  slab_green(mk(br, bi), a.eps_r, a.hs, a.k0, &p, &rb2);
  if (a.extract) {
    const GreenExt ge = ext_green(mk(br, bi), a.eps_eff, 0.0, a.hs, a.k0, false);
    p = p - ge.p;
    rb2 = rb2 - ge.rb2;
  }
  const double ux = br > 0.0 ? kx / br : 1.0, uy = br > 0.0 ? ky / br : 0.0;
  // MBF spectra at k_c = k (1 + i gamma): both sides, x and y components
  const cpx<T> kcx = mk((T)kx, (T)(gamma * kx)), kcy = mk((T)ky, (T)(gamma * ky));
  cpx<T> mt[2][kCartMaxM], mb[2][kCartMaxM];
  for (int d = 0; d < 2; ++d)
    for (int m = 0; m < kCartMaxM; ++m) {
      mt[d][m] = mk((T)0, (T)0);
      mb[d][m] = mk((T)0, (T)0);
    }
  for (int c = 0; c < a.n_shape; ++c) {
    const ShapeClass sc = a.shapes[c];
    cpx<T> acct[kCartMaxM], accb[kCartMaxM];
    for (int m = 0; m < kCartMaxM; ++m) {
      acct[m] = mk((T)0, (T)0);
      accb[m] = mk((T)0, (T)0);
    }
    for (int i = sc.begin; i < sc.end; ++i) {
      const T xi = a.bx[i], yi = a.by[i];
      const T theta = kcx.re * xi + kcy.re * yi, psi = kcx.im * xi + kcy.im * yi;
      T sn, cs;
      sincos_(theta, &sn, &cs);
      const T ex = exp_(psi), iex = (T)1 / ex;
      const cpx<T> ph = mk(cs * ex, -sn * ex);    // exp(-i k_c.r)
      const cpx<T> pb = mk(cs * iex, sn * iex);   // exp(+i k_c.r)
      for (int m = 0; m < a.n_mbf; ++m) {
        const cpx<T> qv = a.q[(size_t)i * a.q_stride + m];
        cmac_conj(acct[m], qv, ph);
        cmac(accb[m], qv, pb);
      }
    }
    const cpx<T> sf = shape_factor<T>(sc, kcx, kcy);
    for (int m = 0; m < a.n_mbf; ++m) {
      mt[sc.dir][m] = mt[sc.dir][m] + sf * acct[m];
      mb[sc.dir][m] = mb[sc.dir][m] + sf * accb[m];
    }
  }
  // Jacobian (1 + i slope)(1 + i gamma) and the Appendix I input sign (-1)^(n1 + n2)
  cpx<double> jac = mk(1.0, slope) * mk(1.0, gamma);
  if ((n1 + n2) & 1) jac = mk(-jac.re, -jac.im);
  for (int ia = 0; ia < a.n_mbf; ++ia)
    for (int ib = 0; ib < a.n_mbf; ++ib) {
      const cpx<double> tx = ccast<double>(mt[0][ia]), ty = ccast<double>(mt[1][ia]);
      const cpx<double> bx = ccast<double>(mb[0][ib]), by = ccast<double>(mb[1][ib]);
      const cpx<double> dot = tx * bx + ty * by;
      const cpx<double> ut = ux * tx + uy * ty, ub = ux * bx + uy * by;
      const cpx<double> h = p * dot - rb2 * (ut * ub);
      im[(ia * a.n_mbf + ib) * nn + e] = ccast<T>(jac * h);
    }
}

// padded input of monomial (a, b): the N x N samples times (gamma kx / H)^a (gamma ky / H)^b
// in the middle of the 2N x 2N grid, zero elsewhere
template <class T>
__global__ void cart_monomial_kernel(const cpx<T>* im, const T* gx, const T* gy, int n, int pa, int pb,
                                     int pairs, cpx<T>* out) {
  const int p = 2 * n, off = n / 2;
  const int64_t pp = (int64_t)p * p, total = pp * pairs;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int pr = (int)(e / pp);
    const int64_t r = e - pr * pp;
    const int i = (int)(r / p) - off, j = (int)(r % p) - off;
    cpx<T> v = mk((T)0, (T)0);
    if (i >= 0 && i < n && j >= 0 && j < n) {
      const int64_t s = (int64_t)i * n + j;
      T f = (T)1;
      const T x = gx[s], y = gy[s];
      for (int t = 0; t < pa; ++t) f *= x;
      for (int t = 0; t < pb; ++t) f *= y;
      v = f * im[(int64_t)pr * n * n + s];
    }
    out[e] = v;
  }
}

// in-place length-L FFT (exp(-2 pi i n k / L)) of each contiguous line: radix-2 Stockham
// in shared memory (ping-pong), natural order in and out
template <class T>
__global__ void line_fft_kernel(cpx<T>* data, int len) {
  extern __shared__ __align__(16) unsigned char sm[];
  cpx<T>* x = reinterpret_cast<cpx<T>*>(sm);
  cpx<T>* y = x + len;
  cpx<T>* line = data + (int64_t)blockIdx.x * len;
  const int half = len / 2;
  for (int i = threadIdx.x; i < len; i += blockDim.x) x[i] = line[i];
  __syncthreads();
  for (int sp = 1; sp < len; sp <<= 1) {
    for (int j = threadIdx.x; j < half; j += blockDim.x) {
      const int k = j & (sp - 1);
      T sv, cv;
      sincospi_((T)(-(double)k / (double)sp), &sv, &cv);
      const cpx<T> x0 = x[j], x1 = x[j + half] * mk(cv, sv);
      const int o = (j - k) * 2 + k;
      y[o] = x0 + x1;
      y[o + sp] = x0 - x1;
    }
    __syncthreads();
    cpx<T>* t = x;
    x = y;
    y = t;
  }
  for (int i = threadIdx.x; i < len; i += blockDim.x) line[i] = x[i];
}

// dst[pair][c][r] = src[pair][r][c] for p x p blocks (32 x 32 tiles)
template <class T>
__global__ void cart_transpose_kernel(const cpx<T>* src, cpx<T>* dst, int p) {
  __shared__ cpx<T> tile[32][33];
  const int64_t base = (int64_t)blockIdx.z * p * p;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int t = threadIdx.y; t < 32; t += blockDim.y) {
    const int r = r0 + t, c = c0 + threadIdx.x;
    if (r < p && c < p) tile[t][threadIdx.x] = src[base + (int64_t)r * p + c];
  }
  __syncthreads();
  for (int t = threadIdx.y; t < 32; t += blockDim.y) {
    const int c = c0 + t, r = r0 + threadIdx.x;
    if (r < p && c < p) dst[base + (int64_t)c * p + r] = tile[threadIdx.x][t];
  }
}

// table[pair][k1][k2] += (-1)^(k1+k2) K' (H x(k1))^a (H x(k2))^b / (a! b!) g[pair][k2][k1]
template <class T>
__global__ void cart_accumulate_kernel(const cpx<T>* g, cpx<T>* table, int p, int pa, int pb, double x0,
                                       double step, double height, double scale) {
  __shared__ cpx<T> tile[32][33];
  const int64_t base = (int64_t)blockIdx.z * p * p;
  const int k1_0 = blockIdx.y * 32, k2_0 = blockIdx.x * 32;
  // coalesced read of g rows k2, columns k1
  for (int t = threadIdx.y; t < 32; t += blockDim.y) {
    const int k2 = k2_0 + t, k1 = k1_0 + threadIdx.x;
    if (k1 < p && k2 < p) tile[t][threadIdx.x] = g[base + (int64_t)k2 * p + k1];
  }
  __syncthreads();
  for (int t = threadIdx.y; t < 32; t += blockDim.y) {
    const int k1 = k1_0 + t, k2 = k2_0 + threadIdx.x;
    if (k1 < p && k2 < p) {
      const double xa = height * (x0 + k1 * step), yb = height * (x0 + k2 * step);
      double c = scale;
      for (int u = 0; u < pa; ++u) c *= xa;
      for (int u = 0; u < pb; ++u) c *= yb;
      if ((k1 + k2) & 1) c = -c;
      cpx<T>& z = table[base + (int64_t)k1 * p + k2];
      z = z + (T)c * tile[threadIdx.x][t];
    }
  }
}

// reduced matrix by three-point Lagrange interpolation in the refined table (one thread per
// element pair, all MBF pairs); err bit 1 when a pair lies outside the valid region
template <class T, class TO>
__global__ void cart_fill_kernel(const cpx<T>* table, int p, int m, double x0, double step, double rho_max,
                                 int n_el, const double* pos, cpx<TO>* z, int64_t ld, int* err) {
  const int64_t total = (int64_t)n_el * n_el;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n_el), j = (int)(e % n_el);
    const double dx = pos[2 * i] - pos[2 * j], dy = pos[2 * i + 1] - pos[2 * j + 1];
    const double u = (dx - x0) / step, v = (dy - x0) / step;
    const int i0 = (int)floor(u + 0.5), j0 = (int)floor(v + 0.5);
    const bool ok = hypot(dx, dy) <= rho_max * (1.0 + 1e-12) && i0 >= 1 && i0 <= p - 2 && j0 >= 1 && j0 <= p - 2;
    if (!ok) atomicOr(err, 1);
    const double fu = u - i0, fv = v - j0;
    const double wu[3] = {0.5 * fu * (fu - 1.0), 1.0 - fu * fu, 0.5 * fu * (fu + 1.0)};
    const double wv[3] = {0.5 * fv * (fv - 1.0), 1.0 - fv * fv, 0.5 * fv * (fv + 1.0)};
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) {
        cpx<double> acc = mk(0.0, 0.0);
        if (ok) {
          const cpx<T>* t = table + (int64_t)(a * m + b) * p * p;
          for (int s = 0; s < 3; ++s)
            for (int r = 0; r < 3; ++r)
              acc = acc + (wu[s] * wv[r]) * ccast<double>(t[(int64_t)(i0 - 1 + s) * p + (j0 - 1 + r)]);
        }
        z[(int64_t)(i * m + a) * ld + j * m + b] = ccast<TO>(acc);
      }
  }
}

}  // namespace

template <class T>
cudaError_t cartesian_tabulate(const CartArgs<T>& a, int order, cpx<T>* table, cpx<T>* work, cpx<T>* work2,
                               cpx<T>* im, T* gx, T* gy, cudaStream_t s) {
  if (a.n < 2 || (a.n & 1) || a.n_mbf < 1 || a.n_mbf > kCartMaxM) return cudaErrorInvalidValue;
  const int p = 2 * a.n;
  if (p & (p - 1) || p > 4096) return cudaErrorInvalidValue;
  const int pairs = a.n_mbf * a.n_mbf;
  const int64_t nn = (int64_t)a.n * a.n, pp = (int64_t)p * p;
  const int sms = current_sm_count();
  cudaError_t e = cudaMemsetAsync(table, 0, (size_t)pairs * pp * sizeof(cpx<T>), s);
  if (e != cudaSuccess) return e;
  cart_spectrum_kernel<T><<<(unsigned)((nn + 127) / 128), 128, 0, s>>>(a, im, gx, gy);
  const size_t fsmem = (size_t)2 * p * sizeof(cpx<T>);
  if ((e = cudaFuncSetAttribute(line_fft_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem)) !=
      cudaSuccess)
    return e;
  const int fthreads = std::min(p / 2, 512);
  const dim3 tgrid((p + 31) / 32, (p + 31) / 32, pairs), tblock(32, 8);
  const double step = 3.14159265358979323846 / (2.0 * a.k_max);
  const double x0 = -(double)a.n * 3.14159265358979323846 / (2.0 * a.k_max);
  const double kprime = a.dk * a.dk / (4.0 * 3.14159265358979323846 * 3.14159265358979323846);
  for (int deg = 0; deg <= order; ++deg)
    for (int pa = deg; pa >= 0; --pa) {
      const int pb = deg - pa;
      double fact = 1.0;
      for (int t = 2; t <= pa; ++t) fact *= t;
      for (int t = 2; t <= pb; ++t) fact *= t;
      cart_monomial_kernel<T><<<(unsigned)std::min<int64_t>((pp * pairs + 255) / 256, (int64_t)sms * 32), 256, 0, s>>>(
          im, gx, gy, a.n, pa, pb, pairs, work);
      line_fft_kernel<T><<<(unsigned)(p * pairs), fthreads, fsmem, s>>>(work, p);
      cart_transpose_kernel<T><<<tgrid, tblock, 0, s>>>(work, work2, p);
      line_fft_kernel<T><<<(unsigned)(p * pairs), fthreads, fsmem, s>>>(work2, p);
      cart_accumulate_kernel<T><<<tgrid, tblock, 0, s>>>(work2, table, p, pa, pb, x0, step, a.height,
                                                         kprime / fact);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  return cudaGetLastError();
}

template <class T, class TO>
cudaError_t cartesian_fill(const cpx<T>* table, int p, int m, double x0, double step, double rho_max, int n_el,
                           const double* pos, void* z, int64_t ld, int* err, cudaStream_t s) {
  const int64_t total = (int64_t)n_el * n_el;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)current_sm_count() * 16));
  cart_fill_kernel<T, TO><<<blocks, 256, 0, s>>>(table, p, m, x0, step, rho_max, n_el, pos,
                                                 reinterpret_cast<cpx<TO>*>(z), ld, err);
  return cudaGetLastError();
}

template cudaError_t cartesian_tabulate<float>(const CartArgs<float>&, int, cpx<float>*, cpx<float>*, cpx<float>*,
                                               cpx<float>*, float*, float*, cudaStream_t);
template cudaError_t cartesian_tabulate<double>(const CartArgs<double>&, int, cpx<double>*, cpx<double>*,
                                                cpx<double>*, cpx<double>*, double*, double*, cudaStream_t);
template cudaError_t cartesian_fill<float, float>(const cpx<float>*, int, int, double, double, double, int,
                                                  const double*, void*, int64_t, int*, cudaStream_t);
template cudaError_t cartesian_fill<float, double>(const cpx<float>*, int, int, double, double, double, int,
                                                   const double*, void*, int64_t, int*, cudaStream_t);
template cudaError_t cartesian_fill<double, double>(const cpx<double>*, int, int, double, double, double, int,
                                                    const double*, void*, int64_t, int*, cudaStream_t);
template cudaError_t cartesian_fill<double, float>(const cpx<double>*, int, int, double, double, double, int,
                                                   const double*, void*, int64_t, int*, cudaStream_t);

}  // namespace cfft
