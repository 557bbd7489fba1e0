// Shared device/host helpers of the GB300 C-FFT kernels: a small complex type,
// precision-overloaded math, and the kernel argument structs.  Nothing here
// is specific to one stage; every formula lives in the kernel that uses it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace cfft {

// streaming multiprocessors of the current device (persistent grids and grid-stride caps
// are sized from it; the runtime caches the attribute)
inline int current_sm_count() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
    cudaGetLastError();
    v = 1;
  }
  return v;
}

template <class T>
struct alignas(2 * sizeof(T)) cpx {
  T re, im;
};

template <class T>
__host__ __device__ __forceinline__ cpx<T> mk(T r, T i) {
  cpx<T> z;
  z.re = r;
  z.im = i;
  return z;
}
template <class T>
__host__ __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) {
  return mk(a.re + b.re, a.im + b.im);
}
template <class T>
__host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) {
  return mk(a.re - b.re, a.im - b.im);
}
template <class T>
__host__ __device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class T>
__host__ __device__ __forceinline__ cpx<T> operator*(T s, cpx<T> a) {
  return mk(s * a.re, s * a.im);
}
template <class T>
__host__ __device__ __forceinline__ cpx<T> conj(cpx<T> a) {
  return mk(a.re, -a.im);
}
// a += b * c
template <class T>
__host__ __device__ __forceinline__ void cmac(cpx<T>& a, cpx<T> b, cpx<T> c) {
  a.re = fma(b.re, c.re, fma(-b.im, c.im, a.re));
  a.im = fma(b.re, c.im, fma(b.im, c.re, a.im));
}
// a += conj(b) * c
template <class T>
__host__ __device__ __forceinline__ void cmac_conj(cpx<T>& a, cpx<T> b, cpx<T> c) {
  a.re = fma(b.re, c.re, fma(b.im, c.im, a.re));
  a.im = fma(b.re, c.im, fma(-b.im, c.re, a.im));
}
template <class T>
__host__ __device__ __forceinline__ cpx<T> cdiv(cpx<T> a, cpx<T> b) {
  // Smith's algorithm
  if (fabs(b.re) >= fabs(b.im)) {
    T r = b.im / b.re, d = b.re + b.im * r;
    return mk((a.re + a.im * r) / d, (a.im - a.re * r) / d);
  }
  T r = b.re / b.im, d = b.im + b.re * r;
  return mk((a.re * r + a.im) / d, (a.im * r - a.re) / d);
}
template <class TO, class TI>
__host__ __device__ __forceinline__ cpx<TO> ccast(cpx<TI> a) {
  return mk<TO>((TO)a.re, (TO)a.im);
}

// precision-overloaded accurate math (never the fast-math intrinsics)
__device__ __forceinline__ void sincospi_(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ void sincos_(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ float exp_(float x) { return expf(x); }
__device__ __forceinline__ double exp_(double x) { return exp(x); }
__device__ __forceinline__ float cospi_(float x) { return cospif(x); }
__device__ __forceinline__ double cospi_(double x) { return cospi(x); }

// e^{i pi x} with x reduced exactly modulo 2 in float64 first
template <class T>
__device__ __forceinline__ cpx<T> expipi(double x) {
  double r = x - 2.0 * floor(0.5 * x);  // [0, 2)
  T s, c;
  sincospi_((T)r, &s, &c);
  return mk(c, s);
}

__device__ __forceinline__ float sinh_(float x) { return sinhf(x); }
__device__ __forceinline__ double sinh_(double x) { return sinh(x); }
__device__ __forceinline__ float cosh_(float x) { return coshf(x); }
__device__ __forceinline__ double cosh_(double x) { return cosh(x); }

// sin(z), cos(z) for complex z.  sinh of the imaginary part comes from the library
// function, not from (e^y - e^-y)/2, whose cancellation for small y leaves an
// absolute error of one ulp of 1 in Im sin z (amplified by 1/|z| in sin(z)/z).
template <class T>
__device__ __forceinline__ void csincos(cpx<T> z, cpx<T>* sz, cpx<T>* cz) {
  T s, c;
  sincos_(z.re, &s, &c);
  const T ch = cosh_(z.im), sh = sinh_(z.im);
  *sz = mk(s * ch, c * sh);
  *cz = mk(c * ch, -s * sh);
}

// sin(z)/z for complex z (series near zero)
template <class T>
__device__ __forceinline__ cpx<T> csinc(cpx<T> z) {
  T a2 = z.re * z.re + z.im * z.im;
  if (a2 < (T)1e-4) {
    cpx<T> z2 = z * z;
    // 1 - z^2/6 + z^4/120 - z^6/5040
    cpx<T> t = mk((T)(-1.0 / 5040.0) * z2.re, (T)(-1.0 / 5040.0) * z2.im);
    t = mk(t.re + (T)(1.0 / 120.0), t.im);
    t = t * z2;
    t = mk(t.re - (T)(1.0 / 6.0), t.im);
    t = t * z2;
    return mk(t.re + (T)1, t.im);
  }
  cpx<T> s, c;
  csincos(z, &s, &c);
  return cdiv(s, z);
}

// principal complex square root
template <class T>
__device__ __forceinline__ cpx<T> csqrt_(cpx<T> z) {
  T r = hypot(z.re, z.im);
  if (r == (T)0) return mk((T)0, (T)0);
  if (z.re >= (T)0) {
    T t = sqrt((T)0.5 * (r + z.re));
    return mk(t, z.im / ((T)2 * t));
  }
  T t = sqrt((T)0.5 * (r - z.re));
  return mk(fabs(z.im) / ((T)2 * t), copysign(t, z.im));
}

// ---------------------------------------------------------------------------
// kernel arguments

struct ContourArgs {
  int n;
  double beta_max, beta_p, height, step;  // step = beta_max / n
  double eps_r, hs, k0;
  int extract;                            // 1: subtract the homogeneous medium and its image
  double eps_eff, deps_eff;               // its permittivity and d eps_eff / d eps_r
  int es_width;                           // > 0: ES precorrection of that kernel width
  double ds;                              // transform grid step (for the precorrection)
};

// per-node contour data written by the contour kernel (float64 throughout)
struct ContourData {
  double2* beta_c;  // beta_R + i beta_I
  double2* weight;  // step * (1 + i dbeta_I/dbeta_R)
  double2* bw;      // beta_c * weight  (the factor of Eq. 9's beta d beta)
  double* bi_rel;   // beta_I / height  (0 beyond beta_p); in [0, 1]
  float* bi_rel_f;  // the same in float32 (read by the float32 transform)
  double2* green_p; // G = P I - R k k^T  (P, R: functions of beta only)
  double2* green_r; // R * beta_c^2
  // optional (null to skip): derivatives of P and R beta_c^2 with respect to
  // eps_r and to the slab thickness h, contour held fixed
  double2* dp_eps;
  double2* dr_eps;
  double2* dp_h;
  double2* dr_h;
  // optional: 1 / phi_hat(omega_j) of the ES interpolation kernel, omega_j = (beta_c,j -
  // beta_max / 2) ds, the precorrection of the FP32-mixed transform input
  float2* prec;
};

struct ShapeClass {
  int kind;      // 0 = rooftop, 1 = cosine strip
  int dir;       // 0 = x, 1 = y
  int begin;     // basis range [begin, end) of this class (bases sorted by class)
  int end;
  double p1, p2; // rooftop: half-length, width; strip: length, width
};

constexpr int kMaxShapeClasses = 32;
constexpr int kMaxBasis = 4096;

template <class T>
struct IntegrandArgs {
  int n, n_alpha, q_max, n_cls;  // n_cls computed classes (1 or 3)
  int n_mbf;                      // real MBF count (q holds a padded column count)
  int n_shape, n_basis;
  const ShapeClass* shapes;       // device, n_shape
  const T* bx;                    // device, basis centres x (sorted by class)
  const T* by;
  const cpx<T>* q;                // device, [n_basis][M padded]
  const double2* beta_c;
  const double2* bw;
  const double2* green_p;
  const double2* green_r;
  cpx<T>* y;                      // out [cls][pair][qi][n]
  // tensor-core spectra (FP32 rooftop elements): float centres, GEMM B operand (with the
  // mirrored columns of the opposite wave direction) and its width (both blocks)
  const float* tc_bx;
  const float* tc_by;
  const float* tc_bmat;
  int tc_ncol;
  float tc_rmax;                  // max |r_i| of the basis centres
  int* err;                       // bit 4: a tensor-core wait ran past its bound
};

template <class T>
struct FftArgs {
  int series, n, sub_len, log2_sub, n_sub;   // n_sub = D = P / sub_len
  int64_t fft_len;                            // P = sigma * n
  int grid_half;                              // K
  int taylor;                                 // highest term index N of the series
  int expansion;                              // contour-factor series: 0 Taylor (Eq. 22), 1 Chebyshev
  int n_active;                               // nodes with beta_I > 0 (prefix)
  int sigma;
  double ds_height;                           // delta_s * height  (series variable scale)
  const cpx<T>* y;                            // [series][n]
  const double* bi_rel;                       // [n]
  const float* bi_rel_f;                      // [n] float32 copy
  const cpx<T>* twiddle;                      // [sub_len] e^{-2 pi i t / sub_len}
  const cpx<T>* prec;                         // [n] input precorrection (null: none)
  cpx<T>* grid;                               // [series][2K+1]
};

template <class T>
struct BackprojArgs {
  int series_per_q;        // classes * pairs
  int n_harm, q_max, n_rho, grid_half, sigma, taps, group, rchunk;
  double d_rho, d_s;       // rho step, s step
  double beta_abs_max;     // max |beta_c| (angular content of the integrand)
  double alpha_margin;
  const cpx<T>* grid;      // [series][2K+1]   series = (cls*pairs + pair) * n_harm + qi
  cpx<T>* table;           // [series][n_rho]
  const int* chunk_nodes;  // [chunks] angular nodes of each chunk of rows
  const int64_t* chunk_off;// [chunks] offset of its cosines in cosv
  const double* cosv;      // node cosines
  int* err;                // tensor-core form: bit 5 set when a wait ran past its bound
  int kern;                // interpolation kernel: 0 Lagrange, 1 ES (precorrected grid)
};

// back-projection with the W x G+- product on the tensor cores (FP32-mixed)
size_t backproject_tc_smem(int max_nodes);
int backproject_tc_ktile();
cudaError_t launch_backproject_tc(const BackprojArgs<float>& a, int n_tiles, int max_nodes, cudaStream_t s);
cudaError_t launch_backproject_tc_batch(const BackprojArgs<float>* items, const int4* tasks, int n_tasks,
                                        int* counter, int taps, int kern, int max_nodes, int n_ctas,
                                        cudaStream_t s);

template <class T, class TO>
struct FillArgs {
  int n_el, n_mbf, q_max, n_harm, n_rho, taps, n_cls;
  double inv_d_rho, rho_max;
  int64_t ld;
  const cpx<T>* table;     // [cls][pair][qi][r]
  const double* pos;       // [2 * n_el]
  const int* rot;          // [n_el] or null
  cpx<TO>* z;              // [(m*M + a) * ld + n*M + b]
  int* err;                // set when a pair lies beyond rho_max
};

// host launchers (one translation unit per stage)
void launch_contour(const ContourArgs& a, const ContourData& d, cudaStream_t s);
template <class T>
void launch_twiddle(cpx<T>* tw, int len, cudaStream_t s);
template <class T>
cudaError_t launch_integrand(const IntegrandArgs<T>& a, int n_mbf_padded, cudaStream_t s);
template <class T>
cudaError_t launch_fft(const FftArgs<T>& a, cudaStream_t s);
template <class T>
int integrand_tile_nodes(const IntegrandArgs<T>& a, int n_mbf_padded);
// fused integrand with the MBF spectra on the tensor cores (FP32, N_alpha = 128 or 256,
// a.tc_* set); false when the form does not apply
bool integrand_tc_applies(const IntegrandArgs<float>& a);
cudaError_t launch_integrand_tc(const IntegrandArgs<float>& a, cudaStream_t s);
// contour nodes per CTA of the tensor-core integrand (n_alpha 128 or 256), and its batched launch
int integrand_tc_nodes(int n_alpha);
cudaError_t launch_integrand_tc_batch(const IntegrandArgs<float>& shape_args, const IntegrandArgs<float>* items,
                                      const int2* map, int n_blocks, cudaStream_t s);
template <class T>
cudaError_t launch_integrand_batch(const IntegrandArgs<T>& shape_args, const IntegrandArgs<T>* items,
                                   const int2* map, int n_blocks, int jt, int n_mbf_padded,
                                   cudaStream_t s);
void launch_contour_batch(const ContourArgs* items, const ContourData* data, const int2* map,
                          int n_blocks, cudaStream_t s);
// shared-memory bytes of one transform task beyond its FFT buffer
template <class T>
__host__ __device__ constexpr size_t fft_task_extra(int /*n_active_max*/, int n_out_max, int hi_max) {
  return (size_t)(128 + hi_max + 128 + 128) * sizeof(cpx<T>) +
         (size_t)n_out_max * (sizeof(cpx<T>) + sizeof(T)) + 64;
}

template <class T>
cudaError_t launch_fft_batch(const FftArgs<T>* items, const int4* tasks, int n_tasks, int* counter,
                             int log2_sub, int max_n_out, int max_active, int max_hi, int zt_arrays,
                             int n_ctas, cudaStream_t s);
template <class T>
size_t backproject_smem(int group, int max_seg, int max_nodes);
template <class T>
cudaError_t launch_backproject_impl(const BackprojArgs<T>& a, const int* chunk_nodes,
                                    const int64_t* chunk_off, const double* cosv,
                                    const double* lag_den, int n_chunks, int max_nodes,
                                    int max_seg, cudaStream_t s);
template <class T>
cudaError_t launch_backproject_batch(const BackprojArgs<T>* items, const int4* tasks, int n_tasks,
                                     int* counter, int taps, int group, int max_nodes, int max_seg,
                                     int n_ctas, cudaStream_t s);
cudaError_t launch_chunk_cosines(const int* n_nodes, const int64_t* offset, int n_chunks,
                                 int max_nodes, double* cosv, cudaStream_t s);
template <class T>
size_t backproject_w_smem(int max_nodes, int series);
// paired-harmonic matrix form (FP32-mixed, taps 8/12/16): tiles of backproject_pm_rows()
// rows, tasks (tile, |q|, chunk of backproject_pm_series_chunk() series per sign)
size_t backproject_pm_smem(int max_nodes);
int backproject_pm_rows();
int backproject_pm_series_chunk();
cudaError_t launch_backproject_pm(const BackprojArgs<float>& a, int n_tiles, int max_nodes, cudaStream_t s);
cudaError_t launch_backproject_pm_batch(const BackprojArgs<float>* items, const int4* tasks, int n_tasks,
                                        int* counter, int taps, int kern, int max_nodes, int n_ctas,
                                        cudaStream_t s);
int backproject_w_rows();
template <class T>
cudaError_t launch_backproject_w(const BackprojArgs<T>& a, int n_tiles, int max_nodes, cudaStream_t s);
template <class T>
cudaError_t launch_backproject_w_batch(const BackprojArgs<T>* items, const int4* tasks, int n_tasks,
                                       int* counter, int taps, int max_nodes, int series, int n_ctas,
                                       cudaStream_t s);
template <class T>
void launch_class_phase(cpx<T>* table, int pairs, int n_harm, int q_max, int n_rho,
                        cudaStream_t s);
template <class T>
void launch_nonfinite(const cpx<T>* buf, int64_t count, int* flag, cudaStream_t s);
template <class T, class TG>
struct FillBackArgs {
  FillArgs<T, float> f;      // geometry and table (f.z unused)
  const cpx<T>* dtab_eps;    // d table / d eps_r  (null: no substrate gradient)
  const cpx<T>* dtab_h;      // d table / d h
  const cpx<TG>* grad;       // dL/dZ (torch convention: dL = Re sum conj(G) dZ)
  int64_t ld_g;
  double d_rho;
  double* grad_pos;          // [2 * n_el], accumulated
  double* grad_theta;        // [2], accumulated (eps_r, h)
};

// plan of the bucketed fill (pairs counting-sorted by rotation class and
// stencil row, table windows staged in shared memory); ok = false: per-row fill
struct FillBucketPlan {
  bool ok;
  bool tc;                 // the tensor-core form (FP32, M = 4, 8 taps)
  int win, n_cells, nb_bits, block_rows, rows_per_wave;
  size_t n_keys_max, smem, scratch;
};
template <class T>
FillBucketPlan plan_fill_bucketed(int n_el, int n_mbf, int n_harm, int n_rho, int taps, int n_cls,
                                  int block_rows, bool tc);
template <class T>
cudaError_t launch_fill_bucketed(const FillArgs<T, T>& a, const FillBucketPlan& plan, void* scratch,
                                 cudaStream_t s);
// adjoint of the bucketed fill: position gradient (grad_pos) and, with both
// derivative tables, the (eps_r, h) gradient (grad_theta[0..1]); both accumulated
template <class T>
struct FillAdjointArgs {
  const cpx<T>* grad;        // dL/dZ, same layout as the matrix, leading dimension ld_g
  int64_t ld_g;
  const cpx<T>* dtab_eps;    // d table / d eps_r, or null
  const cpx<T>* dtab_h;      // d table / d h, or null
  double* grad_pos;          // [2 * n_el] or null
  double* grad_theta;        // [2] or null
};
template <class T>
cudaError_t launch_fill_adjoint_bucketed(const FillArgs<T, T>& a, const FillAdjointArgs<T>& ad,
                                         const FillBucketPlan& plan, void* scratch, cudaStream_t s);

// the bounded mbarrier wait, run out on purpose: flag = 16 after `polls` tries
cudaError_t launch_wait_selftest(unsigned polls, int* flag, cudaStream_t s);

// MBF spectra on the tensor cores (FP32 with TF32 head/tail splitting)
int spectra_tc_columns(int n_shape, int n_mbf);
void spectra_tc_bmatrix(int n_basis, int n_shape, const int* basis_class, int n_mbf,
                        const double* q_re_im, int q_stride, bool mirror, std::vector<float>* out);
cudaError_t launch_spectra_tc(int n_points, int n_basis, int n_shape, int n_mbf, const ShapeClass* shapes,
                              const float* bx, const float* by, const float* bmat, const void* k, void* out,
                              int* err, cudaStream_t s);

template <class T, class TG>
cudaError_t launch_fill_backward(const FillBackArgs<T, TG>& a, cudaStream_t s);
// g[i][j] = 2 r_i conj(v_j), n x n row-major (dL/dZ' of sum |Z' v - t|^2 with r = Z' v - t)
template <class T>
cudaError_t launch_residual_outer(const void* r, const void* v, int n, void* g, cudaStream_t s);
// a posteriori interpolation-error estimate of the fill on a table's rho grid: per series
// (n_rho entries each) out = (max |Z|, max over interior windows of |p-th difference| *
// fac_c, the last window's |p-th difference| * fac_e, 0)
template <class T>
cudaError_t launch_fill_estimate(const void* table, int64_t n_series, int n_rho, int q_max, int taps,
                                 double fac_c, double fac_e, double4* out, cudaStream_t s);
// the 2-D Cartesian C-FFT (k_cartesian.cu): N x N spectral samples on [-k_max, k_max)^2
// (dk = 2 k_max / N), the contour (beta_p, height), the substrate and the element
template <class T>
struct CartArgs {
  int n, n_mbf, n_shape, q_stride;
  double k_max, dk, beta_p, height, eps_r, hs, k0;
  int extract;
  double eps_eff;
  const ShapeClass* shapes;
  const T* bx;
  const T* by;
  const cpx<T>* q;   // [n_basis][q_stride], bases sorted by shape class
};
// the refined table [pairs][2N][2N] (dx-major) up to Taylor order `order`; work, work2:
// [pairs][2N][2N]; im: [pairs][N][N]; gx, gy: [N][N]
template <class T>
cudaError_t cartesian_tabulate(const CartArgs<T>& a, int order, cpx<T>* table, cpx<T>* work, cpx<T>* work2,
                               cpx<T>* im, T* gx, T* gy, cudaStream_t s);
template <class T, class TO>
cudaError_t cartesian_fill(const cpx<T>* table, int p, int m, double x0, double step, double rho_max, int n_el,
                           const double* pos, void* z, int64_t ld, int* err, cudaStream_t s);

// dense LU of the reduced system (k_solve.cu): device work arrays of one factorization
struct LuWork {
  int2* moves;         // [panels][2 * panel width] row moves (source, destination)
  int* n_moves;        // [panels]
  double* cand_val;    // [2][SMs] 64-bit words: the panel CTAs' pivot keys with column tags
  int* cand_row;       // (unused)
  void* cand_data;     // [2][SMs][panel width] complex, the element type: the candidates' entries
  unsigned* bar;       // (unused)
  int* err;            // bit 1: a key poll ran out; bit 2: zero pivot; bit 3: a tensor-core
                       // wait of the trailing update ran out
  int* diag;           // host: [5] panel grid, resident CTAs per SM, shared bytes of the last grid
                       // panel; panels run on one cluster, CTAs per cluster (0: none)
  int tc_update;       // complex64: the trailing update on the tensor cores
  int panel_cluster;   // 1: panels whose rows fit one cluster's shared memory run there
};
int lu_panel_width();
// the largest order whose panels fit the panel CTAs' shared memory on `sms` SMs
template <class T>
int lu_max_order(int sms);
template <class T>
cudaError_t lu_factor(cpx<T>* a, int64_t ld, int n, const LuWork& w, cudaStream_t s);
template <class T>
cudaError_t lu_solve(const cpx<T>* a, int64_t ld, int n, const LuWork& w, cpx<T>* x, cpx<T>* y, cudaStream_t s);
cudaError_t residual_f64(const void* z, int64_t ld, int n, const void* x, const void* b, void* r, double* sums,
                         cudaStream_t s);
cudaError_t residual_f32(const void* z, int64_t ld, int n, const void* x, const void* b, double* sums,
                         cudaStream_t s);
template <class TD, class TS>
cudaError_t copy_matrix(const void* src, int64_t ld, int n, void* dst, cudaStream_t s);
template <class TD, class TS>
cudaError_t copy_vector(const void* src, int n, void* dst, cudaStream_t s);
cudaError_t add_correction(void* x, const void* d, int n, double* sums, cudaStream_t s);
// kind 0: V' = Q^H V; 1: delta-gap port excitation; 2: port currents (q: complex128 [B][M])
template <class T>
cudaError_t launch_excitation(int kind, int n_el, int n_basis, int m, int port, const void* in, const double* q,
                              void* out, cudaStream_t s);

// plan.ok: bucketed fill with `scratch` of plan.scratch bytes; else the per-row fill
template <class T, class TO>
cudaError_t launch_fill(const FillArgs<T, TO>& a, const FillBucketPlan& plan, void* scratch, cudaStream_t s);

}  // namespace cfft
