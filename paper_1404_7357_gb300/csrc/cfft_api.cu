// C ABI of the C-FFT library (declared in include/cfft.h): context, state
// machine, parameter choice, device buffers and the stage launches.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/cfft.h"
#include <type_traits>

#include "cfft_common.cuh"
#include "spectra_tc.cuh"

namespace cfft {
template <class T>
size_t backproject_smem(int group, int max_seg, int max_nodes);
template <class T>
cudaError_t launch_backproject_impl(const BackprojArgs<T>& a, const int* chunk_nodes,
                                    const int64_t* chunk_off, const double* cosv,
                                    const double* lag_den, int n_chunks, int max_nodes,
                                    int max_seg, cudaStream_t s);
cudaError_t launch_chunk_cosines(const int* n_nodes, const int64_t* offset, int n_chunks,
                                 int max_nodes, double* cosv, cudaStream_t s);
}  // namespace cfft

using namespace cfft;

namespace {

constexpr double kPi = 3.14159265358979323846;

// failure injection on the host (cfft_test_fail_allocation): the number of library
// allocations still to succeed before one fails as out of memory; -1 = disarmed
long g_alloc_countdown = -1;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t need) {
    if (need <= bytes && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    if (need == 0) need = 16;
    if (g_alloc_countdown == 0) {   // injected: no allocation is attempted
      g_alloc_countdown = -1;
      return cudaErrorMemoryAllocation;
    }
    if (g_alloc_countdown > 0) --g_alloc_countdown;
    cudaError_t e = cudaMalloc(&p, need);
    if (e == cudaSuccess) bytes = need;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <class U>
  U* as() const {
    return reinterpret_cast<U*>(p);
  }
};

constexpr int kNumOptions = CFFT_OPT_SOLVE_GRID_PANEL + 1;

}  // namespace

struct cfft_ctx {
  int device = 0;
  int sm_count = 1;   // of the device (persistent grids, FFT sub-length choice)
  cudaStream_t stream = nullptr;
  std::string err = "no error";
  // substrate
  bool has_sub = false;
  double eps_r = 1, hs = 0, k0 = 1;
  // Green's function: 1 = the effective homogeneous medium and its image subtracted
  // (eps_eff <= 0: (eps_r + 1) / 2)
  int extract = 0;
  double eps_eff_set = 0.0;
  // element (bases sorted by shape class; Q padded to n_mbf_pad columns)
  bool has_el = false;
  int n_basis = 0, n_mbf = 0, n_mbf_pad = 0;
  std::vector<ShapeClass> shapes;
  std::vector<double> bx, by;
  std::vector<std::complex<double>> q;  // [n_basis][n_mbf_pad]
  double elem_radius = 0;
  // contour
  bool has_contour = false;
  int n = 0, taylor_req = -1;
  double beta_max = 0, beta_p = 0, height = 0;
  // options (<= 0: automatic) and the options the last table was made with
  double opt[kNumOptions] = {};
  double tab_opt[kNumOptions] = {};
  // table
  bool has_table = false;
  int q_max = 0, n_rho = 0, cls_stored = 1, cls_computed = 1, fill_taps = 8;
  double rho_max = 0;
  cfft_precision prec = CFFT_FP64;
  cfft_info info{};
  // the table the fill interpolates: the tabulated one, or (fill_own) d_ftable on n_frho
  // points to frho_max, fill_r times finer than the tabulated grid and reaching beyond
  // rho_max (fill_r = 0: not decided yet; decided at the first fill or adjoint after a
  // tabulation or load)
  int fill_r = 0, n_frho = 0;
  double frho_max = 0;
  bool fill_own = false, table_loaded = false;
  DevBuf d_ftable, d_fest;
  // device buffers
  DevBuf beta_c, weight, bw, bi_rel, green_p, green_r, dp_eps, dr_eps, dp_h, dr_h;
  int channels = 1;  // 1: table; 3: table, d/d eps_r, d/d h
  DevBuf d_shapes, d_bx, d_by, d_q, d_y, d_grid, d_table, d_tw, d_cnodes, d_coff, d_cos, d_lag, d_prec,
      d_flag, d_pos, d_rot, d_zbuf, d_fill, d_gres;
  int tw_len = 0, tw_prec = -1;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // batched sweep: plan arrays, scratch, stream, captured graph, tuned shape
  DevBuf b_cargs, b_cdata, b_iargs, b_fargs, b_bargs, b_cmap, b_imap, b_ftask, b_btask, b_count,
      b_cnodes, b_coff, b_cos, b_contour, b_y, b_grid, b_flag;
  cudaStream_t bstream = nullptr;
  cudaEvent_t bev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaGraphExec_t bgraph = nullptr;
  std::string bsig;           // signature of the captured graph
  std::string bshape;         // what the captured graph bakes in: addresses, launch shapes, task ranges
  struct TunedPlan { int sub_len, rchunk, bp_tc; };
  std::map<std::string, TunedPlan> tuned;  // signature -> tuned shape
  double b_ms[4] = {0, 0, 0, 0};
  double b_work_bp = 0, b_work_fft = 0;
  int b_launches = 0, b_sub_len = 0, b_rchunk = 0, b_waves = 0, b_bp_tc = 0, b_captures = 0;
  // the element's coefficient matrix Q in the caller's basis order ([n_basis][n_mbf]), for
  // the reduced excitation and port currents, and its device copy
  std::vector<std::complex<double>> q_user;
  DevBuf d_quser;
  // dense LU of the reduced system: the factored copy, work arrays, vectors, timing
  DevBuf lu_a, lu_moves, lu_nmoves, lu_cand_v, lu_cand_r, lu_cand_d, lu_bar, lu_err, lu_x, lu_y, lu_x64, lu_r, lu_sums;
  cudaEvent_t lu_ev[3] = {nullptr, nullptr, nullptr};
  int lu_diag[5] = {0, 0, 0, 0, 0};
  cfft_solve_info solve_info{};
  // the 2-D Cartesian C-FFT table and its work buffers
  DevBuf c_tab, c_work, c_work2, c_im, c_gx, c_gy, c_flag;
  bool has_ctab = false;
  cfft_cartesian_info c_info{};
  // tensor-core spectra: float copies of the element and its GEMM B operand
  DevBuf tc_bx, tc_by, tc_bmat, tc_bmat_mirror, tc_shapes;
  bool tc_ready = false;
  float tc_rmax = 0;
};

namespace {

cfft_status fail(cfft_ctx* c, cfft_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

cfft_status cuda_fail(cfft_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(c, CFFT_ERR_OOM, m);
  return fail(c, CFFT_ERR_CUDA, m);
}

#define CFFT_CUDA(call, where)                                  \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where);    \
  } while (0)

cfft_status ensure_tc_element(cfft_ctx* ctx);

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

double lgamma_fact(int n) { return std::lgamma((double)n + 1.0); }

// smallest N_t with x^(N_t+1)/(N_t+1)! e^x <= tol (remainder bound of Eq. 22), or -1
// when no order up to 64 reaches tol (a contour too high for the table's rho_max)
int auto_taylor(double x, double tol) {
  if (x <= 0) return 0;
  for (int nt = 0; nt <= 64; ++nt) {
    double lg = (nt + 1) * std::log(x) - lgamma_fact(nt + 1) + x;
    if (lg <= std::log(tol)) return nt;
  }
  return -1;
}

// modified Bessel function I_m(a), a >= 0, by its power series
double bessel_i_host(int m, double a) {
  const double half = 0.5 * a;
  double t = 1.0;
  for (int i = 1; i <= m; ++i) t *= half / i;
  double sum = t;
  for (int i = 1; i < 200; ++i) {
    t *= half * half / ((double)i * (i + m));
    sum += t;
    if (t <= 1e-18 * sum) break;
  }
  return sum;
}

// smallest degree N of the Chebyshev series of the contour factor (exp(H s b) =
// exp(a) exp(a z), a = H s / 2, z = 2 b - 1) whose remainder bound
// exp(a) * 2 sum_{m > N} I_m(a) at a = x / 2 is <= tol, or -1 beyond degree 64
int auto_chebyshev(double x, double tol) {
  if (x <= 0) return 0;
  const double a = 0.5 * x;
  for (int nc = 0; nc <= 64; ++nc) {
    double tail = 0.0;
    for (int m = nc + 1; m <= nc + 60; ++m) {
      const double im = bessel_i_host(m, a);
      tail += im;
      if (im <= 1e-3 * tail) break;
    }
    if (std::exp(a) * 2.0 * tail <= tol) return nc;
  }
  return -1;
}

// the contour-factor series of a tabulation: {series, highest term index}.  An explicit
// order keeps the paper's Taylor series (Eq. 22) unless the option asks for Chebyshev;
// the automatic choice takes the series with fewer transforms (Taylor: N + 1; Chebyshev:
// N + 2, one of them the nodes beyond the active prefix), Taylor on a tie
struct SeriesChoice {
  int series, order;
};

// remainder bound the automatic order holds the contour-factor series to, relative to the
// summed magnitudes of the transform's inputs: 1e-13 in FP64; 2^-22 in FP32-mixed, below the
// rounding of the float32 transform that follows (about log2(L) 2^-24 of the same sum, 8e-7
// at L = 16384)
constexpr double kSeriesTolFp64 = 1e-13, kSeriesTolFp32 = 0x1p-22;

SeriesChoice choose_series(double x, bool fp64, int order_req, double opt) {
  const double tol = fp64 ? kSeriesTolFp64 : kSeriesTolFp32;
  const int mode = opt > 0 ? (int)opt : 0;   // 0 automatic, 1 Taylor, 2 Chebyshev
  if (order_req >= 0) return {mode == 2 ? 1 : 0, order_req};
  const int nt = auto_taylor(x, tol);
  if (mode == 1) return {0, nt};
  const int nc = auto_chebyshev(x, tol);
  if (mode == 2) return {1, nc};
  if (nc >= 0 && (nt < 0 || nc + 2 < nt + 1)) return {1, nc};
  return {0, nt};
}

// interpolation kernel of the back-projection: ES (spectrally precorrected grid) in
// FP32-mixed for the paired matrix forms with 6 or 8 taps, Lagrange otherwise.  Option
// BP_KERNEL: <= 0 automatic, 1 Lagrange, 2 ES.  Returns -1 for an ES request it cannot take.
int choose_bp_kernel(bool fp64, bool gather, int taps_opt, double kern_opt) {
  const int mode = kern_opt > 0 ? (int)kern_opt : 0;
  const bool es_ok = !fp64 && !gather && (taps_opt <= 0 || taps_opt == 6 || taps_opt == 8);
  if (mode == 1) return 0;
  if (mode == 2) return es_ok ? 1 : -1;
  return es_ok ? 1 : 0;
}

// angular nodes of the back-projection for the largest rho of a chunk.  With z = |beta| rho
// the integrand g(rho cos alpha) holds angular harmonics up to about z, and the midpoint
// rule's error is the first aliased one, J_n(z) with n ~ 2 N - |q|.  Above its order J_n
// falls like Ai(x), x = (2/n)^(1/3) (n - z), so the excess n - z must grow like z^(1/3):
// 2 N = z + |q| + 2 c z^(1/3) + margin keeps x >= 2^(4/3) c at every rho.  c = 2 (x >= 5)
// holds the float32 target; the float64 target needs c = 4 (x >= 10): on the 200-rooftop
// patch at rho = 50 wavelengths (z = 3300) c = 2 leaves 4.5e-10 of the table maximum,
// c = 4 leaves 2e-15
int alpha_nodes(double beta_abs_max, double rho, int q_max, double margin, double cbrt_coef) {
  double z = beta_abs_max * rho;
  return (int)std::ceil(0.5 * (z + q_max) + cbrt_coef * std::cbrt(z) + 0.5 * margin) + 1;
}

double alpha_cbrt_coef(bool fp64) { return fp64 ? 4.0 : 2.0; }

// the extraction fields of a contour for substrate permittivity eps_r
void set_extraction(const cfft_ctx* ctx, double eps_r, int* extract, double* eps_eff, double* deps_eff) {
  *extract = ctx->extract;
  const bool automatic = !(ctx->eps_eff_set > 0.0);
  *eps_eff = automatic ? 0.5 * (eps_r + 1.0) : ctx->eps_eff_set;
  *deps_eff = automatic ? 0.5 : 0.0;
}

// One tabulation into `dst` on n_rho points rho_r = r rho_max / (n_rho - 1).  primary: the
// table of cfft_tabulate_reactions (its diagnostics go to ctx->info); otherwise the table
// that the fill interpolates when the tabulated grid misses the fill's target.
template <class T>
cfft_status tabulate_impl(cfft_ctx* ctx, int n_rho, double rho_max, DevBuf& dst, bool primary) {
  cudaStream_t st = ctx->stream;
  const bool fp64 = sizeof(T) == 8;
  const int n = ctx->n;
  const int M = ctx->n_mbf;
  const int pairs = M * M;
  const int nh = 2 * ctx->q_max + 1;
  const int cls_c = ctx->cls_computed;
  const int series_per_q = cls_c * pairs;
  const int series = series_per_q * nh;
  const double step = ctx->beta_max / n;
  const double beta_abs_max = std::hypot(ctx->beta_max, ctx->height);

  // ---- parameters
  int n_alpha = (int)ctx->opt[CFFT_OPT_N_ALPHA];
  if (n_alpha <= 0) {
    double need = 2.0 * beta_abs_max * ctx->elem_radius + 2.0 * ctx->q_max + 32.0;
    n_alpha = std::max(8, next_pow2((int)std::ceil(need)));
  }
  if (n_alpha % 4 != 0) return fail(ctx, CFFT_ERR_ARG, "n_alpha must be a multiple of 4");
  int sigma = (int)ctx->opt[CFFT_OPT_SIGMA];
  if (sigma <= 0) sigma = fp64 ? 8 : 4;
  if (sigma < 2 || (sigma & (sigma - 1))) return fail(ctx, CFFT_ERR_ARG, "sigma must be a power of two >= 2");
  const int bp_kern = choose_bp_kernel(fp64, ctx->opt[CFFT_OPT_BP_GATHER] > 0, (int)ctx->opt[CFFT_OPT_BP_TAPS],
                                       ctx->opt[CFFT_OPT_BP_KERNEL]);
  if (bp_kern < 0)
    return fail(ctx, CFFT_ERR_ARG,
                "the ES back-projection kernel needs FP32-mixed, the matrix form and 6 or 8 taps");
  const bool bp_es = bp_kern == 1;
  int bp_taps = (int)ctx->opt[CFFT_OPT_BP_TAPS];
  if (bp_taps <= 0) bp_taps = fp64 ? 16 : (bp_es ? 6 : 12);
  int fill_taps = (int)ctx->opt[CFFT_OPT_FILL_TAPS];
  if (fill_taps <= 0) fill_taps = fp64 ? 16 : 8;
  if (!(bp_taps == 4 || bp_taps == 6 || bp_taps == 8 || bp_taps == 10 || bp_taps == 12 ||
        bp_taps == 16 || bp_taps == 20 || bp_taps == 24) ||
      fill_taps < 2 || fill_taps > 16 || (fill_taps & 1))
    return fail(ctx, CFFT_ERR_ARG,
                "back-projection taps must be one of 4,6,8,10,12,16,20,24; fill taps even, 2..16");
  if (n_rho < 2 * fill_taps) return fail(ctx, CFFT_ERR_ARG, "n_rho must be >= 2 * fill taps");
  double margin = ctx->opt[CFFT_OPT_ALPHA_MARGIN] > 0 ? ctx->opt[CFFT_OPT_ALPHA_MARGIN] : 24.0;
  const SeriesChoice sc = choose_series(ctx->height * rho_max, fp64, ctx->taylor_req,
                                        ctx->opt[CFFT_OPT_CONTOUR_SERIES]);
  const int taylor = sc.order;
  if (taylor < 0)
    return fail(ctx, CFFT_ERR_ARG, "height * rho_max too large: no series order up to 64 converges");
  const int n_terms = taylor + (sc.series == 1 ? 2 : 1);
  const int64_t P = (int64_t)sigma * n;
  const double ds = 2.0 * kPi / ((double)P * step);
  const int K = (int)std::ceil(rho_max / ds) + bp_taps / 2 + 2;
  if (2 * (int64_t)K + 1 > P)
    return fail(ctx, CFFT_ERR_ARG, "rho_max exceeds the unaliased range 2 pi / step of the contour");
  // sub-FFT length: power of two dividing P, within shared memory
  const int l_max = fp64 ? 8192 : 16384;
  int L = 1;
  while ((P % (2 * (int64_t)L)) == 0 && 2 * L <= l_max) L *= 2;
  if (L < 64) return fail(ctx, CFFT_ERR_ARG, "sigma * n must be divisible by 64");
  while (L > 256 && (int64_t)series * (P / L) < 2 * ctx->sm_count) L /= 2;
  const double l_req = ctx->opt[CFFT_OPT_FFT_SUB_LEN];
  if (l_req > 0) {
    const int lr = (int)l_req;
    if ((double)lr != l_req || lr < 64 || lr > l_max || (lr & (lr - 1)) || P % lr != 0)
      return fail(ctx, CFFT_ERR_ARG, "FFT_SUB_LEN must be a power of two in 64.." + std::to_string(l_max) +
                                         " dividing sigma * n");
    L = lr;
  }
  int log2L = 0;
  while ((1 << log2L) < L) ++log2L;
  const int D = (int)(P / L);
  // nodes with beta_I > 0 form a prefix of the contour
  int n_active = (int)std::min<double>(n, std::ceil(ctx->beta_p / step - 0.5));
  if (ctx->height <= 0) n_active = 0;
  if (n_active < 0) n_active = 0;

  // ---- buffers
  CFFT_CUDA(ctx->beta_c.ensure(n * sizeof(double2)), "alloc contour");
  CFFT_CUDA(ctx->weight.ensure(n * sizeof(double2)), "alloc contour");
  CFFT_CUDA(ctx->bw.ensure(n * sizeof(double2)), "alloc contour");
  CFFT_CUDA(ctx->bi_rel.ensure(n * (sizeof(double) + sizeof(float)) + 16), "alloc contour");
  CFFT_CUDA(ctx->green_p.ensure(n * sizeof(double2)), "alloc contour");
  CFFT_CUDA(ctx->green_r.ensure(n * sizeof(double2)), "alloc contour");
  CFFT_CUDA(ctx->d_y.ensure((size_t)series * n * sizeof(cpx<T>)), "alloc harmonics");
  if (bp_es) CFFT_CUDA(ctx->d_prec.ensure((size_t)n * sizeof(float2)), "alloc precorrection");
  CFFT_CUDA(ctx->d_grid.ensure((size_t)series * (2 * K + 1) * sizeof(cpx<T>)), "alloc grid");
  const int cls_s = ctx->cls_stored;
  const int channels = ctx->opt[CFFT_OPT_DERIVATIVES] > 0 ? 3 : 1;
  const size_t table_elems = (size_t)cls_s * pairs * nh * n_rho;
  CFFT_CUDA(dst.ensure(channels * table_elems * sizeof(cpx<T>)), "alloc table");
  if (channels == 3) {
    CFFT_CUDA(ctx->dp_eps.ensure(n * sizeof(double2)), "alloc contour");
    CFFT_CUDA(ctx->dr_eps.ensure(n * sizeof(double2)), "alloc contour");
    CFFT_CUDA(ctx->dp_h.ensure(n * sizeof(double2)), "alloc contour");
    CFFT_CUDA(ctx->dr_h.ensure(n * sizeof(double2)), "alloc contour");
  }
  CFFT_CUDA(ctx->d_flag.ensure(sizeof(int) * 4), "alloc flag");
  CFFT_CUDA(cudaMemsetAsync(ctx->d_flag.as<int>() + 2, 0, sizeof(int), st), "flag");
  // MBF spectra on the tensor cores (FP32-mixed rooftop elements), unless disabled
  bool tc_spectra = false;
  if (!fp64 && !(ctx->opt[CFFT_OPT_SPECTRA_SIMT] > 0) && (n_alpha == 128 || n_alpha == 256)) {
    bool rooftop = true;
    for (const ShapeClass& c : ctx->shapes) rooftop = rooftop && c.kind == 0;
    if (rooftop && spectra_tc_columns((int)ctx->shapes.size(), ctx->n_mbf) > 0 && ctx->n_mbf <= 4)
      tc_spectra = ensure_tc_element(ctx) == CFFT_OK;
  }

  // element data in T
  {
    std::vector<T> hx(ctx->n_basis), hy(ctx->n_basis);
    std::vector<cpx<T>> hq((size_t)ctx->n_basis * ctx->n_mbf_pad);
    for (int i = 0; i < ctx->n_basis; ++i) {
      hx[i] = (T)ctx->bx[i];
      hy[i] = (T)ctx->by[i];
    }
    for (size_t i = 0; i < hq.size(); ++i) hq[i] = mk((T)ctx->q[i].real(), (T)ctx->q[i].imag());
    CFFT_CUDA(ctx->d_bx.ensure(hx.size() * sizeof(T)), "alloc element");
    CFFT_CUDA(ctx->d_by.ensure(hy.size() * sizeof(T)), "alloc element");
    CFFT_CUDA(ctx->d_q.ensure(hq.size() * sizeof(cpx<T>)), "alloc element");
    CFFT_CUDA(ctx->d_shapes.ensure(ctx->shapes.size() * sizeof(ShapeClass)), "alloc element");
    CFFT_CUDA(cudaMemcpyAsync(ctx->d_bx.p, hx.data(), hx.size() * sizeof(T), cudaMemcpyHostToDevice, st), "upload");
    CFFT_CUDA(cudaMemcpyAsync(ctx->d_by.p, hy.data(), hy.size() * sizeof(T), cudaMemcpyHostToDevice, st), "upload");
    CFFT_CUDA(cudaMemcpyAsync(ctx->d_q.p, hq.data(), hq.size() * sizeof(cpx<T>), cudaMemcpyHostToDevice, st), "upload");
    CFFT_CUDA(cudaMemcpyAsync(ctx->d_shapes.p, ctx->shapes.data(), ctx->shapes.size() * sizeof(ShapeClass),
                              cudaMemcpyHostToDevice, st), "upload");
    // the staging vectors die at scope end: wait for the copies
    CFFT_CUDA(cudaStreamSynchronize(st), "upload");
  }

  for (auto& e : ctx->ev)
    if (!e) CFFT_CUDA(cudaEventCreate(&e), "event");
  CFFT_CUDA(cudaEventRecord(ctx->ev[0], st), "event");

  // ---- a1: contour + Green's function (float64)
  ContourArgs ca{n, ctx->beta_max, ctx->beta_p, ctx->height, step, ctx->eps_r, ctx->hs, ctx->k0};
  set_extraction(ctx, ctx->eps_r, &ca.extract, &ca.eps_eff, &ca.deps_eff);
  ContourData cd{ctx->beta_c.as<double2>(), ctx->weight.as<double2>(), ctx->bw.as<double2>(),
                 ctx->bi_rel.as<double>(), reinterpret_cast<float*>(ctx->bi_rel.as<double>() + n),
                 ctx->green_p.as<double2>(), ctx->green_r.as<double2>(),
                 nullptr, nullptr, nullptr, nullptr, nullptr};
  if (bp_es) {
    ca.es_width = bp_taps;
    ca.ds = ds;
    cd.prec = ctx->d_prec.as<float2>();
  }
  if (channels == 3) {
    cd.dp_eps = ctx->dp_eps.as<double2>();
    cd.dr_eps = ctx->dr_eps.as<double2>();
    cd.dp_h = ctx->dp_h.as<double2>();
    cd.dr_h = ctx->dr_h.as<double2>();
  }
  int launches = 0;
  launch_contour(ca, cd, st);
  ++launches;
  CFFT_CUDA(cudaGetLastError(), "contour kernel");
  CFFT_CUDA(cudaEventRecord(ctx->ev[1], st), "event");

  double bp_nodes = 0, bp_macs = 0, bp_stencils = 0, tc_int_flops = 0, tc_bp_flops = 0;
  int bp_form_used = 0;
  bool in_tc = false, bp_tc = false;
  for (int ch = 0; ch < channels; ++ch) {
  // ---- a2/a3: spectra, kernel, harmonics
  IntegrandArgs<T> ia{};
  ia.n = n;
  ia.n_alpha = n_alpha;
  ia.q_max = ctx->q_max;
  ia.n_cls = cls_c;
  ia.n_mbf = M;
  ia.n_shape = (int)ctx->shapes.size();
  ia.n_basis = ctx->n_basis;
  ia.shapes = ctx->d_shapes.as<ShapeClass>();
  ia.bx = ctx->d_bx.as<T>();
  ia.by = ctx->d_by.as<T>();
  ia.q = ctx->d_q.as<cpx<T>>();
  ia.beta_c = ctx->beta_c.as<double2>();
  ia.bw = ctx->bw.as<double2>();
  const double2* gp_ch[3] = {ctx->green_p.as<double2>(), ctx->dp_eps.as<double2>(), ctx->dp_h.as<double2>()};
  const double2* gr_ch[3] = {ctx->green_r.as<double2>(), ctx->dr_eps.as<double2>(), ctx->dr_h.as<double2>()};
  ia.green_p = gp_ch[ch];
  ia.green_r = gr_ch[ch];
  ia.y = ctx->d_y.as<cpx<T>>();
  bool ran_tc = false;
  if constexpr (sizeof(T) == 4) {
    if (tc_spectra) {
      ia.tc_bx = ctx->tc_bx.as<float>();
      ia.tc_by = ctx->tc_by.as<float>();
      ia.tc_bmat = ctx->tc_bmat_mirror.as<float>();
      ia.tc_ncol = 2 * spectra_tc_columns((int)ctx->shapes.size(), ctx->n_mbf);
      ia.tc_rmax = ctx->tc_rmax;
      ia.err = ctx->d_flag.as<int>() + 2;
      if (integrand_tc_applies(ia)) {
        CFFT_CUDA(launch_integrand_tc(ia, st), "integrand kernel (tensor cores)");
        ran_tc = true;
        // executed: per CTA of integrand_tc_nodes contour nodes, 256 A rows x K = 4 per
        // (padded) basis function x tc_ncol columns, three TF32 products
        const int jt = integrand_tc_nodes(n_alpha);
        const double nb_pad = (double)((ctx->n_basis + kTcBasis - 1) / kTcBasis * kTcBasis);
        tc_int_flops += (double)((n + jt - 1) / jt) * 3.0 * 2.0 * 256.0 * 4.0 * nb_pad * ia.tc_ncol;
      }
    }
  }
  if (!ran_tc) CFFT_CUDA(launch_integrand<T>(ia, ctx->n_mbf_pad, st), "integrand kernel");
  in_tc = in_tc || ran_tc;
  ++launches;
  if (ch == 0) CFFT_CUDA(cudaEventRecord(ctx->ev[2], st), "event");

  // ---- a4: Taylor terms x pruned zero-padded FFTs
  const int prec_id = fp64 ? 1 : 0;
  if (ctx->tw_len != L || ctx->tw_prec != prec_id) {
    CFFT_CUDA(ctx->d_tw.ensure((size_t)L * sizeof(cpx<T>)), "alloc twiddles");
    launch_twiddle<T>(ctx->d_tw.as<cpx<T>>(), L, st);
    ++launches;
    CFFT_CUDA(cudaGetLastError(), "twiddle kernel");
    ctx->tw_len = L;
    ctx->tw_prec = prec_id;
  }
  FftArgs<T> fa{};
  fa.series = series;
  fa.n = n;
  fa.sub_len = L;
  fa.log2_sub = log2L;
  fa.n_sub = D;
  fa.fft_len = P;
  fa.grid_half = K;
  fa.taylor = taylor;
  fa.expansion = sc.series;
  fa.n_active = n_active;
  fa.sigma = sigma;
  fa.ds_height = ds * ctx->height;
  fa.y = ctx->d_y.as<cpx<T>>();
  fa.bi_rel = ctx->bi_rel.as<double>();
  fa.bi_rel_f = reinterpret_cast<const float*>(ctx->bi_rel.as<double>() + n);
  fa.twiddle = ctx->d_tw.as<cpx<T>>();
  if constexpr (sizeof(T) == 4) fa.prec = bp_es ? ctx->d_prec.as<cpx<float>>() : nullptr;
  fa.grid = ctx->d_grid.as<cpx<T>>();
  CFFT_CUDA(launch_fft<T>(fa, st), "fft kernel");
  ++launches;
  if (ch == 0) CFFT_CUDA(cudaEventRecord(ctx->ev[3], st), "event");

  // ---- a5: back-projection to the rho grid
  // the matrix-form back-projection handles up to 64 series per harmonic with 8/12/16 taps;
  // otherwise the direct gather form runs
  // FP32-mixed: the paired-harmonic matrix form (one interpolation matrix per |q|)
  const bool taps_ok = bp_es ? (bp_taps == 6 || bp_taps == 8) : (bp_taps == 8 || bp_taps == 12 || bp_taps == 16);
  const bool gather = ctx->opt[CFFT_OPT_BP_GATHER] > 0;
  const bool pform = !fp64 && taps_ok && !gather;
  const bool tform = pform && !(ctx->opt[CFFT_OPT_BP_SIMT] > 0);   // its products on the tensor cores
  const bool wform = !pform && series_per_q <= 64 && taps_ok && !gather;
  const int rchunk = pform ? backproject_pm_rows() : (wform ? backproject_w_rows() : 32);
  const int n_chunks = (n_rho + rchunk - 1) / rchunk;
  const double d_rho = rho_max / (n_rho - 1);
  std::vector<int> cn(n_chunks);
  std::vector<int64_t> coff(n_chunks);
  int64_t tot = 0;
  int max_nodes = 0, max_seg = 0;
  bp_nodes = 0;
  bp_macs = 0;
  bp_stencils = 0;
  // grid columns per matrix tile of the matrix forms
  const int ktile = tform ? backproject_tc_ktile() : (pform ? 32 : 64);
  for (int c = 0; c < n_chunks; ++c) {
    int r_top = std::min((c + 1) * rchunk, n_rho) - 1;
    double rho_top = r_top * d_rho;
    cn[c] = alpha_nodes(beta_abs_max, rho_top, ctx->q_max, margin, alpha_cbrt_coef(fp64));
    const int rows_c = r_top + 1 - c * rchunk;
    bp_nodes += (double)cn[c] * rows_c * series;
    if (pform || wform) {
      // matrix columns: both signs of k (matrix form) or k >= -(taps/2) with the grid folded
      // about k = 0 (paired-harmonic form, which also visits only the nodes alpha <= pi/2)
      const int kmax_c = std::min(K - 1, (int)std::ceil(rho_top / ds) + bp_taps);
      const int n_kt = pform ? (kmax_c + bp_taps / 2 + ktile) / ktile : (2 * kmax_c + ktile) / ktile;
      bp_macs += (double)rows_c * n_kt * ktile * series;
      if (tform)
        // executed: per row tile (rchunk rows), |q| and chunk of 16 series per sign, each
        // K-tile is a (rchunk x 2 ktile) x (2 ktile x 64) product, three TF32 products
        tc_bp_flops += 3.0 * 2.0 * rchunk * (2.0 * ktile) * 64.0 * n_kt * (ctx->q_max + 1) *
                       ((series_per_q + 15) / 16);
      const int n_mat = pform ? (ctx->q_max + 1) * ((series_per_q + 15) / 16) : nh;
      bp_stencils += (double)rows_c * (pform ? (cn[c] + 1) / 2 : cn[c]) * n_mat;
    }
    coff[c] = tot;
    tot += cn[c];
    max_nodes = std::max(max_nodes, cn[c]);
    int kseg = std::min(K, (int)std::ceil(rho_top / ds) + bp_taps / 2 + 2);
    max_seg = std::max(max_seg, 2 * kseg + 1);
  }
  std::vector<double> lag(bp_taps);
  for (int m = 0; m < bp_taps; ++m) {
    double den = std::exp(lgamma_fact(m) + lgamma_fact(bp_taps - 1 - m));
    lag[m] = (((bp_taps - 1 - m) & 1) ? -1.0 : 1.0) / den;
  }
  CFFT_CUDA(ctx->d_cnodes.ensure(n_chunks * sizeof(int)), "alloc bp");
  CFFT_CUDA(ctx->d_coff.ensure(n_chunks * sizeof(int64_t)), "alloc bp");
  CFFT_CUDA(ctx->d_cos.ensure(tot * sizeof(double)), "alloc bp");
  CFFT_CUDA(ctx->d_lag.ensure(bp_taps * sizeof(double)), "alloc bp");
  CFFT_CUDA(cudaMemcpyAsync(ctx->d_cnodes.p, cn.data(), n_chunks * sizeof(int), cudaMemcpyHostToDevice, st), "upload");
  CFFT_CUDA(cudaMemcpyAsync(ctx->d_coff.p, coff.data(), n_chunks * sizeof(int64_t), cudaMemcpyHostToDevice, st), "upload");
  CFFT_CUDA(cudaMemcpyAsync(ctx->d_lag.p, lag.data(), bp_taps * sizeof(double), cudaMemcpyHostToDevice, st), "upload");
  if (ch == 0) {
    CFFT_CUDA(launch_chunk_cosines(ctx->d_cnodes.as<int>(), ctx->d_coff.as<int64_t>(), n_chunks,
                                   max_nodes, ctx->d_cos.as<double>(), st), "cosine kernel");
    ++launches;
  }
  int group = 8;
  const size_t smem_cap = 225 * 1024;
  while (group > 1 && backproject_smem<T>(group, max_seg, max_nodes) > smem_cap) --group;
  if (!wform && backproject_smem<T>(group, max_seg, max_nodes) > smem_cap)
    return fail(ctx, CFFT_ERR_ARG, "rho_max too large for one shared-memory segment");
  if (wform && backproject_w_smem<T>(max_nodes, series_per_q) > smem_cap)
    return fail(ctx, CFFT_ERR_ARG, "rho_max too large for the angular node table");
  if (pform && (tform ? backproject_tc_smem(max_nodes) : backproject_pm_smem(max_nodes)) > smem_cap)
    return fail(ctx, CFFT_ERR_ARG, "rho_max too large for the angular node table");
  group = std::min(group, series_per_q);
  BackprojArgs<T> ba{};
  ba.series_per_q = series_per_q;
  ba.n_harm = nh;
  ba.q_max = ctx->q_max;
  ba.n_rho = n_rho;
  ba.grid_half = K;
  ba.sigma = sigma;
  ba.taps = bp_taps;
  ba.group = group;
  ba.rchunk = rchunk;
  ba.d_rho = d_rho;
  ba.d_s = ds;
  ba.beta_abs_max = beta_abs_max;
  ba.alpha_margin = margin;
  ba.grid = ctx->d_grid.as<cpx<T>>();
  ba.table = dst.as<cpx<T>>() + ch * table_elems;
  ba.kern = bp_es ? 1 : 0;
  bp_form_used = tform ? 3 : (pform ? 2 : (wform ? 1 : 0));
  if (pform || wform) {
    ba.chunk_nodes = ctx->d_cnodes.as<int>();
    ba.chunk_off = ctx->d_coff.as<int64_t>();
    ba.cosv = ctx->d_cos.as<double>();
    if constexpr (sizeof(T) == 4) {
      if (tform) {
        ba.err = ctx->d_flag.as<int>() + 2;
        CFFT_CUDA(launch_backproject_tc(ba, n_chunks, max_nodes, st), "backprojection kernel (tensor cores)");
        bp_tc = true;
      } else if (pform) {
        CFFT_CUDA(launch_backproject_pm(ba, n_chunks, max_nodes, st), "backprojection kernel");
      } else {
        CFFT_CUDA(launch_backproject_w<T>(ba, n_chunks, max_nodes, st), "backprojection kernel");
      }
    } else {
      CFFT_CUDA(launch_backproject_w<T>(ba, n_chunks, max_nodes, st), "backprojection kernel");
    }
  } else {
    CFFT_CUDA(launch_backproject_impl<T>(ba, ctx->d_cnodes.as<int>(), ctx->d_coff.as<int64_t>(),
                                         ctx->d_cos.as<double>(), ctx->d_lag.as<double>(), n_chunks,
                                         max_nodes, max_seg, st), "backprojection kernel");
  }
  ++launches;
  if (cls_s == 4) {
    launch_class_phase<T>(dst.as<cpx<T>>() + ch * table_elems, pairs, nh, ctx->q_max, n_rho, st);
    ++launches;
    CFFT_CUDA(cudaGetLastError(), "class phase kernel");
  }
  }
  CFFT_CUDA(cudaEventRecord(ctx->ev[4], st), "event");

  // ---- NaN / Inf check (synchronizes)
  bool check = !(ctx->opt[CFFT_OPT_CHECK_FINITE] < 0);
  if (check) {
    CFFT_CUDA(cudaMemsetAsync(ctx->d_flag.p, 0, sizeof(int), st), "flag");
    launch_nonfinite<T>(dst.as<cpx<T>>(), (int64_t)(channels * table_elems), ctx->d_flag.as<int>(), st);
    ++launches;
    CFFT_CUDA(cudaGetLastError(), "nonfinite kernel");
  }
  int flag = 0, tc_flag = 0;
  if (check) CFFT_CUDA(cudaMemcpyAsync(&flag, ctx->d_flag.p, sizeof(int), cudaMemcpyDeviceToHost, st), "flag");
  if (in_tc || bp_tc) CFFT_CUDA(cudaMemcpyAsync(&tc_flag, ctx->d_flag.as<int>() + 2, sizeof(int), cudaMemcpyDeviceToHost, st), "flag");
  CFFT_CUDA(cudaStreamSynchronize(st), "tabulate");
  if (tc_flag & 16) return fail(ctx, CFFT_ERR_TIMEOUT, "integrand: a tensor-core wait ran past its bound");
  if (tc_flag & 32) return fail(ctx, CFFT_ERR_TIMEOUT, "back-projection: a tensor-core wait ran past its bound");

  cfft_info scratch_info{};
  cfft_info& in = primary ? ctx->info : scratch_info;
  in.taylor_order = taylor;
  in.contour_series = sc.series;
  in.n_alpha = n_alpha;
  in.sigma = sigma;
  in.fft_len = (int)P;
  in.sub_len = L;
  in.grid_half = K;
  in.bp_taps = bp_taps;
  in.bp_kernel = bp_es ? 1 : 0;
  in.fill_taps = fill_taps;
  in.series = series;
  in.classes = cls_s;
  in.n_pairs = pairs;
  in.n_harm = nh;
  in.delta_s = ds;
  float ms = 0;
  cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
  in.ms_contour = ms;
  cudaEventElapsedTime(&ms, ctx->ev[1], ctx->ev[2]);
  in.ms_integrand = ms;
  cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]);
  in.ms_fft = ms;
  cudaEventElapsedTime(&ms, ctx->ev[3], ctx->ev[4]);
  in.ms_backproject = ms;
  in.launches = launches;
  in.n_basis = ctx->n_basis;
  in.work_points = (double)n * n_alpha;
  in.work_subffts = (double)series * D * n_terms;
  in.work_bp_nodes = bp_nodes;
  in.spectra_tc = in_tc ? 1 : 0;
  in.bp_form = bp_form_used;
  in.work_bp_macs = bp_macs;
  in.work_bp_stencils = bp_stencils;
  in.tc_flops_integrand = tc_int_flops;
  in.tc_flops_backproject = tc_bp_flops;
  in.fill_err_est = -1.0;
  in.fill_refine = 0;
  in.fill_n_rho = 0;
  if (flag) return fail(ctx, CFFT_ERR_NUMERIC, "non-finite value in the reaction table");
  if (primary) {
    ctx->fill_taps = fill_taps;
    ctx->channels = channels;
    ctx->has_table = true;
  }
  return CFFT_OK;
}

// largest |prod_{t=0}^{p-1} (x - t)| / p! over x in [x0, x1] (the Lagrange remainder's
// node polynomial of a p-tap stencil), by dense sampling of the interval
double lagrange_node_factor(int p, double x0, double x1) {
  double best = 0.0;
  const int steps = 4096;
  for (int k = 0; k <= steps; ++k) {
    const double x = x0 + (x1 - x0) * k / steps;
    double prod = 1.0;
    for (int t = 0; t < p; ++t) prod *= (x - t);
    best = std::max(best, std::fabs(prod));
  }
  return best / std::exp(lgamma_fact(p));
}

// Decide, once per table, which table the fill interpolates.  The fill targets the
// precision's tolerance (1e-10 of the table maximum in FP64, 1e-5 in FP32-mixed, per
// (class, pair)); the interpolation may use a quarter of it.  The a posteriori estimate
// (the p-th differences of the table, launch_fill_estimate) bounds the interpolation
// error on the tabulated grid, for the interior stencils and for the last one, which is
// shifted inward at rho_max (its node polynomial is far larger).  When either misses that
// share, the same tabulation runs again on a grid finer by the integer factor r (interior
// error falling like r^-p) that reaches p/2 rows beyond rho_max, so that the stencil of
// every pair up to rho_max is centred, and the fill uses that table.  A loaded table cannot
// be tabulated again: it is refused instead.  CFFT_OPT_FILL_REFINE >= 1 fixes r (1: the
// tabulated grid as it is, no estimate).
template <class T>
cfft_status ensure_fill_table_t(cfft_ctx* ctx) {
  if (ctx->fill_r > 0) return CFFT_OK;
  cudaStream_t st = ctx->stream;
  const int p = ctx->fill_taps;
  const int nh = 2 * ctx->q_max + 1;
  const int forced = (int)std::lround(ctx->opt[CFFT_OPT_FILL_REFINE]);
  double est_c = -1.0, est_e = -1.0;
  int r = 1;
  bool own = false;   // the fill gets a table of its own (finer and/or extended)
  const double share = 0.25 * (ctx->prec == CFFT_FP64 ? 1e-10 : 1e-5);
  if (forced >= 1) {
    r = forced;
    own = r > 1;
  } else {
    // the table itself (channel 0): the derivative tables share its grid and integrand
    const int64_t groups = (int64_t)ctx->cls_stored * ctx->n_mbf * ctx->n_mbf;
    const int64_t n_series = groups * nh;
    CFFT_CUDA(ctx->d_fest.ensure((size_t)n_series * sizeof(double4)), "alloc fill estimate");
    const double fac_c = lagrange_node_factor(p, 0.5 * p - 1.0, 0.5 * p);
    const double fac_e = lagrange_node_factor(p, 0.5 * p - 1.0, p - 1.0);
    CFFT_CUDA(launch_fill_estimate<T>(ctx->d_table.p, n_series, ctx->n_rho, ctx->q_max, p, fac_c, fac_e,
                                      ctx->d_fest.as<double4>(), st), "fill estimate kernel");
    std::vector<double4> h((size_t)n_series);
    CFFT_CUDA(cudaMemcpyAsync(h.data(), ctx->d_fest.p, h.size() * sizeof(double4), cudaMemcpyDeviceToHost, st),
              "fill estimate");
    CFFT_CUDA(cudaStreamSynchronize(st), "fill estimate");
    est_c = 0.0;
    est_e = 0.0;
    for (int64_t g = 0; g < groups; ++g) {
      double zmax = 0.0, ec = 0.0, ee = 0.0;
      for (int q = 0; q < nh; ++q) {
        const double4& v = h[(size_t)(g * nh + q)];
        zmax = std::max(zmax, v.x);
        ec = std::max(ec, v.y);
        ee = std::max(ee, v.z);
      }
      if (zmax > 0.0) {
        est_c = std::max(est_c, ec / zmax);
        est_e = std::max(est_e, ee / zmax);
      }
    }
    if (std::max(est_c, est_e) > share) {
      own = true;
      // aim the interior at a quarter of the share, so that the finer grid keeps a margin
      if (est_c > 0.25 * share) r = (int)std::ceil(std::pow(4.0 * est_c / share, 1.0 / p) - 1e-9);
      r = std::max(r, 1);
    }
  }
  ctx->info.fill_err_est = std::max(est_c, est_e);
  const int ext = own ? p / 2 : 0;   // rows beyond rho_max
  const int64_t n_f = (int64_t)(ctx->n_rho - 1) * r + 1 + ext;
  if (own && ctx->table_loaded)
    return fail(ctx, CFFT_ERR_ARG,
                "the loaded table's rho grid misses the fill's target (estimated interpolation error " +
                std::to_string(est_c) + " inside, " + std::to_string(est_e) +
                " at rho_max, of the table maximum): load a table on a finer grid that reaches " +
                std::to_string(p / 2) + " rows beyond the largest element distance, or set "
                "CFFT_OPT_FILL_REFINE = 1 to fill on this grid");
  if (n_f > (1 << 20))
    return fail(ctx, CFFT_ERR_ARG, "the fill needs a table of " + std::to_string(n_f) +
                " rho points (more than 1048576): tabulate to a smaller rho_max or raise the fill taps");
  const double d_f = ctx->rho_max / ((double)(ctx->n_rho - 1) * r);
  const double rho_f = d_f * (double)(n_f - 1);
  if (own) {
    // the same tabulation on the fill's grid, with the options the table was made with
    double saved[kNumOptions];
    std::memcpy(saved, ctx->opt, sizeof(saved));
    std::memcpy(ctx->opt, ctx->tab_opt, sizeof(saved));
    cfft_status stt = tabulate_impl<T>(ctx, (int)n_f, rho_f, ctx->d_ftable, false);
    std::memcpy(ctx->opt, saved, sizeof(saved));
    if (stt != CFFT_OK) return stt;
  }
  ctx->fill_r = r;
  ctx->fill_own = own;
  ctx->n_frho = own ? (int)n_f : ctx->n_rho;
  ctx->frho_max = own ? rho_f : ctx->rho_max;
  ctx->info.fill_refine = r;
  ctx->info.fill_n_rho = ctx->n_frho;
  return CFFT_OK;
}

cfft_status ensure_fill_table(cfft_ctx* ctx) {
  return ctx->prec == CFFT_FP64 ? ensure_fill_table_t<double>(ctx) : ensure_fill_table_t<float>(ctx);
}

// the table the fill and its adjoint interpolate
template <class T>
const cpx<T>* fill_table(const cfft_ctx* ctx) {
  return (ctx->fill_own ? ctx->d_ftable : ctx->d_table).template as<cpx<T>>();
}

template <class T, class TO>
cfft_status fill_impl(cfft_ctx* ctx, int n_el, const double* pos, const int* rot, void* z,
                      int64_t ld) {
  cfft_status fs = ensure_fill_table(ctx);
  if (fs != CFFT_OK) return fs;
  FillArgs<T, TO> fa{};
  fa.n_el = n_el;
  fa.n_mbf = ctx->n_mbf;
  fa.q_max = ctx->q_max;
  fa.n_harm = 2 * ctx->q_max + 1;
  fa.n_rho = ctx->n_frho;
  fa.taps = ctx->fill_taps;
  fa.n_cls = ctx->cls_stored;
  fa.inv_d_rho = (ctx->n_frho - 1) / ctx->frho_max;
  fa.rho_max = ctx->rho_max;
  fa.ld = ld;
  fa.table = fill_table<T>(ctx);
  fa.pos = pos;
  fa.rot = rot;
  fa.z = reinterpret_cast<cpx<TO>*>(z);
  CFFT_CUDA(ctx->d_flag.ensure(sizeof(int) * 4), "alloc flag");   // a loaded table skips tabulation
  fa.err = ctx->d_flag.as<int>() + 1;
  FillBucketPlan plan{};
  plan.ok = false;
  if (std::is_same<T, TO>::value && ctx->opt[CFFT_OPT_FILL_BLOCK] >= 0)
    plan = plan_fill_bucketed<T>(n_el, fa.n_mbf, fa.n_harm, fa.n_rho, fa.taps, fa.n_cls,
                                 (int)ctx->opt[CFFT_OPT_FILL_BLOCK], !(ctx->opt[CFFT_OPT_FILL_SIMT] > 0));
  if (plan.ok) CFFT_CUDA(ctx->d_fill.ensure(plan.scratch), "alloc fill scratch");
  CFFT_CUDA(cudaMemsetAsync(fa.err, 0, sizeof(int), ctx->stream), "flag");
  ctx->info.fill_form = plan.ok ? (plan.tc ? 3 : 2) : 1;
  cudaError_t le = launch_fill<T, TO>(fa, plan, ctx->d_fill.p, ctx->stream);
  if (le != cudaSuccess) return cuda_fail(ctx, le, "fill kernel");
  int flag = 0;
  CFFT_CUDA(cudaMemcpyAsync(&flag, fa.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "flag");
  CFFT_CUDA(cudaStreamSynchronize(ctx->stream), "fill");
  if (flag & 16) return fail(ctx, CFFT_ERR_TIMEOUT, "fill: a tensor-core wait ran past its bound");
  if (flag & 2) return fail(ctx, CFFT_ERR_NUMERIC, "fill: a stencil left its bucket (internal error)");
  if (flag) return fail(ctx, CFFT_ERR_ARG, "an element pair lies beyond the table's rho_max");
  return CFFT_OK;
}

template <class T, class TG>
cfft_status fill_backward_impl(cfft_ctx* ctx, int n_el, const double* pos, const int* rot,
                               const void* grad, int64_t ld_g, double* grad_pos, double* grad_theta) {
  cfft_status fs = ensure_fill_table(ctx);
  if (fs != CFFT_OK) return fs;
  FillBackArgs<T, TG> b{};
  FillArgs<T, float>& fa = b.f;
  fa.n_el = n_el;
  fa.n_mbf = ctx->n_mbf;
  fa.q_max = ctx->q_max;
  fa.n_harm = 2 * ctx->q_max + 1;
  fa.n_rho = ctx->n_frho;
  fa.taps = ctx->fill_taps;
  fa.n_cls = ctx->cls_stored;
  fa.inv_d_rho = (ctx->n_frho - 1) / ctx->frho_max;
  fa.rho_max = ctx->rho_max;
  fa.ld = 0;
  fa.table = fill_table<T>(ctx);
  fa.pos = pos;
  fa.rot = rot;
  fa.z = nullptr;
  CFFT_CUDA(ctx->d_flag.ensure(sizeof(int) * 4), "alloc flag");   // a loaded table skips tabulation
  fa.err = ctx->d_flag.as<int>() + 1;
  const size_t table_elems = (size_t)ctx->cls_stored * ctx->n_mbf * ctx->n_mbf * fa.n_harm * ctx->n_frho;
  if (ctx->channels == 3) {
    b.dtab_eps = fa.table + table_elems;
    b.dtab_h = fa.table + 2 * table_elems;
  }
  b.grad = reinterpret_cast<const cpx<TG>*>(grad);
  b.ld_g = ld_g;
  b.d_rho = ctx->frho_max / (ctx->n_frho - 1);
  b.grad_pos = grad_pos;
  b.grad_theta = grad_theta;
  CFFT_CUDA(cudaMemsetAsync(fa.err, 0, sizeof(int), ctx->stream), "flag");
  if (grad_pos) CFFT_CUDA(cudaMemsetAsync(grad_pos, 0, (size_t)2 * n_el * sizeof(double), ctx->stream), "zero");
  if (grad_theta) CFFT_CUDA(cudaMemsetAsync(grad_theta, 0, 2 * sizeof(double), ctx->stream), "zero");
  cudaError_t le = cudaSuccess;
  bool bucketed = false;
  if constexpr (std::is_same<T, TG>::value) {
    // the adjoint over the fill's buckets (same plan and scratch as the fill)
    FillBucketPlan plan{};
    if (ctx->opt[CFFT_OPT_FILL_BLOCK] >= 0)
    {
      // the tensor-core adjoint stages each stencil cell's table slice three times (position
      // and two substrate passes): it pays from about 512 pairs per cell (class) upwards
      const double per_cell = (double)n_el * n_el / ((double)fa.n_cls * fa.n_rho);
      const double sel = ctx->opt[CFFT_OPT_FILL_SIMT];
      const bool tc = sel < 0 || (sel == 0 && per_cell >= 512.0);
      plan = plan_fill_bucketed<T>(n_el, fa.n_mbf, fa.n_harm, fa.n_rho, fa.taps, fa.n_cls,
                                   (int)ctx->opt[CFFT_OPT_FILL_BLOCK], tc);
    }
    if (plan.ok) {
      CFFT_CUDA(ctx->d_fill.ensure(plan.scratch), "alloc fill scratch");
      FillArgs<T, T> ft{};
      ft.n_el = fa.n_el;
      ft.n_mbf = fa.n_mbf;
      ft.q_max = fa.q_max;
      ft.n_harm = fa.n_harm;
      ft.n_rho = fa.n_rho;
      ft.taps = fa.taps;
      ft.n_cls = fa.n_cls;
      ft.inv_d_rho = fa.inv_d_rho;
      ft.rho_max = fa.rho_max;
      ft.ld = 0;
      ft.table = fa.table;
      ft.pos = fa.pos;
      ft.rot = fa.rot;
      ft.z = nullptr;
      ft.err = fa.err;
      FillAdjointArgs<T> ad{};
      ad.grad = b.grad;
      ad.ld_g = ld_g;
      ad.dtab_eps = b.dtab_eps;
      ad.dtab_h = b.dtab_h;
      ad.grad_pos = grad_pos;
      ad.grad_theta = grad_theta;
      le = launch_fill_adjoint_bucketed<T>(ft, ad, plan, ctx->d_fill.p, ctx->stream);
      bucketed = true;
    }
  }
  if (!bucketed) le = launch_fill_backward<T, TG>(b, ctx->stream);
  if (le != cudaSuccess) return cuda_fail(ctx, le, "fill backward kernel");
  int flag = 0;
  CFFT_CUDA(cudaMemcpyAsync(&flag, fa.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "flag");
  CFFT_CUDA(cudaStreamSynchronize(ctx->stream), "fill backward");
  if (flag & 16) return fail(ctx, CFFT_ERR_TIMEOUT, "fill adjoint: a tensor-core wait ran past its bound");
  if (flag & 2) return fail(ctx, CFFT_ERR_NUMERIC, "fill adjoint: a stencil left its bucket (internal error)");
  if (flag) return fail(ctx, CFFT_ERR_ARG, "an element pair lies beyond the table's rho_max");
  return CFFT_OK;
}

cfft_status fill_dispatch(cfft_ctx* ctx, int n_el, const double* pos, const int* rot, void* z,
                          int64_t ld, int out128) {
  const bool t64 = ctx->prec == CFFT_FP64;
  if (t64 && out128) return fill_impl<double, double>(ctx, n_el, pos, rot, z, ld);
  if (t64) return fill_impl<double, float>(ctx, n_el, pos, rot, z, ld);
  if (out128) return fill_impl<float, double>(ctx, n_el, pos, rot, z, ld);
  return fill_impl<float, float>(ctx, n_el, pos, rot, z, ld);
}

cfft_status check_fill_args(cfft_ctx* ctx, int n_el, const double* pos, const int* rot,
                            void* z, int64_t ld) {
  if (!ctx) return CFFT_ERR_ARG;
  if (!ctx->has_table) return fail(ctx, CFFT_ERR_STATE, "fill before tabulate_reactions");
  if (n_el < 1 || n_el > 65535) return fail(ctx, CFFT_ERR_ARG, "n_elements must be in 1..65535");
  if (!pos || !z) return fail(ctx, CFFT_ERR_ARG, "null pointer");
  if (ld < (int64_t)n_el * ctx->n_mbf) return fail(ctx, CFFT_ERR_ARG, "ld < n_elements * M");
  if (ctx->cls_stored == 4 && !rot) return fail(ctx, CFFT_ERR_ARG, "rot is required with 4 rotation classes");
  return CFFT_OK;
}

// ---------------------------------------------------------------------------
// Batched sweep: many (substrate, frequency) items of one element, every stage
// one persistent or multi-item launch over all items of a wave, the whole
// sequence captured once into a CUDA graph and replayed.

struct BatchItemPlan {
  int n, taylor, series, n_active, K, D;
  int na_need;   // angular samples the item's own spectra need (a power of two)
  int64_t P;
  double step, ds, beta_abs;
};

constexpr size_t kWaveScratch = size_t(24) << 30;  // Y + grid bytes per wave

template <class T>
cfft_status batch_impl(cfft_ctx* ctx, int n_items, const cfft_batch_item* items, int q_max,
                       double rho_max, int n_rho, void* tables, int flags) {
  const bool fp64 = sizeof(T) == 8;
  const int M = ctx->n_mbf;
  const int pairs = M * M;
  const int nh = 2 * q_max + 1;
  const int series = pairs * nh;
  const int sigma = ctx->opt[CFFT_OPT_SIGMA] > 0 ? (int)ctx->opt[CFFT_OPT_SIGMA] : (fp64 ? 8 : 4);
  if (sigma < 2 || (sigma & (sigma - 1))) return fail(ctx, CFFT_ERR_ARG, "sigma must be a power of two >= 2");
  const int bp_kern = choose_bp_kernel(fp64, false, (int)ctx->opt[CFFT_OPT_BP_TAPS], ctx->opt[CFFT_OPT_BP_KERNEL]);
  if (bp_kern < 0)
    return fail(ctx, CFFT_ERR_ARG, "batch: the ES back-projection kernel needs FP32-mixed and 6 or 8 taps");
  const bool bp_es = bp_kern == 1;
  const int bp_taps = ctx->opt[CFFT_OPT_BP_TAPS] > 0 ? (int)ctx->opt[CFFT_OPT_BP_TAPS] : (fp64 ? 16 : (bp_es ? 6 : 12));
  if (bp_es ? (bp_taps != 6 && bp_taps != 8) : (bp_taps != 8 && bp_taps != 12 && bp_taps != 16))
    return fail(ctx, CFFT_ERR_ARG, "batched back-projection taps must be 8, 12 or 16 (6 or 8 with the ES kernel)");
  const bool pform_b = !fp64;  // paired-harmonic matrix form in FP32-mixed
  // its products on the tensor cores (unless disabled; the autotuner may choose the FP32 pipe)
  bool tform_b = pform_b && !(ctx->opt[CFFT_OPT_BP_SIMT] > 0);
  const double margin = ctx->opt[CFFT_OPT_ALPHA_MARGIN] > 0 ? ctx->opt[CFFT_OPT_ALPHA_MARGIN] : 24.0;
  const double d_rho = rho_max / (n_rho - 1);
  const size_t table_elems = (size_t)pairs * nh * n_rho;
  cudaStream_t st = ctx->bstream;

  // ---- per-item parameters (same rules as the single tabulation)
  std::vector<BatchItemPlan> ip(n_items);
  int n_alpha = (int)ctx->opt[CFFT_OPT_N_ALPHA];
  int l_common = fp64 ? 8192 : 16384;
  for (int i = 0; i < n_items; ++i) {
    const cfft_batch_item& it = items[i];
    BatchItemPlan& p = ip[i];
    p.n = it.n;
    p.step = it.beta_max / it.n;
    p.beta_abs = std::hypot(it.beta_max, it.height);
    const SeriesChoice sc = choose_series(it.height * rho_max, fp64, it.taylor_order,
                                          ctx->opt[CFFT_OPT_CONTOUR_SERIES]);
    p.taylor = sc.order;
    p.series = sc.series;
    if (p.taylor < 0)
      return fail(ctx, CFFT_ERR_ARG, "batch item: height * rho_max too large for the contour-factor series");
    p.P = (int64_t)sigma * it.n;
    p.ds = 2.0 * kPi / ((double)p.P * p.step);
    p.K = (int)std::ceil(rho_max / p.ds) + bp_taps / 2 + 2;
    if (2 * (int64_t)p.K + 1 > p.P)
      return fail(ctx, CFFT_ERR_ARG, "batch item: rho_max exceeds the unaliased range of its contour");
    p.n_active = it.height > 0 ? (int)std::min<double>(it.n, std::ceil(it.beta_p / p.step - 0.5)) : 0;
    int lp = 1;
    while ((p.P % (2 * (int64_t)lp)) == 0 && 2 * lp <= l_common) lp *= 2;
    l_common = std::min(l_common, lp);
    p.na_need = 0;
    if (ctx->opt[CFFT_OPT_N_ALPHA] <= 0) {
      double need = 2.0 * p.beta_abs * ctx->elem_radius + 2.0 * q_max + 32.0;
      p.na_need = std::max(8, next_pow2((int)std::ceil(need)));
      n_alpha = std::max(n_alpha, p.na_need);
    }
  }
  if (l_common < 1024) return fail(ctx, CFFT_ERR_ARG, "batch: sigma * n must be divisible by 1024");
  if (n_alpha % 4 != 0) return fail(ctx, CFFT_ERR_ARG, "n_alpha must be a multiple of 4");

  // ---- signature (graph and tuning cache key)
  std::string sig = std::to_string(n_items) + ":" + std::to_string(q_max) + ":" + std::to_string(n_rho) +
                    ":" + std::to_string(rho_max) + ":" + std::to_string(sizeof(T)) + ":" +
                    std::to_string(n_alpha) + ":" + std::to_string((size_t)tables) + ":" +
                    std::to_string(ctx->n_basis) + ":" + std::to_string(M) + ":" + std::to_string(bp_taps) + ":" +
                    std::to_string(bp_kern);
  for (int i = 0; i < n_items; ++i)
    sig += ":" + std::to_string(ip[i].n) + "/" + std::to_string(ip[i].taylor) + "/" + std::to_string(ip[i].series) +
           "/" + std::to_string(ip[i].na_need);

  // ---- element data in T (shared by all items)
  {
    std::vector<T> hx(ctx->n_basis), hy(ctx->n_basis);
    std::vector<cpx<T>> hq((size_t)ctx->n_basis * ctx->n_mbf_pad);
    for (int i = 0; i < ctx->n_basis; ++i) {
      hx[i] = (T)ctx->bx[i];
      hy[i] = (T)ctx->by[i];
    }
    for (size_t i = 0; i < hq.size(); ++i) hq[i] = mk((T)ctx->q[i].real(), (T)ctx->q[i].imag());
    CFFT_CUDA(ctx->d_bx.ensure(hx.size() * sizeof(T)), "alloc element");
    CFFT_CUDA(ctx->d_by.ensure(hy.size() * sizeof(T)), "alloc element");
    CFFT_CUDA(ctx->d_q.ensure(hq.size() * sizeof(cpx<T>)), "alloc element");
    CFFT_CUDA(ctx->d_shapes.ensure(ctx->shapes.size() * sizeof(ShapeClass)), "alloc element");
    CFFT_CUDA(cudaMemcpy(ctx->d_bx.p, hx.data(), hx.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
    CFFT_CUDA(cudaMemcpy(ctx->d_by.p, hy.data(), hy.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
    CFFT_CUDA(cudaMemcpy(ctx->d_q.p, hq.data(), hq.size() * sizeof(cpx<T>), cudaMemcpyHostToDevice), "upload");
    CFFT_CUDA(cudaMemcpy(ctx->d_shapes.p, ctx->shapes.data(), ctx->shapes.size() * sizeof(ShapeClass),
                         cudaMemcpyHostToDevice), "upload");
  }

  // ---- waves: consecutive items whose harmonics + transform grids fit the wave scratch
  struct Wave { int i0, i1; };
  std::vector<Wave> waves;
  size_t max_nodes_wave = 0, max_y = 0, max_grid = 0;
  {
    int i0 = 0;
    size_t nodes = 0, yb = 0, gb = 0;
    for (int i = 0; i < n_items; ++i) {
      size_t yi = (size_t)series * ip[i].n * sizeof(cpx<T>);
      size_t gi = (size_t)series * (2 * ip[i].K + 1) * sizeof(cpx<T>);
      if (i > i0 && yb + gb + yi + gi > kWaveScratch) {
        waves.push_back({i0, i});
        i0 = i;
        nodes = yb = gb = 0;
      }
      nodes += ip[i].n;
      yb += yi;
      gb += gi;
      max_nodes_wave = std::max(max_nodes_wave, nodes);
      max_y = std::max(max_y, yb);
      max_grid = std::max(max_grid, gb);
    }
    waves.push_back({i0, n_items});
  }
  CFFT_CUDA(ctx->b_contour.ensure(max_nodes_wave * (4 * sizeof(double2) + sizeof(double) + sizeof(double2) + 64)), "alloc batch contour");
  CFFT_CUDA(ctx->b_y.ensure(max_y), "alloc batch harmonics");
  CFFT_CUDA(ctx->b_grid.ensure(max_grid), "alloc batch grid");

  // contour buffers carved from b_contour: beta_c, weight, bw, green_p, green_r (double2), bi_rel (double)
  double2* c_beta = ctx->b_contour.as<double2>();
  double2* c_w = c_beta + max_nodes_wave;
  double2* c_bw = c_w + max_nodes_wave;
  double2* c_gp = c_bw + max_nodes_wave;
  double2* c_gr = c_gp + max_nodes_wave;
  double* c_bi = reinterpret_cast<double*>(c_gr + max_nodes_wave);
  float* c_bif = reinterpret_cast<float*>(c_bi + max_nodes_wave);
  float2* c_prec = reinterpret_cast<float2*>(c_bif + max_nodes_wave + (max_nodes_wave & 1));

  // integrand tile height (the same element and n_alpha for every item)
  IntegrandArgs<T> shape_args{};
  shape_args.n_alpha = n_alpha;
  shape_args.n_mbf = M;
  shape_args.n_basis = ctx->n_basis;
  int jt = integrand_tile_nodes<T>(shape_args, ctx->n_mbf_pad);
  if (jt < 1) return fail(ctx, CFFT_ERR_ARG, "element too large for the integrand tile");
  // MBF spectra on the tensor cores (FP32-mixed rooftop elements), unless disabled
  bool tc_b = false;
  if constexpr (sizeof(T) == 4) {
    if (!(ctx->opt[CFFT_OPT_SPECTRA_SIMT] > 0) && (n_alpha == 128 || n_alpha == 256) && ctx->n_mbf <= 4) {
      bool rooftop = true;
      for (const ShapeClass& c : ctx->shapes) rooftop = rooftop && c.kind == 0;
      if (rooftop && spectra_tc_columns((int)ctx->shapes.size(), ctx->n_mbf) > 0 &&
          ensure_tc_element(ctx) == CFFT_OK) {
        shape_args.tc_bx = ctx->tc_bx.as<float>();
        shape_args.tc_by = ctx->tc_by.as<float>();
        shape_args.tc_bmat = ctx->tc_bmat_mirror.as<float>();
        shape_args.tc_ncol = 2 * spectra_tc_columns((int)ctx->shapes.size(), ctx->n_mbf);
        shape_args.tc_rmax = ctx->tc_rmax;
        tc_b = integrand_tc_applies(shape_args);
        if (tc_b) jt = integrand_tc_nodes(n_alpha);
      }
    }
  }
  // the tensor-core integrand at 256 angles for the items that need them and at 128 for
  // the others (automatic angle count only): one launch per angle count and wave
  std::vector<int> item_na(n_items, n_alpha);
  IntegrandArgs<T> shape128 = shape_args;
  shape128.n_alpha = 128;
  bool split_na = false;
  if constexpr (sizeof(T) == 4)
    split_na = tc_b && n_alpha == 256 && ctx->opt[CFFT_OPT_N_ALPHA] <= 0 && integrand_tc_applies(shape128);
  if (split_na)
    for (int i = 0; i < n_items; ++i) item_na[i] = ip[i].na_need <= 128 ? 128 : 256;
  const int jt128 = split_na ? integrand_tc_nodes(128) : jt;
  CFFT_CUDA(ctx->b_flag.ensure(2 * sizeof(int)), "alloc flag");
  CFFT_CUDA(cudaMemsetAsync(ctx->b_flag.p, 0, 2 * sizeof(int), st), "flag");

  // back-projection chunk shapes depend on rchunk; FFT tasks on the sub-FFT length
  // mode 0: plan + plain launches; 1: plan + capture into a new graph; 2: plan only
  // (the captured graph reads the refreshed plan); 3: plan + launches, time one stage
  auto build_and_run = [&](int L, int rchunk, int mode, int stage_to_time,
                           float* stage_ms) -> cfft_status {
    int log2L = 0;
    while ((1 << log2L) < L) ++log2L;
    const int n_chunks = (n_rho + rchunk - 1) / rchunk;
    std::vector<ContourArgs> hca(n_items);
    std::vector<ContourData> hcd(n_items);
    std::vector<IntegrandArgs<T>> hia(n_items);
    std::vector<FftArgs<T>> hfa(n_items);
    std::vector<BackprojArgs<T>> hba(n_items);
    std::vector<int2> cmap, imap;
    std::vector<int4> ftask, btask;
    std::vector<int> cnodes((size_t)n_items * n_chunks);
    std::vector<int64_t> coff((size_t)n_items * n_chunks);
    struct FftBucket { int log2L; size_t f0, f1; int max_nout; };
    // integrand blocks of a wave: [i0, im) at 128 angles when the counts are split, [im, i1)
    // at n_alpha
    struct WaveRanges { size_t c0, c1, i0, im, i1, f0, f1, b0, b1; std::vector<FftBucket> fb; };
    std::vector<WaveRanges> wr;
    int64_t cos_total = 0;
    int max_nodes = 0, max_seg = 0, max_nout = 0, max_active = 0, max_n_item = 0, zt_arrays = 1;
    for (int i = 0; i < n_items; ++i) {
      max_active = std::max(max_active, ip[i].n_active);
      max_n_item = std::max(max_n_item, ip[i].n);
      if (ip[i].series == 1) zt_arrays = 2;   // the Chebyshev recurrence keeps two terms
    }
    for (int i = 0; i < n_items; ++i) {
      for (int c = 0; c < n_chunks; ++c) {
        int r_top = std::min((c + 1) * rchunk, n_rho) - 1;
        double rho_top = r_top * d_rho;
        int np = alpha_nodes(ip[i].beta_abs, rho_top, q_max, margin, alpha_cbrt_coef(fp64));
        cnodes[(size_t)i * n_chunks + c] = np;
        coff[(size_t)i * n_chunks + c] = cos_total;
        cos_total += np;
        max_nodes = std::max(max_nodes, np);
        int kseg = std::min(ip[i].K, (int)std::ceil(rho_top / ip[i].ds) + bp_taps / 2 + 2);
        max_seg = std::max(max_seg, 2 * kseg + 1);
      }
    }
    // every buffer the per-item arguments point into is sized here, before those
    // pointers are taken (a later reallocation would leave them dangling)
    CFFT_CUDA(ctx->b_cnodes.ensure(cnodes.size() * sizeof(int)), "alloc plan");
    CFFT_CUDA(ctx->b_coff.ensure(coff.size() * sizeof(int64_t)), "alloc plan");
    CFFT_CUDA(ctx->b_cos.ensure(cos_total * sizeof(double)), "alloc plan");
    CFFT_CUDA(ctx->d_tw.ensure((size_t)L * sizeof(cpx<T>)), "alloc twiddles");
    if (pform_b ? (tform_b ? backproject_tc_smem(max_nodes) : backproject_pm_smem(max_nodes)) > 225 * 1024
                : (backproject_w_smem<T>(max_nodes, pairs) > 225 * 1024 || pairs > 64))
      return fail(ctx, CFFT_ERR_ARG, "batch: rho_max too large for the angular node table");
    const int group = std::min(8, pairs);
    double work_bp = 0, work_fft = 0;
    // sub-FFT length of each item: at most L, a divisor of its P, at least 4 residues
    // when the item allows, and a shared-memory footprint that fits
    std::vector<int> li(n_items);
    for (int i = 0; i < n_items; ++i) {
      const BatchItemPlan& p = ip[i];
      int l = 1;
      while ((p.P % (2 * (int64_t)l)) == 0 && 2 * l <= L) l *= 2;
      while (l > 1024 && p.P / l < 4) l /= 2;
      auto smem_of = [&](int ll) {
        int d = (int)(p.P / ll);
        // the transform buffer is padded by one entry in 16 for lengths >= 1024
        return (size_t)(ll >= 1024 ? ll + ll / 16 : ll) * sizeof(cpx<T>) +
               fft_task_extra<T>(0, (2 * p.K + 1) / d + 4, (p.n + 127) / 128);
      };
      while (l > 1024 && smem_of(l) > 220 * 1024) l /= 2;
      if (smem_of(l) > 220 * 1024)
        return fail(ctx, CFFT_ERR_ARG, "batch item too large for a shared-memory transform");
      li[i] = l;
    }
    for (const Wave& w : waves) {
      WaveRanges r{cmap.size(), 0, imap.size(), 0, 0, ftask.size(), 0, btask.size(), 0, {}};
      // the 128-angle items' integrand blocks first
      for (int i = w.i0; i < w.i1; ++i)
        if (item_na[i] != n_alpha)
          for (int j0 = 0; j0 < items[i].n; j0 += jt128) imap.push_back(make_int2(i, j0));
      r.im = imap.size();
      for (int i = w.i0; i < w.i1; ++i)
        if (item_na[i] == n_alpha)
          for (int j0 = 0; j0 < items[i].n; j0 += jt) imap.push_back(make_int2(i, j0));
      int64_t node_off = 0, grid_off = 0;
      for (int i = w.i0; i < w.i1; ++i) {
        const cfft_batch_item& it = items[i];
        const BatchItemPlan& p = ip[i];
        hca[i] = ContourArgs{it.n, it.beta_max, it.beta_p, it.height, p.step, it.eps_r, it.h, it.k0};
        if (bp_es) {
          hca[i].es_width = bp_taps;
          hca[i].ds = p.ds;
        }
        set_extraction(ctx, it.eps_r, &hca[i].extract, &hca[i].eps_eff, &hca[i].deps_eff);
        hcd[i] = ContourData{c_beta + node_off, c_w + node_off, c_bw + node_off, c_bi + node_off,
                             c_bif + node_off, c_gp + node_off, c_gr + node_off,
                             nullptr, nullptr, nullptr, nullptr, bp_es ? c_prec + node_off : nullptr};
        for (int j0 = 0; j0 < it.n; j0 += 256) cmap.push_back(make_int2(i, j0));
        IntegrandArgs<T>& ia = hia[i];
        ia = IntegrandArgs<T>{};
        ia.n = it.n;
        ia.n_alpha = item_na[i];
        ia.q_max = q_max;
        ia.n_cls = 1;
        ia.n_mbf = M;
        ia.n_shape = (int)ctx->shapes.size();
        ia.n_basis = ctx->n_basis;
        ia.shapes = ctx->d_shapes.as<ShapeClass>();
        ia.bx = ctx->d_bx.as<T>();
        ia.by = ctx->d_by.as<T>();
        ia.q = ctx->d_q.as<cpx<T>>();
        ia.beta_c = c_beta + node_off;
        ia.bw = c_bw + node_off;
        ia.green_p = c_gp + node_off;
        ia.green_r = c_gr + node_off;
        ia.y = ctx->b_y.as<cpx<T>>() + (size_t)series * node_off;
        if (tc_b) {
          ia.tc_bx = shape_args.tc_bx;
          ia.tc_by = shape_args.tc_by;
          ia.tc_bmat = shape_args.tc_bmat;
          ia.tc_ncol = shape_args.tc_ncol;
          ia.tc_rmax = shape_args.tc_rmax;
          ia.err = ctx->b_flag.as<int>() + 1;
        }
        const int Li = li[i];
        int log2Li = 0;
        while ((1 << log2Li) < Li) ++log2Li;
        const int D = (int)(p.P / Li);
        FftArgs<T>& fa = hfa[i];
        fa = FftArgs<T>{};
        fa.series = series;
        fa.n = it.n;
        fa.sub_len = Li;
        fa.log2_sub = log2Li;
        fa.n_sub = D;
        fa.fft_len = p.P;
        fa.grid_half = p.K;
        fa.taylor = p.taylor;
        fa.expansion = p.series;
        fa.n_active = p.n_active;
        fa.sigma = sigma;
        fa.ds_height = p.ds * it.height;
        fa.y = ia.y;
        fa.bi_rel = c_bi + node_off;
        fa.bi_rel_f = c_bif + node_off;
        fa.twiddle = ctx->d_tw.as<cpx<T>>();
        if constexpr (sizeof(T) == 4) fa.prec = bp_es ? reinterpret_cast<const cpx<float>*>(c_prec + node_off) : nullptr;
        fa.grid = ctx->b_grid.as<cpx<T>>() + grid_off;
        max_nout = std::max(max_nout, (2 * p.K + 1) / D + 2);
        for (int sr = 0; sr < series; ++sr)
          for (int k2 = 0; k2 < D; ++k2) ftask.push_back(make_int4(i, sr, k2, log2Li));
        work_fft += (double)series * D * (p.taylor + (p.series == 1 ? 2 : 1));
        BackprojArgs<T>& ba = hba[i];
        ba = BackprojArgs<T>{};
        ba.series_per_q = pairs;
        ba.n_harm = nh;
        ba.q_max = q_max;
        ba.n_rho = n_rho;
        ba.grid_half = p.K;
        ba.sigma = sigma;
        ba.taps = bp_taps;
        ba.group = group;
        ba.rchunk = rchunk;
        ba.d_rho = d_rho;
        ba.d_s = p.ds;
        ba.beta_abs_max = p.beta_abs;
        ba.alpha_margin = margin;
        ba.grid = fa.grid;
        ba.table = reinterpret_cast<cpx<T>*>(tables) + (size_t)i * table_elems;
        ba.chunk_nodes = ctx->b_cnodes.as<int>() + (size_t)i * n_chunks;
        ba.chunk_off = ctx->b_coff.as<int64_t>() + (size_t)i * n_chunks;
        ba.cosv = ctx->b_cos.as<double>();
        ba.err = tform_b ? ctx->b_flag.as<int>() + 1 : nullptr;
        ba.kern = bp_es ? 1 : 0;
        for (int c = n_chunks - 1; c >= 0; --c) {  // larger rho (more nodes) first
          int rows = std::min((c + 1) * rchunk, n_rho) - c * rchunk;
          if (pform_b) {
            const int n_sc = (pairs + backproject_pm_series_chunk() - 1) / backproject_pm_series_chunk();
            for (int pq = 0; pq <= q_max; ++pq)
              for (int sc = 0; sc < n_sc; ++sc) btask.push_back(make_int4(i, pq, c, sc));
          } else {
            for (int q = 0; q < nh; ++q) btask.push_back(make_int4(i, q, c, 0));
          }
          work_bp += (double)cnodes[(size_t)i * n_chunks + c] * rows * series;
        }
        node_off += it.n;
        grid_off += (int64_t)series * (2 * p.K + 1);
      }
      r.c1 = cmap.size();
      r.i1 = imap.size();
      r.f1 = ftask.size();
      r.b1 = btask.size();
      // FFT tasks of the wave grouped by sub-FFT length (one persistent launch per length),
      // the larger transforms first inside each group
      std::stable_sort(ftask.begin() + r.f0, ftask.end(),
                       [](const int4& a, const int4& b) { return a.w > b.w; });
      for (size_t t = r.f0; t < r.f1;) {
        size_t u = t;
        int mo = 0;
        while (u < r.f1 && ftask[u].w == ftask[t].w) {
          const int i = ftask[u].x;
          mo = std::max(mo, (2 * ip[i].K + 1) / (int)(ip[i].P / li[i]) + 2);
          ++u;
        }
        r.fb.push_back(FftBucket{ftask[t].w, t, u, mo});
        t = u;
      }
      if (r.fb.size() > 7)  // one completion counter per sub-FFT length, seven per wave
        return fail(ctx, CFFT_ERR_ARG, "batch: more than seven sub-FFT lengths in one wave");
      // within a wave, the costliest back-projection tasks (largest rho) first
      std::stable_sort(btask.begin() + r.b0, btask.end(),
                       [](const int4& a, const int4& b) { return a.z > b.z; });
      wr.push_back(r);
    }
    // upload the plan
    auto up = [&](DevBuf& b, const void* src, size_t bytes) -> cudaError_t {
      cudaError_t e = b.ensure(bytes);
      if (e != cudaSuccess) return e;
      return cudaMemcpy(b.p, src, bytes, cudaMemcpyHostToDevice);
    };
    CFFT_CUDA(up(ctx->b_cargs, hca.data(), hca.size() * sizeof(ContourArgs)), "upload plan");
    CFFT_CUDA(up(ctx->b_cdata, hcd.data(), hcd.size() * sizeof(ContourData)), "upload plan");
    CFFT_CUDA(up(ctx->b_iargs, hia.data(), hia.size() * sizeof(IntegrandArgs<T>)), "upload plan");
    CFFT_CUDA(up(ctx->b_fargs, hfa.data(), hfa.size() * sizeof(FftArgs<T>)), "upload plan");
    CFFT_CUDA(up(ctx->b_bargs, hba.data(), hba.size() * sizeof(BackprojArgs<T>)), "upload plan");
    CFFT_CUDA(up(ctx->b_cmap, cmap.data(), cmap.size() * sizeof(int2)), "upload plan");
    CFFT_CUDA(up(ctx->b_imap, imap.data(), imap.size() * sizeof(int2)), "upload plan");
    CFFT_CUDA(up(ctx->b_ftask, ftask.data(), ftask.size() * sizeof(int4)), "upload plan");
    CFFT_CUDA(up(ctx->b_btask, btask.data(), btask.size() * sizeof(int4)), "upload plan");
    CFFT_CUDA(up(ctx->b_cnodes, cnodes.data(), cnodes.size() * sizeof(int)), "upload plan");
    CFFT_CUDA(up(ctx->b_coff, coff.data(), coff.size() * sizeof(int64_t)), "upload plan");
    CFFT_CUDA(ctx->b_count.ensure(8 * wr.size() * sizeof(int)), "alloc plan");
    ctx->tw_len = -1;  // the single-table cache no longer holds these twiddles
    ctx->b_work_bp = work_bp;
    ctx->b_work_fft = work_fft;
    ctx->b_sub_len = L;
    ctx->b_rchunk = rchunk;
    ctx->b_bp_tc = tform_b ? 1 : 0;
    ctx->b_waves = (int)waves.size();

    // everything a captured graph holds by value: buffer addresses, launch shapes and
    // task ranges.  A replay is valid only while all of them are unchanged; the per-item
    // values (substrate, contour) live in the argument buffers refreshed above.
    std::string shape;
    auto add = [&](long long v) {
      shape += std::to_string(v);
      shape += ',';
    };
    for (long long v : {(long long)L, (long long)rchunk, (long long)tform_b, (long long)tc_b, (long long)jt,
                        (long long)split_na,
                        (long long)n_chunks, (long long)max_nodes, (long long)max_seg, (long long)max_nout,
                        (long long)max_active, (long long)max_n_item, (long long)cos_total,
                        (long long)zt_arrays})
      add(v);
    for (const void* ptr : {ctx->d_tw.p, ctx->b_cnodes.p, ctx->b_coff.p, ctx->b_cos.p, ctx->b_count.p,
                            ctx->b_cargs.p, ctx->b_cdata.p, ctx->b_iargs.p, ctx->b_fargs.p, ctx->b_bargs.p,
                            ctx->b_cmap.p, ctx->b_imap.p, ctx->b_ftask.p, ctx->b_btask.p, ctx->b_flag.p,
                            ctx->b_y.p, ctx->b_grid.p, ctx->b_contour.p, ctx->d_bx.p, ctx->d_by.p, ctx->d_q.p,
                            ctx->d_shapes.p, ctx->tc_bx.p, ctx->tc_by.p, ctx->tc_bmat_mirror.p})
      add((long long)(uintptr_t)ptr);
    for (const WaveRanges& r : wr) {
      for (size_t v : {r.c0, r.c1, r.i0, r.i1, r.f0, r.f1, r.b0, r.b1}) add((long long)v);
      for (const FftBucket& fb : r.fb) {
        add(fb.log2L);
        add((long long)fb.f0);
        add((long long)fb.f1);
        add(fb.max_nout);
      }
    }
    if (mode == 2 && shape != ctx->bshape) mode = 1;  // the plan moved: capture again

    // the launch sequence (stream-ordered on the batch stream)
    int launches = 0;
    // stage events: inside a capture they become event-record nodes of the graph
    auto rec = [&](cudaEvent_t ev) {
      if (mode == 1) cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
      else cudaEventRecord(ev, st);
    };
    auto issue = [&]() -> cudaError_t {
      launch_twiddle<T>(ctx->d_tw.as<cpx<T>>(), L, st);
      ++launches;
      cudaError_t e = launch_chunk_cosines(ctx->b_cnodes.as<int>(), ctx->b_coff.as<int64_t>(),
                                           n_items * n_chunks, max_nodes, ctx->b_cos.as<double>(), st);
      if (e != cudaSuccess) return e;
      ++launches;
      e = cudaMemsetAsync(ctx->b_count.p, 0, 8 * wr.size() * sizeof(int), st);
      if (e != cudaSuccess) return e;
      const size_t n_waves = mode == 3 ? 1 : wr.size();  // tuning times the first wave only
      for (size_t w = 0; w < n_waves; ++w) {
        const WaveRanges& r = wr[w];
        int* counters = ctx->b_count.as<int>() + 8 * w;  // [0]: back-projection, [1..]: FFT buckets
        if (w == 0) rec(ctx->bev[0]);
        launch_contour_batch(ctx->b_cargs.as<ContourArgs>(), ctx->b_cdata.as<ContourData>(),
                             ctx->b_cmap.as<int2>() + r.c0, (int)(r.c1 - r.c0), st);
        ++launches;
        if constexpr (sizeof(T) == 4) {
          if (tc_b) {
            e = cudaSuccess;
            if (r.im > r.i0) {
              e = launch_integrand_tc_batch(shape128, ctx->b_iargs.as<IntegrandArgs<float>>(),
                                            ctx->b_imap.as<int2>() + r.i0, (int)(r.im - r.i0), st);
              ++launches;
            }
            if (e == cudaSuccess && r.i1 > r.im)
              e = launch_integrand_tc_batch(shape_args, ctx->b_iargs.as<IntegrandArgs<float>>(),
                                            ctx->b_imap.as<int2>() + r.im, (int)(r.i1 - r.im), st);
            else if (e == cudaSuccess)
              --launches;   // no block at n_alpha in this wave
          } else
            e = launch_integrand_batch<T>(shape_args, ctx->b_iargs.as<IntegrandArgs<T>>(),
                                          ctx->b_imap.as<int2>() + r.i0, (int)(r.i1 - r.i0), jt,
                                          ctx->n_mbf_pad, st);
        } else {
          e = launch_integrand_batch<T>(shape_args, ctx->b_iargs.as<IntegrandArgs<T>>(),
                                        ctx->b_imap.as<int2>() + r.i0, (int)(r.i1 - r.i0), jt,
                                        ctx->n_mbf_pad, st);
        }
        if (e != cudaSuccess) return e;
        ++launches;
        if (w == 0) rec(ctx->bev[1]);
        for (size_t bkt = 0; bkt < r.fb.size() && bkt < 7; ++bkt) {
          const FftBucket& fb = r.fb[bkt];
          e = launch_fft_batch<T>(ctx->b_fargs.as<FftArgs<T>>(), ctx->b_ftask.as<int4>() + fb.f0,
                                  (int)(fb.f1 - fb.f0), counters + 1 + bkt, fb.log2L, fb.max_nout,
                                  max_active, (max_n_item + 127) / 128, zt_arrays, ctx->sm_count, st);
          if (e != cudaSuccess) return e;
          ++launches;
        }
        if (w == 0) rec(ctx->bev[2]);
        if constexpr (sizeof(T) == 4) {
          if (tform_b)
            e = launch_backproject_tc_batch(ctx->b_bargs.as<BackprojArgs<float>>(),
                                            ctx->b_btask.as<int4>() + r.b0, (int)(r.b1 - r.b0), counters,
                                            bp_taps, bp_kern, max_nodes, ctx->sm_count, st);
          else if (pform_b)
            e = launch_backproject_pm_batch(ctx->b_bargs.as<BackprojArgs<float>>(),
                                            ctx->b_btask.as<int4>() + r.b0, (int)(r.b1 - r.b0), counters,
                                            bp_taps, bp_kern, max_nodes, ctx->sm_count, st);
          else
            e = launch_backproject_w_batch<T>(ctx->b_bargs.as<BackprojArgs<T>>(),
                                              ctx->b_btask.as<int4>() + r.b0, (int)(r.b1 - r.b0),
                                              counters, bp_taps, max_nodes, pairs, ctx->sm_count, st);
        } else {
          e = launch_backproject_w_batch<T>(ctx->b_bargs.as<BackprojArgs<T>>(),
                                            ctx->b_btask.as<int4>() + r.b0, (int)(r.b1 - r.b0),
                                            counters, bp_taps, max_nodes, pairs, ctx->sm_count, st);
        }
        if (e != cudaSuccess) return e;
        ++launches;
        if (w == 0) rec(ctx->bev[3]);
      }
      return cudaGetLastError();
    };
    if (mode == 2) return CFFT_OK;
    if (mode == 3) {
      // tuning run: plain launches, time the requested stage of the first wave
      CFFT_CUDA(issue(), "batch launch");
      CFFT_CUDA(cudaStreamSynchronize(st), "batch tuning");
      float ms = 0;
      cudaEventElapsedTime(&ms, ctx->bev[stage_to_time], ctx->bev[stage_to_time + 1]);
      *stage_ms = ms;
      return CFFT_OK;
    }
    if (mode == 1) {
      if (ctx->bgraph) {
        cudaGraphExecDestroy(ctx->bgraph);
        ctx->bgraph = nullptr;
      }
      cudaGraph_t graph = nullptr;
      CFFT_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed), "graph capture");
      cudaError_t e = issue();
      cudaError_t e2 = cudaStreamEndCapture(st, &graph);
      if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(ctx, e, "batch capture");
      }
      CFFT_CUDA(e2, "graph capture");
      e = cudaGraphInstantiate(&ctx->bgraph, graph, 0);
      cudaGraphDestroy(graph);
      CFFT_CUDA(e, "graph instantiate");
      ctx->bsig = sig;
      ctx->bshape = shape;
      ++ctx->b_captures;
    } else {
      CFFT_CUDA(issue(), "batch launch");
    }
    ctx->b_launches = launches;
    return CFFT_OK;
  };

  for (auto& e : ctx->bev)
    if (!e) CFFT_CUDA(cudaEventCreate(&e), "event");

  // ---- autotune the sub-FFT length and the back-projection row chunk (cached per signature)
  int L = std::min(l_common, fp64 ? 8192 : 16384);
  // row tile of the matrix-form back-projection (paired-harmonic form in FP32-mixed)
  int rchunk = pform_b ? backproject_pm_rows() : backproject_w_rows();
  auto tc = ctx->tuned.find(sig);
  if (tc != ctx->tuned.end()) {
    L = tc->second.sub_len;
    rchunk = tc->second.rchunk;
    tform_b = tform_b && tc->second.bp_tc != 0;
  } else if (flags & 2) {
    float best = 1e30f;
    for (int cand = 2048; cand <= l_common; cand *= 2) {
      float ms = 0;
      cfft_status s = build_and_run(cand, rchunk, 3, 1, &ms);
      if (s != CFFT_OK) return s;
      if (ms < best) {
        best = ms;
        L = cand;
      }
    }
    if (tform_b) {
      // back-projection products: tensor cores or the FP32 pipe, whichever is faster here
      float ms_tc = 0, ms_simt = 0;
      cfft_status s = build_and_run(L, rchunk, 3, 2, &ms_tc);
      if (s != CFFT_OK) return s;
      tform_b = false;
      s = build_and_run(L, rchunk, 3, 2, &ms_simt);
      if (s != CFFT_OK) return s;
      tform_b = ms_tc <= ms_simt;
    }
    ctx->tuned[sig] = {L, rchunk, tform_b ? 1 : 0};
  }

  const bool use_graph = (flags & 1) != 0;
  const bool reuse = use_graph && ctx->bgraph && ctx->bsig == sig && ctx->b_sub_len == L &&
                     ctx->b_rchunk == rchunk && ctx->b_bp_tc == (tform_b ? 1 : 0);
  {
    // same structure: refresh the per-item parameters (substrate, contour) that the
    // captured graph reads; otherwise plan again and launch or capture
    cfft_status s = build_and_run(L, rchunk, reuse ? 2 : (use_graph ? 1 : 0), -1, nullptr);
    if (s != CFFT_OK) return s;
  }
  if (use_graph) {
    CFFT_CUDA(cudaEventRecord(ctx->bev[4], st), "event");
    CFFT_CUDA(cudaGraphLaunch(ctx->bgraph, st), "graph launch");
    CFFT_CUDA(cudaEventRecord(ctx->bev[5], st), "event");
  }
  // NaN / Inf scan of all tables
  CFFT_CUDA(ctx->b_flag.ensure(sizeof(int)), "alloc flag");
  CFFT_CUDA(cudaMemsetAsync(ctx->b_flag.p, 0, sizeof(int), st), "flag");
  launch_nonfinite<T>(reinterpret_cast<const cpx<T>*>(tables), (int64_t)(n_items * table_elems),
                      ctx->b_flag.as<int>(), st);
  int flag = 0, tc_flag = 0;
  CFFT_CUDA(cudaMemcpyAsync(&flag, ctx->b_flag.p, sizeof(int), cudaMemcpyDeviceToHost, st), "flag");
  CFFT_CUDA(cudaMemcpyAsync(&tc_flag, ctx->b_flag.as<int>() + 1, sizeof(int), cudaMemcpyDeviceToHost, st), "flag");
  CFFT_CUDA(cudaStreamSynchronize(st), "batch");
  if (tc_flag & 16) return fail(ctx, CFFT_ERR_TIMEOUT, "batch integrand: a tensor-core wait ran past its bound");
  if (tc_flag & 32)
    return fail(ctx, CFFT_ERR_TIMEOUT, "batch back-projection: a tensor-core wait ran past its bound");
  float ms = 0;
  if (cudaEventElapsedTime(&ms, ctx->bev[0], ctx->bev[1]) == cudaSuccess) ctx->b_ms[0] = ms;
  if (cudaEventElapsedTime(&ms, ctx->bev[1], ctx->bev[2]) == cudaSuccess) ctx->b_ms[1] = ms;
  if (cudaEventElapsedTime(&ms, ctx->bev[2], ctx->bev[3]) == cudaSuccess) ctx->b_ms[2] = ms;
  if (use_graph && cudaEventElapsedTime(&ms, ctx->bev[4], ctx->bev[5]) == cudaSuccess) ctx->b_ms[3] = ms;
  cudaGetLastError();  // an unrecorded timing event is not an error of the batch
  if (flag) return fail(ctx, CFFT_ERR_NUMERIC, "non-finite value in a batch table");
  return CFFT_OK;
}

}  // namespace

extern "C" {

cfft_status cfft_create(cfft_ctx** out, int device, void* cuda_stream) {
  if (!out) return CFFT_ERR_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return CFFT_ERR_CUDA;
  }
  cfft_ctx* c = new (std::nothrow) cfft_ctx();
  if (!c) return CFFT_ERR_OOM;
  c->device = device;
  c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      c->sm_count < 1) {
    cudaGetLastError();
    delete c;
    return CFFT_ERR_CUDA;
  }
  *out = c;
  return CFFT_OK;
}

void cfft_destroy(cfft_ctx* ctx) {
  if (!ctx) return;
  {
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    DevBuf* bufs[] = {&ctx->beta_c, &ctx->weight, &ctx->bw, &ctx->bi_rel, &ctx->green_p,
                      &ctx->green_r, &ctx->dp_eps, &ctx->dr_eps, &ctx->dp_h, &ctx->dr_h, &ctx->d_shapes, &ctx->d_bx, &ctx->d_by, &ctx->d_q,
                      &ctx->d_y, &ctx->d_grid, &ctx->d_table, &ctx->d_tw, &ctx->d_cnodes,
                      &ctx->d_coff, &ctx->d_cos, &ctx->d_lag, &ctx->d_flag, &ctx->d_pos,
                      &ctx->d_rot, &ctx->d_zbuf, &ctx->d_fill, &ctx->d_gres, &ctx->d_ftable, &ctx->d_fest, &ctx->d_quser, &ctx->lu_a, &ctx->lu_moves,
                      &ctx->lu_nmoves, &ctx->lu_cand_v, &ctx->lu_cand_r, &ctx->lu_cand_d, &ctx->lu_bar, &ctx->lu_err, &ctx->lu_x,
                      &ctx->lu_y, &ctx->lu_x64, &ctx->lu_r, &ctx->lu_sums, &ctx->c_tab, &ctx->c_work,
                      &ctx->c_work2, &ctx->c_im, &ctx->c_gx, &ctx->c_gy, &ctx->c_flag, &ctx->tc_bx, &ctx->tc_by, &ctx->tc_bmat,
                      &ctx->tc_bmat_mirror, &ctx->tc_shapes};
    for (DevBuf* b : bufs) b->release();
    for (auto& e : ctx->ev)
      if (e) cudaEventDestroy(e);
    for (auto& e : ctx->lu_ev)
      if (e) cudaEventDestroy(e);
    DevBuf* bb[] = {&ctx->b_cargs, &ctx->b_cdata, &ctx->b_iargs, &ctx->b_fargs, &ctx->b_bargs,
                    &ctx->b_cmap, &ctx->b_imap, &ctx->b_ftask, &ctx->b_btask, &ctx->b_count,
                    &ctx->b_cnodes, &ctx->b_coff, &ctx->b_cos, &ctx->b_contour, &ctx->b_y,
                    &ctx->b_grid, &ctx->b_flag};
    for (DevBuf* b : bb) b->release();
    for (auto& e : ctx->bev)
      if (e) cudaEventDestroy(e);
    if (ctx->bgraph) cudaGraphExecDestroy(ctx->bgraph);
    if (ctx->bstream) cudaStreamDestroy(ctx->bstream);
  }
  delete ctx;
}

const char* cfft_last_error(const cfft_ctx* ctx) {
  return ctx ? ctx->err.c_str() : "null context";
}

cfft_status cfft_set_substrate(cfft_ctx* ctx, double eps_r, double h, double k0) {
  if (!ctx) return CFFT_ERR_ARG;
  if (!(eps_r > 0) || !(h >= 0) || !(k0 > 0) || !std::isfinite(eps_r) || !std::isfinite(h) ||
      !std::isfinite(k0))
    return fail(ctx, CFFT_ERR_ARG, "substrate: need eps_r > 0, h >= 0, k0 > 0");
  ctx->eps_r = eps_r;
  ctx->hs = h;
  ctx->k0 = k0;
  ctx->has_sub = true;
  ctx->has_contour = false;
  ctx->has_table = false;
  return CFFT_OK;
}

cfft_status cfft_set_green_extraction(cfft_ctx* ctx, int extract, double eps_eff) {
  if (!ctx) return CFFT_ERR_ARG;
  if (extract != 0 && extract != 1) return fail(ctx, CFFT_ERR_ARG, "extract must be 0 or 1");
  if (!std::isfinite(eps_eff)) return fail(ctx, CFFT_ERR_ARG, "eps_eff must be finite");
  ctx->extract = extract;
  ctx->eps_eff_set = eps_eff;
  ctx->has_table = false;
  return CFFT_OK;
}

cfft_status cfft_set_mbf_spectra_strip(cfft_ctx* ctx, double length, double width) {
  if (!ctx) return CFFT_ERR_ARG;
  if (!(length > 0) || !(width > 0)) return fail(ctx, CFFT_ERR_ARG, "strip: need length, width > 0");
  ctx->shapes.assign(1, ShapeClass{1, 0, 0, 1, length, width});
  ctx->bx.assign(1, 0.0);
  ctx->by.assign(1, 0.0);
  ctx->n_basis = 1;
  ctx->n_mbf = 1;
  ctx->n_mbf_pad = 1;
  ctx->q.assign(1, {1.0, 0.0});
  ctx->q_user.assign(1, {1.0, 0.0});
  ctx->elem_radius = 0.5 * std::hypot(length, width);
  ctx->has_el = true;
  ctx->has_table = false;
  ctx->tc_ready = false;
  return CFFT_OK;
}

cfft_status cfft_set_mbf_spectra(cfft_ctx* ctx, int n_basis, const double* centers,
                                 const int* dir, const double* half_len, const double* width,
                                 int n_mbf, const double* q) {
  if (!ctx) return CFFT_ERR_ARG;
  if (n_basis < 1 || n_basis > kMaxBasis) return fail(ctx, CFFT_ERR_ARG, "n_basis must be in 1..4096");
  if (n_mbf < 1 || n_mbf > 8) return fail(ctx, CFFT_ERR_ARG, "n_mbf must be in 1..8");
  if (!centers || !dir || !half_len || !width || !q) return fail(ctx, CFFT_ERR_ARG, "null pointer");
  // group bases by shape class (direction, half-length, width)
  std::map<std::tuple<int, double, double>, std::vector<int>> groups;
  double radius = 0;
  for (int i = 0; i < n_basis; ++i) {
    if (dir[i] != 0 && dir[i] != 1) return fail(ctx, CFFT_ERR_ARG, "dir must be 0 or 1");
    if (!(half_len[i] > 0) || !(width[i] > 0)) return fail(ctx, CFFT_ERR_ARG, "rooftop sizes must be > 0");
    groups[std::make_tuple(dir[i], half_len[i], width[i])].push_back(i);
    double ext = std::max(half_len[i], 0.5 * width[i]);
    radius = std::max(radius, std::hypot(centers[2 * i], centers[2 * i + 1]) + ext);
  }
  if ((int)groups.size() > kMaxShapeClasses) return fail(ctx, CFFT_ERR_ARG, "too many distinct rooftop shapes (max 32)");
  int pad = n_mbf <= 1 ? 1 : n_mbf <= 2 ? 2 : n_mbf <= 4 ? 4 : 8;
  ctx->shapes.clear();
  ctx->bx.clear();
  ctx->by.clear();
  ctx->q.assign((size_t)n_basis * pad, {0.0, 0.0});
  int pos = 0;
  for (auto& kv : groups) {
    ShapeClass sc{0, std::get<0>(kv.first), pos, pos + (int)kv.second.size(), std::get<1>(kv.first),
                  std::get<2>(kv.first)};
    for (int i : kv.second) {
      ctx->bx.push_back(centers[2 * i]);
      ctx->by.push_back(centers[2 * i + 1]);
      for (int a = 0; a < n_mbf; ++a)
        ctx->q[(size_t)pos * pad + a] = {q[2 * ((size_t)i * n_mbf + a)], q[2 * ((size_t)i * n_mbf + a) + 1]};
      ++pos;
    }
    ctx->shapes.push_back(sc);
  }
  ctx->q_user.resize((size_t)n_basis * n_mbf);
  for (size_t e = 0; e < ctx->q_user.size(); ++e) ctx->q_user[e] = {q[2 * e], q[2 * e + 1]};
  ctx->n_basis = n_basis;
  ctx->n_mbf = n_mbf;
  ctx->n_mbf_pad = pad;
  ctx->elem_radius = radius;
  ctx->has_el = true;
  ctx->has_table = false;
  ctx->tc_ready = false;
  return CFFT_OK;
}

cfft_status cfft_build_contour(cfft_ctx* ctx, int n, double beta_max, double beta_p,
                               double height, int taylor_order) {
  if (!ctx) return CFFT_ERR_ARG;
  if (!ctx->has_sub) return fail(ctx, CFFT_ERR_STATE, "build_contour before set_substrate");
  if (n < 16 || n > (1 << 20)) return fail(ctx, CFFT_ERR_ARG, "n must be in 16..1048576");
  if (!(beta_max > 0) || !(beta_p > 0) || !(beta_p < beta_max) || !(height >= 0))
    return fail(ctx, CFFT_ERR_ARG, "contour: need 0 < beta_p < beta_max, height >= 0");
  if (taylor_order < -1 || taylor_order > 64) return fail(ctx, CFFT_ERR_ARG, "taylor_order must be in -1..64");
  if (height > 0 && !(beta_p > ctx->k0 * std::sqrt(ctx->eps_r)))
    return fail(ctx, CFFT_ERR_ARG, "beta_p must exceed k0 sqrt(eps_r) (all surface-wave poles)");
  ctx->n = n;
  ctx->beta_max = beta_max;
  ctx->beta_p = beta_p;
  ctx->height = height;
  ctx->taylor_req = taylor_order;
  ctx->has_contour = true;
  ctx->has_table = false;
  return CFFT_OK;
}

cfft_status cfft_contour_series_order(double x, cfft_precision precision, int series_opt, int* series,
                                      int* order, int* n_ffts) {
  if (!series || !order || !n_ffts || !std::isfinite(x) || !(x >= 0.0)) return CFFT_ERR_ARG;
  if (precision != CFFT_FP64 && precision != CFFT_FP32_MIXED) return CFFT_ERR_ARG;
  const SeriesChoice sc = choose_series(x, precision == CFFT_FP64, -1, (double)series_opt);
  if (sc.order < 0) return CFFT_ERR_ARG;
  *series = sc.series;
  *order = sc.order;
  *n_ffts = sc.order + (sc.series == 1 ? 2 : 1);
  return CFFT_OK;
}

cfft_status cfft_set_option(cfft_ctx* ctx, cfft_option key, double value) {
  if (!ctx) return CFFT_ERR_ARG;
  if ((int)key < 0 || (int)key >= kNumOptions) return fail(ctx, CFFT_ERR_ARG, "unknown option");
  ctx->opt[(int)key] = value;
  if (key == CFFT_OPT_FILL_REFINE) ctx->fill_r = 0;   // decided again at the next fill
  return CFFT_OK;
}

cfft_status cfft_tabulate_reactions(cfft_ctx* ctx, int q_max, double rho_max, int n_rho,
                                    cfft_precision precision, int rotation_classes) {
  if (!ctx) return CFFT_ERR_ARG;
  if (!ctx->has_sub || !ctx->has_el || !ctx->has_contour)
    return fail(ctx, CFFT_ERR_STATE, "tabulate needs substrate, element and contour");
  if (q_max < 0 || q_max > 64) return fail(ctx, CFFT_ERR_ARG, "q_max must be in 0..64");
  if (n_rho < 2 || n_rho > (1 << 20)) return fail(ctx, CFFT_ERR_ARG, "n_rho must be in 2..1048576");
  if (!(rho_max > 0) || !std::isfinite(rho_max)) return fail(ctx, CFFT_ERR_ARG, "rho_max must be > 0");
  if (precision != CFFT_FP64 && precision != CFFT_FP32_MIXED) return fail(ctx, CFFT_ERR_ARG, "bad precision");
  if (rotation_classes != 1 && rotation_classes != 4) return fail(ctx, CFFT_ERR_ARG, "rotation_classes must be 1 or 4");
  if (ctx->n % 32 != 0) return fail(ctx, CFFT_ERR_ARG, "contour n must be a multiple of 32");
  DeviceGuard g(ctx->device);
  ctx->has_table = false;
  ctx->q_max = q_max;
  ctx->rho_max = rho_max;
  ctx->n_rho = n_rho;
  ctx->prec = precision;
  ctx->cls_stored = rotation_classes;
  ctx->cls_computed = rotation_classes == 4 ? 3 : 1;
  ctx->fill_r = 0;
  ctx->table_loaded = false;
  std::memcpy(ctx->tab_opt, ctx->opt, sizeof(ctx->tab_opt));
  if (precision == CFFT_FP64) return tabulate_impl<double>(ctx, n_rho, rho_max, ctx->d_table, true);
  return tabulate_impl<float>(ctx, n_rho, rho_max, ctx->d_table, true);
}

cfft_status cfft_get_table(const cfft_ctx* ctx, const void** dev_ptr, int64_t shape[4],
                           int* is_complex128) {
  if (!ctx || !dev_ptr || !shape) return CFFT_ERR_ARG;
  if (!ctx->has_table) return CFFT_ERR_STATE;
  *dev_ptr = ctx->d_table.p;
  shape[0] = ctx->cls_stored;
  shape[1] = (int64_t)ctx->n_mbf * ctx->n_mbf;
  shape[2] = 2 * ctx->q_max + 1;
  shape[3] = ctx->n_rho;
  if (is_complex128) *is_complex128 = ctx->prec == CFFT_FP64;
  return CFFT_OK;
}

cfft_status cfft_copy_table(const cfft_ctx* cctx, void* dst, int64_t bytes, int dst_is_host) {
  cfft_ctx* ctx = const_cast<cfft_ctx*>(cctx);
  if (!ctx || !dst) return CFFT_ERR_ARG;
  if (!ctx->has_table) return fail(ctx, CFFT_ERR_STATE, "no table");
  size_t es = ctx->prec == CFFT_FP64 ? 16 : 8;
  size_t need = (size_t)ctx->cls_stored * ctx->n_mbf * ctx->n_mbf * (2 * ctx->q_max + 1) * ctx->n_rho * es;
  if ((size_t)bytes != need) return fail(ctx, CFFT_ERR_ARG, "bytes must equal the table size");
  DeviceGuard g(ctx->device);
  CFFT_CUDA(cudaMemcpyAsync(dst, ctx->d_table.p, need,
                            dst_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                            ctx->stream), "copy table");
  if (dst_is_host) CFFT_CUDA(cudaStreamSynchronize(ctx->stream), "copy table");
  return CFFT_OK;
}

cfft_status cfft_load_table(cfft_ctx* ctx, int n_mbf, int q_max, double rho_max, int n_rho,
                            cfft_precision precision, int rotation_classes, int fill_taps, const void* table,
                            int src_is_host) {
  if (!ctx) return CFFT_ERR_ARG;
  if (!table) return fail(ctx, CFFT_ERR_ARG, "null table");
  if (n_mbf < 1 || n_mbf > 8 || q_max < 0 || q_max > 64 || !(rho_max > 0.0) || !std::isfinite(rho_max) ||
      (precision != CFFT_FP64 && precision != CFFT_FP32_MIXED) ||
      (rotation_classes != 1 && rotation_classes != 4) || fill_taps < 2 || fill_taps > 16 || (fill_taps & 1) ||
      n_rho < 2 * fill_taps || n_rho > (1 << 20))
    return fail(ctx, CFFT_ERR_ARG, "bad table description");
  if (ctx->has_el && ctx->n_mbf != n_mbf)
    return fail(ctx, CFFT_ERR_ARG, "the table's MBF count differs from the context's element");
  DeviceGuard g(ctx->device);
  const size_t es = precision == CFFT_FP64 ? 16 : 8;
  const size_t need = (size_t)rotation_classes * n_mbf * n_mbf * (2 * q_max + 1) * n_rho * es;
  ctx->has_table = false;
  CFFT_CUDA(ctx->d_flag.ensure(sizeof(int) * 4), "alloc flag");
  CFFT_CUDA(ctx->d_table.ensure(need), "alloc table");
  CFFT_CUDA(cudaMemcpyAsync(ctx->d_table.p, table, need, src_is_host ? cudaMemcpyHostToDevice
                                                                      : cudaMemcpyDeviceToDevice,
                            ctx->stream), "load table");
  if (src_is_host) CFFT_CUDA(cudaStreamSynchronize(ctx->stream), "load table");
  if (!ctx->has_el) {
    ctx->n_mbf = n_mbf;
    ctx->n_mbf_pad = n_mbf <= 1 ? 1 : n_mbf <= 2 ? 2 : n_mbf <= 4 ? 4 : 8;
  }
  ctx->q_max = q_max;
  ctx->rho_max = rho_max;
  ctx->n_rho = n_rho;
  ctx->prec = precision;
  ctx->cls_stored = rotation_classes;
  ctx->cls_computed = rotation_classes == 4 ? 3 : 1;
  ctx->fill_taps = fill_taps;
  ctx->channels = 1;
  ctx->fill_r = 0;
  ctx->table_loaded = true;
  ctx->info.fill_err_est = -1.0;
  ctx->info.fill_refine = 0;
  ctx->info.fill_n_rho = 0;
  ctx->has_table = true;
  return CFFT_OK;
}

cfft_status cfft_fill_reduced_matrix(cfft_ctx* ctx, int n_elements, const double* pos_xy,
                                     const int* rot, void* z_out, int64_t ld,
                                     int out_complex128) {
  cfft_status s = check_fill_args(ctx, n_elements, pos_xy, rot, z_out, ld);
  if (s != CFFT_OK) return s;
  DeviceGuard g(ctx->device);
  return fill_dispatch(ctx, n_elements, pos_xy, ctx->cls_stored == 4 ? rot : nullptr, z_out, ld,
                       out_complex128);
}

cfft_status cfft_fill_reduced_matrix_host(cfft_ctx* ctx, int n_elements, const double* pos_xy,
                                          const int* rot, void* z_out, int64_t ld,
                                          int out_complex128) {
  cfft_status s = check_fill_args(ctx, n_elements, pos_xy, rot, z_out, ld);
  if (s != CFFT_OK) return s;
  DeviceGuard g(ctx->device);
  const size_t rows = (size_t)n_elements * ctx->n_mbf;
  const size_t zbytes = rows * (size_t)ld * (out_complex128 ? 16 : 8);
  CFFT_CUDA(ctx->d_pos.ensure((size_t)2 * n_elements * sizeof(double)), "alloc fill");
  CFFT_CUDA(ctx->d_zbuf.ensure(zbytes), "alloc fill");
  CFFT_CUDA(cudaMemcpyAsync(ctx->d_pos.p, pos_xy, (size_t)2 * n_elements * sizeof(double),
                            cudaMemcpyHostToDevice, ctx->stream), "upload");
  const int* drot = nullptr;
  if (ctx->cls_stored == 4) {
    CFFT_CUDA(ctx->d_rot.ensure((size_t)n_elements * sizeof(int)), "alloc fill");
    CFFT_CUDA(cudaMemcpyAsync(ctx->d_rot.p, rot, (size_t)n_elements * sizeof(int),
                              cudaMemcpyHostToDevice, ctx->stream), "upload");
    drot = ctx->d_rot.as<int>();
  }
  s = fill_dispatch(ctx, n_elements, ctx->d_pos.as<double>(), drot, ctx->d_zbuf.p, ld, out_complex128);
  if (s != CFFT_OK) return s;
  CFFT_CUDA(cudaMemcpyAsync(z_out, ctx->d_zbuf.p, zbytes, cudaMemcpyDeviceToHost, ctx->stream), "download");
  CFFT_CUDA(cudaStreamSynchronize(ctx->stream), "download");
  return CFFT_OK;
}

cfft_status cfft_tabulate_batch(cfft_ctx* ctx, int n_items, const cfft_batch_item* items,
                                int q_max, double rho_max, int n_rho, cfft_precision precision,
                                void* tables, int flags) {
  if (!ctx) return CFFT_ERR_ARG;
  if (!ctx->has_el) return fail(ctx, CFFT_ERR_STATE, "batch needs the element (set_mbf_spectra)");
  if (n_items < 1 || n_items > (1 << 19) || !items || !tables)
    return fail(ctx, CFFT_ERR_ARG, "batch: need 1..524288 items and a table buffer");
  if (q_max < 0 || q_max > 64 || n_rho < 16 || n_rho > (1 << 20) || !(rho_max > 0))
    return fail(ctx, CFFT_ERR_ARG, "batch: bad q_max, n_rho or rho_max");
  if (precision != CFFT_FP64 && precision != CFFT_FP32_MIXED) return fail(ctx, CFFT_ERR_ARG, "bad precision");
  for (int i = 0; i < n_items; ++i) {
    const cfft_batch_item& it = items[i];
    if (!(it.eps_r > 0) || !(it.h >= 0) || !(it.k0 > 0) || it.n < 256 || it.n > (1 << 20) ||
        it.n % 256 != 0 || !(it.beta_p > 0) || !(it.beta_p < it.beta_max) || !(it.height >= 0) ||
        it.taylor_order < -1 || it.taylor_order > 64 ||
        (it.height > 0 && !(it.beta_p > it.k0 * std::sqrt(it.eps_r))))
      return fail(ctx, CFFT_ERR_ARG, "batch item " + std::to_string(i) + " is invalid");
  }
  DeviceGuard g(ctx->device);
  if (!ctx->bstream) CFFT_CUDA(cudaStreamCreateWithFlags(&ctx->bstream, cudaStreamNonBlocking), "stream");
  // order the batch after the work already issued on the context stream
  if (!ctx->ev[0]) CFFT_CUDA(cudaEventCreate(&ctx->ev[0]), "event");
  CFFT_CUDA(cudaEventRecord(ctx->ev[0], ctx->stream), "event");
  CFFT_CUDA(cudaStreamWaitEvent(ctx->bstream, ctx->ev[0], 0), "event");
  cfft_status s = precision == CFFT_FP64
                      ? batch_impl<double>(ctx, n_items, items, q_max, rho_max, n_rho, tables, flags)
                      : batch_impl<float>(ctx, n_items, items, q_max, rho_max, n_rho, tables, flags);
  return s;
}

cfft_status cfft_get_batch_info(const cfft_ctx* ctx, cfft_batch_info* info) {
  if (!ctx || !info) return CFFT_ERR_ARG;
  info->ms_integrand = ctx->b_ms[0];
  info->ms_fft = ctx->b_ms[1];
  info->ms_backproject = ctx->b_ms[2];
  info->ms_graph = ctx->b_ms[3];
  info->work_subffts = ctx->b_work_fft;
  info->work_bp_nodes = ctx->b_work_bp;
  info->sub_len = ctx->b_sub_len;
  info->rchunk = ctx->b_rchunk;
  info->waves = ctx->b_waves;
  info->launches = ctx->b_launches;
  info->bp_tc = ctx->b_bp_tc;
  info->captures = ctx->b_captures;
  return CFFT_OK;
}

cfft_status cfft_get_derivative_table(const cfft_ctx* ctx, int which, const void** dev_ptr,
                                      int64_t shape[4]) {
  if (!ctx || !dev_ptr || !shape || which < 0 || which > 2) return CFFT_ERR_ARG;
  if (!ctx->has_table || (which > 0 && ctx->channels != 3)) return CFFT_ERR_STATE;
  const size_t es = ctx->prec == CFFT_FP64 ? 16 : 8;
  const size_t elems = (size_t)ctx->cls_stored * ctx->n_mbf * ctx->n_mbf * (2 * ctx->q_max + 1) * ctx->n_rho;
  *dev_ptr = reinterpret_cast<const unsigned char*>(ctx->d_table.p) + which * elems * es;
  shape[0] = ctx->cls_stored;
  shape[1] = (int64_t)ctx->n_mbf * ctx->n_mbf;
  shape[2] = 2 * ctx->q_max + 1;
  shape[3] = ctx->n_rho;
  return CFFT_OK;
}

cfft_status cfft_fill_backward(cfft_ctx* ctx, int n_elements, const double* pos_xy, const int* rot,
                               const void* grad_z, int64_t ld, int grad_complex128,
                               double* grad_pos, double* grad_eps_h) {
  cfft_status s = check_fill_args(ctx, n_elements, pos_xy, rot, const_cast<void*>(grad_z), ld);
  if (s != CFFT_OK) return s;
  if (!grad_pos && !grad_eps_h) return fail(ctx, CFFT_ERR_ARG, "nothing to compute");
  if (grad_eps_h && ctx->channels != 3)
    return fail(ctx, CFFT_ERR_STATE, "substrate gradient needs a tabulation with CFFT_OPT_DERIVATIVES");
  DeviceGuard g(ctx->device);
  const int* r = ctx->cls_stored == 4 ? rot : nullptr;
  const bool t64 = ctx->prec == CFFT_FP64;
  if (t64 && grad_complex128)
    return fill_backward_impl<double, double>(ctx, n_elements, pos_xy, r, grad_z, ld, grad_pos, grad_eps_h);
  if (t64) return fill_backward_impl<double, float>(ctx, n_elements, pos_xy, r, grad_z, ld, grad_pos, grad_eps_h);
  if (grad_complex128)
    return fill_backward_impl<float, double>(ctx, n_elements, pos_xy, r, grad_z, ld, grad_pos, grad_eps_h);
  return fill_backward_impl<float, float>(ctx, n_elements, pos_xy, r, grad_z, ld, grad_pos, grad_eps_h);
}

cfft_status cfft_fill_backward_residual(cfft_ctx* ctx, int n_elements, const double* pos_xy, const int* rot,
                                        const void* v, const void* resid, int complex128, double* grad_pos,
                                        double* grad_eps_h) {
  if (!ctx) return CFFT_ERR_ARG;
  if (!v || !resid) return fail(ctx, CFFT_ERR_ARG, "null v or residual");
  const int64_t n = (int64_t)n_elements * ctx->n_mbf;
  cfft_status s = check_fill_args(ctx, n_elements, pos_xy, rot, const_cast<void*>(resid), n);
  if (s != CFFT_OK) return s;
  if (!grad_pos && !grad_eps_h) return fail(ctx, CFFT_ERR_ARG, "nothing to compute");
  DeviceGuard g(ctx->device);
  // dL/dZ' = 2 r v^H, formed in the context's scratch, then the general adjoint
  const size_t es = complex128 ? 16 : 8;
  CFFT_CUDA(ctx->d_gres.ensure((size_t)n * (size_t)n * es), "alloc dL/dZ'");
  cudaError_t e = complex128 ? launch_residual_outer<double>(resid, v, (int)n, ctx->d_gres.p, ctx->stream)
                             : launch_residual_outer<float>(resid, v, (int)n, ctx->d_gres.p, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "residual outer-product kernel");
  return cfft_fill_backward(ctx, n_elements, pos_xy, rot, ctx->d_gres.p, n, complex128, grad_pos, grad_eps_h);
}

cfft_status cfft_get_info(const cfft_ctx* ctx, cfft_info* info) {
  if (!ctx || !info) return CFFT_ERR_ARG;
  if (!ctx->has_table) return CFFT_ERR_STATE;
  *info = ctx->info;
  return CFFT_OK;
}

cfft_status cfft_debug_buffer(const cfft_ctx* ctx, const char* name, const void** dev_ptr,
                              int64_t shape[4]) {
  if (!ctx || !name || !dev_ptr || !shape) return CFFT_ERR_ARG;
  if (!ctx->has_table) return CFFT_ERR_STATE;
  const int64_t pairs = (int64_t)ctx->n_mbf * ctx->n_mbf;
  if (std::strcmp(name, "harmonics") == 0) {
    *dev_ptr = ctx->d_y.p;
    shape[0] = ctx->cls_computed;
    shape[1] = pairs;
    shape[2] = 2 * ctx->q_max + 1;
    shape[3] = ctx->n;
    return CFFT_OK;
  }
  if (std::strcmp(name, "grid") == 0) {
    *dev_ptr = ctx->d_grid.p;
    shape[0] = ctx->cls_computed;
    shape[1] = pairs;
    shape[2] = 2 * ctx->q_max + 1;
    shape[3] = 2 * (int64_t)ctx->info.grid_half + 1;
    return CFFT_OK;
  }
  if (std::strcmp(name, "contour") == 0) {
    *dev_ptr = ctx->beta_c.p;  // beta_c then weight are separate buffers: expose beta_c
    shape[0] = 1;
    shape[1] = ctx->n;
    shape[2] = 1;
    shape[3] = 1;
    return CFFT_OK;
  }
  return CFFT_ERR_ARG;
}

cfft_status cfft_synchronize(cfft_ctx* ctx) {
  if (!ctx) return CFFT_ERR_ARG;
  DeviceGuard g(ctx->device);
  CFFT_CUDA(cudaStreamSynchronize(ctx->stream), "synchronize");
  return CFFT_OK;
}

}  // extern "C"

namespace {

// device copies of the element for the tensor-core spectra (built once per element)
cfft_status ensure_tc_element(cfft_ctx* ctx) {
  if (ctx->tc_ready) return CFFT_OK;
  for (const ShapeClass& c : ctx->shapes)
    if (c.kind != 0) return fail(ctx, CFFT_ERR_ARG, "tensor-core spectra: rooftop elements only");
  const int n_shape = (int)ctx->shapes.size();
  if (spectra_tc_columns(n_shape, ctx->n_mbf) == 0)
    return fail(ctx, CFFT_ERR_ARG, "tensor-core spectra: too many rooftop shapes x MBFs for one GEMM tile");
  std::vector<int> cls(ctx->n_basis);
  for (int s = 0; s < n_shape; ++s)
    for (int i = ctx->shapes[s].begin; i < ctx->shapes[s].end; ++i) cls[i] = s;
  std::vector<float> bm, bmm;
  spectra_tc_bmatrix(ctx->n_basis, n_shape, cls.data(), ctx->n_mbf,
                     reinterpret_cast<const double*>(ctx->q.data()), ctx->n_mbf_pad, false, &bm);
  spectra_tc_bmatrix(ctx->n_basis, n_shape, cls.data(), ctx->n_mbf,
                     reinterpret_cast<const double*>(ctx->q.data()), ctx->n_mbf_pad, true, &bmm);
  std::vector<float> fx(ctx->bx.begin(), ctx->bx.end()), fy(ctx->by.begin(), ctx->by.end());
  double rmax = 0;
  for (size_t i = 0; i < fx.size(); ++i) rmax = std::max(rmax, std::hypot(ctx->bx[i], ctx->by[i]));
  ctx->tc_rmax = (float)(rmax * (1.0 + 1e-6));
  CFFT_CUDA(ctx->tc_bmat.ensure(bm.size() * sizeof(float)), "alloc tensor-core operand");
  CFFT_CUDA(ctx->tc_bmat_mirror.ensure(bmm.size() * sizeof(float)), "alloc tensor-core operand");
  CFFT_CUDA(cudaMemcpy(ctx->tc_bmat_mirror.p, bmm.data(), bmm.size() * sizeof(float), cudaMemcpyHostToDevice),
            "upload");
  CFFT_CUDA(ctx->tc_bx.ensure(fx.size() * sizeof(float)), "alloc element");
  CFFT_CUDA(ctx->tc_by.ensure(fy.size() * sizeof(float)), "alloc element");
  CFFT_CUDA(ctx->tc_shapes.ensure(ctx->shapes.size() * sizeof(ShapeClass)), "alloc element");
  CFFT_CUDA(cudaMemcpy(ctx->tc_bmat.p, bm.data(), bm.size() * sizeof(float), cudaMemcpyHostToDevice), "upload");
  CFFT_CUDA(cudaMemcpy(ctx->tc_bx.p, fx.data(), fx.size() * sizeof(float), cudaMemcpyHostToDevice), "upload");
  CFFT_CUDA(cudaMemcpy(ctx->tc_by.p, fy.data(), fy.size() * sizeof(float), cudaMemcpyHostToDevice), "upload");
  CFFT_CUDA(cudaMemcpy(ctx->tc_shapes.p, ctx->shapes.data(), ctx->shapes.size() * sizeof(ShapeClass),
                       cudaMemcpyHostToDevice), "upload");
  ctx->tc_ready = true;
  return CFFT_OK;
}

}  // namespace

extern "C" void cfft_test_fail_allocation(int after) { g_alloc_countdown = after < 0 ? -1 : after; }

extern "C" cfft_status cfft_selftest_bounded_wait(cfft_ctx* ctx, unsigned polls) {
  if (!ctx) return CFFT_ERR_ARG;
  if (polls < 1 || polls > (1u << 20)) return fail(ctx, CFFT_ERR_ARG, "polls must be in 1 .. 2^20");
  DeviceGuard g(ctx->device);
  CFFT_CUDA(ctx->d_flag.ensure(sizeof(int) * 4), "alloc flag");
  int* flag = ctx->d_flag.as<int>() + 3;
  CFFT_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream), "flag");
  cudaError_t e = launch_wait_selftest(polls, flag, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "bounded-wait self-test kernel");
  int h = 0;
  CFFT_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "flag");
  CFFT_CUDA(cudaStreamSynchronize(ctx->stream), "self-test");
  if (h & 16) return fail(ctx, CFFT_ERR_TIMEOUT, "self-test: the bounded wait ran out (as designed)");
  return CFFT_OK;
}

extern "C" cfft_status cfft_mbf_spectra(cfft_ctx* ctx, int n_points, const void* k, void* out) {
  if (!ctx) return CFFT_ERR_ARG;
  if (n_points < 0 || (n_points > 0 && (!k || !out))) return fail(ctx, CFFT_ERR_ARG, "bad spectra arguments");
  if (!ctx->has_el) return fail(ctx, CFFT_ERR_STATE, "spectra need an element (cfft_set_mbf_spectra)");
  if (n_points == 0) return CFFT_OK;
  DeviceGuard g(ctx->device);
  cfft_status st = ensure_tc_element(ctx);
  if (st != CFFT_OK) return st;
  CFFT_CUDA(ctx->d_flag.ensure(sizeof(int) * 4), "alloc flag");
  int* flag = ctx->d_flag.as<int>() + 2;
  CFFT_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream), "flag");
  cudaError_t e = launch_spectra_tc(n_points, ctx->n_basis, (int)ctx->shapes.size(), ctx->n_mbf,
                                    ctx->tc_shapes.as<ShapeClass>(), ctx->tc_bx.as<float>(),
                                    ctx->tc_by.as<float>(), ctx->tc_bmat.as<float>(), k, out, flag, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tensor-core spectra kernel");
  int h = 0;
  CFFT_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "flag");
  CFFT_CUDA(cudaStreamSynchronize(ctx->stream), "spectra");
  if (h & 16) return fail(ctx, CFFT_ERR_TIMEOUT, "tensor-core spectra: an mbarrier wait ran past its bound");
  return CFFT_OK;
}

// ---------------------------------------------------------------------------
// Reduced MBF system (Section II): excitation, direct solution, port currents.

namespace {

cfft_status upload_quser(cfft_ctx* ctx) {
  const size_t bytes = ctx->q_user.size() * sizeof(std::complex<double>);
  CFFT_CUDA(ctx->d_quser.ensure(bytes), "alloc Q");
  CFFT_CUDA(cudaMemcpyAsync(ctx->d_quser.p, ctx->q_user.data(), bytes, cudaMemcpyHostToDevice, ctx->stream),
            "upload Q");
  return CFFT_OK;
}

cfft_status excitation_call(cfft_ctx* ctx, int kind, int n_el, int port, const void* in, void* out, int c128) {
  if (!ctx) return CFFT_ERR_ARG;
  if (!ctx->has_el) return fail(ctx, CFFT_ERR_STATE, "the excitation needs the element's MBFs (set_mbf_spectra)");
  if (n_el < 1 || !in || !out) return fail(ctx, CFFT_ERR_ARG, "need n_elements >= 1 and device buffers");
  if (kind != 0 && (port < 0 || port >= ctx->n_basis))
    return fail(ctx, CFFT_ERR_ARG, "port must index a basis function of the element");
  DeviceGuard g(ctx->device);
  cfft_status st = upload_quser(ctx);
  if (st != CFFT_OK) return st;
  const double* q = ctx->d_quser.as<double>();
  cudaError_t e = c128 ? launch_excitation<double>(kind, n_el, ctx->n_basis, ctx->n_mbf, port, in, q, out, ctx->stream)
                       : launch_excitation<float>(kind, n_el, ctx->n_basis, ctx->n_mbf, port, in, q, out, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "excitation kernel");
  CFFT_CUDA(cudaStreamSynchronize(ctx->stream), "excitation");   // Q's staging copy is the context's
  return CFFT_OK;
}

cfft_status lu_work(cfft_ctx* ctx, int n, LuWork* w) {
  const int nb = lu_panel_width();
  const int panels = (n + nb - 1) / nb;
  CFFT_CUDA(ctx->lu_moves.ensure((size_t)panels * 2 * nb * sizeof(int2)), "alloc LU");
  CFFT_CUDA(ctx->lu_nmoves.ensure((size_t)panels * sizeof(int)), "alloc LU");
  CFFT_CUDA(ctx->lu_cand_v.ensure((size_t)ctx->sm_count * 2 * sizeof(double)), "alloc LU");
  CFFT_CUDA(ctx->lu_cand_r.ensure((size_t)ctx->sm_count * 2 * sizeof(int)), "alloc LU");
  CFFT_CUDA(ctx->lu_cand_d.ensure((size_t)ctx->sm_count * 2 * nb * 16), "alloc LU");
  CFFT_CUDA(ctx->lu_bar.ensure((size_t)panels * sizeof(unsigned)), "alloc LU");
  CFFT_CUDA(ctx->lu_err.ensure(sizeof(int)), "alloc LU");
  CFFT_CUDA(ctx->lu_sums.ensure(4 * sizeof(double)), "alloc LU");
  w->moves = ctx->lu_moves.as<int2>();
  w->n_moves = ctx->lu_nmoves.as<int>();
  w->cand_val = ctx->lu_cand_v.as<double>();
  w->cand_row = ctx->lu_cand_r.as<int>();
  w->cand_data = ctx->lu_cand_d.p;
  w->diag = ctx->lu_diag;
  w->bar = ctx->lu_bar.as<unsigned>();
  w->err = ctx->lu_err.as<int>();
  w->tc_update = ctx->opt[CFFT_OPT_SOLVE_SIMT] > 0 ? 0 : 1;
  w->panel_cluster = ctx->opt[CFFT_OPT_SOLVE_GRID_PANEL] > 0 ? 0 : 1;
  return CFFT_OK;
}

// factor the context's copy of Z (element type T, dense n x n) and report the panel status
template <class T>
cfft_status lu_factor_checked(cfft_ctx* ctx, int n, const LuWork& w) {
  cudaError_t e = lu_factor<T>(ctx->lu_a.as<cpx<T>>(), n, n, w, ctx->stream);
  if (e != cudaSuccess) {
    cfft_status st = cuda_fail(ctx, e, "LU factorization");
    ctx->err += " (panel grid " + std::to_string(w.diag[0]) + ", resident per SM " + std::to_string(w.diag[1]) +
                ", shared bytes " + std::to_string(w.diag[2]) + ")";
    return st;
  }
  int flag = 0;
  CFFT_CUDA(cudaMemcpyAsync(&flag, w.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "LU flag");
  CFFT_CUDA(cudaStreamSynchronize(ctx->stream), "LU factorization");
  if (flag & 2) return fail(ctx, CFFT_ERR_TIMEOUT, "LU panel: a poll of the pivot keys ran past its bound");
  if (flag & 4) return fail(ctx, CFFT_ERR_NUMERIC, "LU: the reduced matrix is singular (zero pivot)");
  if (flag & 8) return fail(ctx, CFFT_ERR_TIMEOUT, "LU update: a tensor-core wait ran past its bound");
  return CFFT_OK;
}

cfft_status read_sums(cfft_ctx* ctx, double* h, int count) {
  CFFT_CUDA(cudaMemcpyAsync(h, ctx->lu_sums.p, count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "sums");
  CFFT_CUDA(cudaStreamSynchronize(ctx->stream), "sums");
  return CFFT_OK;
}

}  // namespace

extern "C" cfft_status cfft_reduced_excitation(cfft_ctx* ctx, int n_elements, const void* v, void* v_red,
                                               int complex128) {
  return excitation_call(ctx, 0, n_elements, 0, v, v_red, complex128);
}

extern "C" cfft_status cfft_port_excitation(cfft_ctx* ctx, int n_elements, int port, const void* amplitudes,
                                            void* v_red, int complex128) {
  return excitation_call(ctx, 1, n_elements, port, amplitudes, v_red, complex128);
}

extern "C" cfft_status cfft_port_currents(cfft_ctx* ctx, int n_elements, int port, const void* i_red,
                                          void* i_port, int complex128) {
  return excitation_call(ctx, 2, n_elements, port, i_red, i_port, complex128);
}

extern "C" cfft_status cfft_solve_reduced(cfft_ctx* ctx, int n, const void* z, int64_t ld, const void* v,
                                          void* i_out, int complex128, int mode) {
  if (!ctx) return CFFT_ERR_ARG;
  if (n < 1 || n > (1 << 18) || ld < n || !z || !v || !i_out)
    return fail(ctx, CFFT_ERR_ARG, "solve: need 1 <= n <= 262144, ld >= n and device buffers");
  if (mode != 0 && mode != 1) return fail(ctx, CFFT_ERR_ARG, "solve: mode must be 0 or 1");
  if (mode == 1 && !complex128) return fail(ctx, CFFT_ERR_ARG, "solve: refinement needs a complex128 matrix");
  DeviceGuard g(ctx->device);
  cudaStream_t st = ctx->stream;
  for (auto& e : ctx->lu_ev)
    if (!e) CFFT_CUDA(cudaEventCreate(&e), "event");
  LuWork w{};
  cfft_status s = lu_work(ctx, n, &w);
  if (s != CFFT_OK) return s;
  const bool fp64_lu = complex128 && mode == 0;
  // the panel's rows must fit the shared memory of the panel CTAs, and rows and columns are
  // 16-bit fields of the pivot keys
  const int n_lim = std::min(65535, fp64_lu ? lu_max_order<double>(ctx->sm_count) : lu_max_order<float>(ctx->sm_count));
  if (n > n_lim)
    return fail(ctx, CFFT_ERR_ARG, "solve: order " + std::to_string(n) + " exceeds " + std::to_string(n_lim) +
                " (the panel's rows must fit the shared memory of the panel CTAs; pivot keys hold 16-bit rows)");
  const size_t es = fp64_lu ? 16 : 8;
  CFFT_CUDA(ctx->lu_a.ensure((size_t)n * n * es), "alloc LU matrix");
  CFFT_CUDA(ctx->lu_x.ensure((size_t)n * es), "alloc LU vectors");
  CFFT_CUDA(ctx->lu_y.ensure((size_t)n * es), "alloc LU vectors");
  double h[4] = {0, 0, 0, 0};
  int steps = 0;
  CFFT_CUDA(cudaEventRecord(ctx->lu_ev[0], st), "event");
  if (!complex128) {
    CFFT_CUDA((copy_matrix<float, float>(z, ld, n, ctx->lu_a.p, st)), "LU copy");
    if ((s = lu_factor_checked<float>(ctx, n, w)) != CFFT_OK) return s;
    CFFT_CUDA(cudaEventRecord(ctx->lu_ev[1], st), "event");
    CFFT_CUDA((copy_vector<float, float>(v, n, ctx->lu_x.p, st)), "LU copy");
    CFFT_CUDA(lu_solve<float>(ctx->lu_a.as<cpx<float>>(), n, n, w, ctx->lu_x.as<cpx<float>>(),
                              ctx->lu_y.as<cpx<float>>(), st), "LU solve");
    CFFT_CUDA((copy_vector<float, float>(ctx->lu_x.p, n, i_out, st)), "LU copy");
    CFFT_CUDA(cudaEventRecord(ctx->lu_ev[2], st), "event");
    CFFT_CUDA(residual_f32(z, ld, n, i_out, v, ctx->lu_sums.as<double>(), st), "residual");
  } else if (fp64_lu) {
    CFFT_CUDA((copy_matrix<double, double>(z, ld, n, ctx->lu_a.p, st)), "LU copy");
    if ((s = lu_factor_checked<double>(ctx, n, w)) != CFFT_OK) return s;
    CFFT_CUDA(cudaEventRecord(ctx->lu_ev[1], st), "event");
    CFFT_CUDA((copy_vector<double, double>(v, n, ctx->lu_x.p, st)), "LU copy");
    CFFT_CUDA(lu_solve<double>(ctx->lu_a.as<cpx<double>>(), n, n, w, ctx->lu_x.as<cpx<double>>(),
                               ctx->lu_y.as<cpx<double>>(), st), "LU solve");
    CFFT_CUDA((copy_vector<double, double>(ctx->lu_x.p, n, i_out, st)), "LU copy");
    CFFT_CUDA(cudaEventRecord(ctx->lu_ev[2], st), "event");
    CFFT_CUDA(residual_f64(z, ld, n, i_out, v, nullptr, ctx->lu_sums.as<double>(), st), "residual");
  } else {
    // float32 factorization, float64 iterative refinement against the float64 matrix:
    // x_0 = 0, r_0 = v; d = LU^-1 r (float32), x += d, r = v - Z x (float64)
    CFFT_CUDA(ctx->lu_x64.ensure((size_t)n * 16), "alloc LU vectors");
    CFFT_CUDA(ctx->lu_r.ensure((size_t)n * 16), "alloc LU vectors");
    CFFT_CUDA((copy_matrix<float, double>(z, ld, n, ctx->lu_a.p, st)), "LU copy");
    if ((s = lu_factor_checked<float>(ctx, n, w)) != CFFT_OK) return s;
    CFFT_CUDA(cudaEventRecord(ctx->lu_ev[1], st), "event");
    CFFT_CUDA(cudaMemsetAsync(ctx->lu_x64.p, 0, (size_t)n * 16, st), "LU zero");
    CFFT_CUDA((copy_vector<double, double>(v, n, ctx->lu_r.p, st)), "LU copy");
    double rr_prev = -1.0;
    for (steps = 1; steps <= 30; ++steps) {
      CFFT_CUDA((copy_vector<float, double>(ctx->lu_r.p, n, ctx->lu_x.p, st)), "LU copy");
      CFFT_CUDA(lu_solve<float>(ctx->lu_a.as<cpx<float>>(), n, n, w, ctx->lu_x.as<cpx<float>>(),
                                ctx->lu_y.as<cpx<float>>(), st), "LU solve");
      CFFT_CUDA(add_correction(ctx->lu_x64.p, ctx->lu_x.p, n, ctx->lu_sums.as<double>() + 2, st), "refinement");
      CFFT_CUDA(residual_f64(z, ld, n, ctx->lu_x64.p, v, ctx->lu_r.p, ctx->lu_sums.as<double>(), st), "residual");
      if ((s = read_sums(ctx, h, 4)) != CFFT_OK) return s;
      const double rr = h[0], dd = h[2], xx = h[3];
      // stop when the correction is below float64 resolution or the residual stops falling
      if (!(dd > 1e-30 * xx) || (rr_prev >= 0.0 && rr > 0.25 * rr_prev)) break;
      rr_prev = rr;
    }
    if (steps > 30) steps = 30;
    CFFT_CUDA((copy_vector<double, double>(ctx->lu_x64.p, n, i_out, st)), "LU copy");
    CFFT_CUDA(cudaEventRecord(ctx->lu_ev[2], st), "event");
    CFFT_CUDA(residual_f64(z, ld, n, i_out, v, nullptr, ctx->lu_sums.as<double>(), st), "residual");
  }
  if ((s = read_sums(ctx, h, 2)) != CFFT_OK) return s;
  float ms = 0.f;
  cfft_solve_info& in = ctx->solve_info;
  in = cfft_solve_info{};
  if (cudaEventElapsedTime(&ms, ctx->lu_ev[0], ctx->lu_ev[1]) == cudaSuccess) in.ms_factor = ms;
  if (cudaEventElapsedTime(&ms, ctx->lu_ev[1], ctx->lu_ev[2]) == cudaSuccess) in.ms_solve = ms;
  in.residual = h[1] > 0 ? std::sqrt(h[0] / h[1]) : 0.0;
  in.n = n;
  in.mode = mode;
  in.refinements = steps;
  in.panel_width = lu_panel_width();
  in.update_tc = (w.tc_update && (!complex128 || mode == 1)) ? 1 : 0;   // complex64 factorization
  in.cluster_panels = w.diag[3];
  in.panel_cluster = w.diag[3] > 0 ? w.diag[4] : 0;
  if (!std::isfinite(in.residual)) return fail(ctx, CFFT_ERR_NUMERIC, "solve: non-finite solution");
  return CFFT_OK;
}

extern "C" cfft_status cfft_get_solve_info(const cfft_ctx* ctx, cfft_solve_info* info) {
  if (!ctx || !info) return CFFT_ERR_ARG;
  *info = ctx->solve_info;
  return CFFT_OK;
}

// ---------------------------------------------------------------------------
// The paper's 2-D Cartesian C-FFT (Section III-B-2/3, Eq. 21-24, Appendix I).

namespace {

template <class T>
cfft_status cartesian_impl(cfft_ctx* ctx, int n, double rho_max, int order) {
  cudaStream_t st = ctx->stream;
  const int m = ctx->n_mbf, pairs = m * m, p = 2 * n;
  const size_t es = sizeof(cpx<T>);
  // element data in T (bases sorted by shape class, Q padded)
  std::vector<T> hx(ctx->n_basis), hy(ctx->n_basis);
  std::vector<cpx<T>> hq((size_t)ctx->n_basis * ctx->n_mbf_pad);
  for (int i = 0; i < ctx->n_basis; ++i) {
    hx[i] = (T)ctx->bx[i];
    hy[i] = (T)ctx->by[i];
  }
  for (size_t i = 0; i < hq.size(); ++i) hq[i] = mk((T)ctx->q[i].real(), (T)ctx->q[i].imag());
  CFFT_CUDA(ctx->d_bx.ensure(hx.size() * sizeof(T)), "alloc element");
  CFFT_CUDA(ctx->d_by.ensure(hy.size() * sizeof(T)), "alloc element");
  CFFT_CUDA(ctx->d_q.ensure(hq.size() * sizeof(cpx<T>)), "alloc element");
  CFFT_CUDA(ctx->d_shapes.ensure(ctx->shapes.size() * sizeof(ShapeClass)), "alloc element");
  CFFT_CUDA(cudaMemcpyAsync(ctx->d_bx.p, hx.data(), hx.size() * sizeof(T), cudaMemcpyHostToDevice, st), "upload");
  CFFT_CUDA(cudaMemcpyAsync(ctx->d_by.p, hy.data(), hy.size() * sizeof(T), cudaMemcpyHostToDevice, st), "upload");
  CFFT_CUDA(cudaMemcpyAsync(ctx->d_q.p, hq.data(), hq.size() * sizeof(cpx<T>), cudaMemcpyHostToDevice, st), "upload");
  CFFT_CUDA(cudaMemcpyAsync(ctx->d_shapes.p, ctx->shapes.data(), ctx->shapes.size() * sizeof(ShapeClass),
                            cudaMemcpyHostToDevice, st), "upload");
  CFFT_CUDA(cudaStreamSynchronize(st), "upload");   // the staging vectors die at scope end
  const size_t big = (size_t)pairs * p * p * es;
  CFFT_CUDA(ctx->c_tab.ensure(big), "alloc Cartesian table");
  CFFT_CUDA(ctx->c_work.ensure(big), "alloc Cartesian work");
  CFFT_CUDA(ctx->c_work2.ensure(big), "alloc Cartesian work");
  CFFT_CUDA(ctx->c_im.ensure((size_t)pairs * n * n * es), "alloc Cartesian spectrum");
  CFFT_CUDA(ctx->c_gx.ensure((size_t)n * n * sizeof(T)), "alloc Cartesian spectrum");
  CFFT_CUDA(ctx->c_gy.ensure((size_t)n * n * sizeof(T)), "alloc Cartesian spectrum");
  CFFT_CUDA(ctx->c_flag.ensure(sizeof(int)), "alloc flag");
  CartArgs<T> a{};
  a.n = n;
  a.n_mbf = m;
  a.n_shape = (int)ctx->shapes.size();
  a.q_stride = ctx->n_mbf_pad;
  a.k_max = ctx->beta_max;
  a.dk = 2.0 * ctx->beta_max / n;
  a.beta_p = ctx->beta_p;
  a.height = ctx->height;
  a.eps_r = ctx->eps_r;
  a.hs = ctx->hs;
  a.k0 = ctx->k0;
  {
    double deps = 0.0;
    set_extraction(ctx, ctx->eps_r, &a.extract, &a.eps_eff, &deps);
  }
  a.shapes = ctx->d_shapes.as<ShapeClass>();
  a.bx = ctx->d_bx.as<T>();
  a.by = ctx->d_by.as<T>();
  a.q = ctx->d_q.as<cpx<T>>();
  for (auto& e : ctx->ev)
    if (!e) CFFT_CUDA(cudaEventCreate(&e), "event");
  CFFT_CUDA(cudaEventRecord(ctx->ev[0], st), "event");
  cudaError_t e = cartesian_tabulate<T>(a, order, ctx->c_tab.as<cpx<T>>(), ctx->c_work.as<cpx<T>>(),
                                        ctx->c_work2.as<cpx<T>>(), ctx->c_im.as<cpx<T>>(), ctx->c_gx.as<T>(),
                                        ctx->c_gy.as<T>(), st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "Cartesian C-FFT");
  CFFT_CUDA(cudaEventRecord(ctx->ev[1], st), "event");
  CFFT_CUDA(cudaMemsetAsync(ctx->c_flag.p, 0, sizeof(int), st), "flag");
  launch_nonfinite<T>(ctx->c_tab.as<cpx<T>>(), (int64_t)pairs * p * p, ctx->c_flag.as<int>(), st);
  int flag = 0;
  CFFT_CUDA(cudaMemcpyAsync(&flag, ctx->c_flag.p, sizeof(int), cudaMemcpyDeviceToHost, st), "flag");
  CFFT_CUDA(cudaStreamSynchronize(st), "Cartesian C-FFT");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
  cfft_cartesian_info& in = ctx->c_info;
  in.n_grid = n;
  in.n_table = p;
  in.taylor_order = order;
  in.monomials = (order + 1) * (order + 2) / 2;
  in.complex128 = sizeof(T) == 8;
  in.x0 = -(double)n * kPi / (2.0 * ctx->beta_max);
  in.step = kPi / (2.0 * ctx->beta_max);
  in.rho_max = 0.0;
  in.ms = ms;
  if (flag) return fail(ctx, CFFT_ERR_NUMERIC, "non-finite value in the Cartesian table");
  return CFFT_OK;
}

template <class T, class TO>
cfft_status cartesian_fill_impl(cfft_ctx* ctx, int n_el, const double* pos, void* z, int64_t ld) {
  const cfft_cartesian_info& in = ctx->c_info;
  CFFT_CUDA(ctx->c_flag.ensure(sizeof(int)), "alloc flag");
  CFFT_CUDA(cudaMemsetAsync(ctx->c_flag.p, 0, sizeof(int), ctx->stream), "flag");
  cudaError_t e = cartesian_fill<T, TO>(ctx->c_tab.as<cpx<T>>(), in.n_table, ctx->n_mbf, in.x0, in.step,
                                        in.rho_max, n_el, pos, z, ld, ctx->c_flag.as<int>(), ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "Cartesian fill");
  int flag = 0;
  CFFT_CUDA(cudaMemcpyAsync(&flag, ctx->c_flag.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "flag");
  CFFT_CUDA(cudaStreamSynchronize(ctx->stream), "Cartesian fill");
  if (flag) return fail(ctx, CFFT_ERR_ARG, "an element pair lies beyond the Cartesian table's rho_max");
  return CFFT_OK;
}

}  // namespace

extern "C" cfft_status cfft_tabulate_cartesian(cfft_ctx* ctx, int n_grid, double rho_max, int taylor_order,
                                               cfft_precision precision) {
  if (!ctx) return CFFT_ERR_ARG;
  if (!ctx->has_sub || !ctx->has_el || !ctx->has_contour)
    return fail(ctx, CFFT_ERR_STATE, "the Cartesian tabulation needs substrate, element and contour");
  if (n_grid < 16 || n_grid > 2048 || (n_grid & (n_grid - 1)))
    return fail(ctx, CFFT_ERR_ARG, "n_grid must be a power of two in 16..2048");
  if (precision != CFFT_FP64 && precision != CFFT_FP32_MIXED) return fail(ctx, CFFT_ERR_ARG, "bad precision");
  if (taylor_order < -1 || taylor_order > 40) return fail(ctx, CFFT_ERR_ARG, "taylor_order must be in -1..40");
  const double step = kPi / (2.0 * ctx->beta_max);
  const double x_m = (double)n_grid * kPi / (2.0 * ctx->beta_max);
  if (!(rho_max > 0.0) || !(rho_max <= x_m - 2.0 * step))
    return fail(ctx, CFFT_ERR_ARG, "rho_max must be > 0 and inside the table (below n_grid pi / (2 beta_max) "
                                   "less two steps): raise n_grid");
  const bool fp64 = precision == CFFT_FP64;
  int order = taylor_order;
  if (order < 0) order = auto_taylor(ctx->height * rho_max, fp64 ? 1e-13 : 1e-7);
  if (order < 0 || order > 40)
    return fail(ctx, CFFT_ERR_ARG, "height * rho_max too large: no Taylor order up to 40 converges");
  if (ctx->height == 0.0) order = 0;
  DeviceGuard g(ctx->device);
  ctx->has_ctab = false;
  cfft_status s = fp64 ? cartesian_impl<double>(ctx, n_grid, rho_max, order)
                       : cartesian_impl<float>(ctx, n_grid, rho_max, order);
  if (s != CFFT_OK) return s;
  ctx->c_info.rho_max = rho_max;
  ctx->has_ctab = true;
  return CFFT_OK;
}

extern "C" cfft_status cfft_get_cartesian_table(const cfft_ctx* ctx, const void** dev_ptr,
                                                cfft_cartesian_info* info) {
  if (!ctx || !dev_ptr || !info) return CFFT_ERR_ARG;
  if (!ctx->has_ctab) return CFFT_ERR_STATE;
  *dev_ptr = ctx->c_tab.p;
  *info = ctx->c_info;
  return CFFT_OK;
}

extern "C" cfft_status cfft_fill_cartesian(cfft_ctx* ctx, int n_elements, const double* pos_xy, void* z_out,
                                           int64_t ld, int out_complex128) {
  if (!ctx) return CFFT_ERR_ARG;
  if (!ctx->has_ctab) return fail(ctx, CFFT_ERR_STATE, "fill before cfft_tabulate_cartesian");
  if (n_elements < 1 || n_elements > 65535 || !pos_xy || !z_out)
    return fail(ctx, CFFT_ERR_ARG, "need 1..65535 elements and device buffers");
  if (ld < (int64_t)n_elements * ctx->n_mbf) return fail(ctx, CFFT_ERR_ARG, "ld < n_elements * M");
  DeviceGuard g(ctx->device);
  const bool t64 = ctx->c_info.complex128 != 0;
  if (t64 && out_complex128) return cartesian_fill_impl<double, double>(ctx, n_elements, pos_xy, z_out, ld);
  if (t64) return cartesian_fill_impl<double, float>(ctx, n_elements, pos_xy, z_out, ld);
  if (out_complex128) return cartesian_fill_impl<float, double>(ctx, n_elements, pos_xy, z_out, ld);
  return cartesian_fill_impl<float, float>(ctx, n_elements, pos_xy, z_out, ld);
}
