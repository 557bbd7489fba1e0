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
#include "cfft_common.cuh"

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

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t need) {
    if (need <= bytes && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    if (need == 0) need = 16;
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

}  // namespace

struct cfft_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err = "no error";
  // substrate
  bool has_sub = false;
  double eps_r = 1, hs = 0, k0 = 1;
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
  // options (<= 0: automatic)
  double opt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  // table
  bool has_table = false;
  int q_max = 0, n_rho = 0, cls_stored = 1, cls_computed = 1, fill_taps = 8;
  double rho_max = 0;
  cfft_precision prec = CFFT_FP64;
  cfft_info info{};
  // device buffers
  DevBuf beta_c, weight, bw, bi_rel, green_p, green_r;
  DevBuf d_shapes, d_bx, d_by, d_q, d_y, d_grid, d_table, d_tw, d_cnodes, d_coff, d_cos, d_lag,
      d_flag, d_pos, d_rot, d_zbuf;
  int tw_len = 0, tw_prec = -1;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
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

// smallest N_t with x^(N_t+1)/(N_t+1)! e^x <= tol (remainder bound of Eq. 22)
int auto_taylor(double x, double tol) {
  if (x <= 0) return 0;
  for (int nt = 0; nt <= 64; ++nt) {
    double lg = (nt + 1) * std::log(x) - lgamma_fact(nt + 1) + x;
    if (lg <= std::log(tol)) return nt;
  }
  return 64;
}

// angular nodes of the back-projection for the largest rho of a chunk
int alpha_nodes(double beta_abs_max, double rho, int q_max, double margin) {
  double z = beta_abs_max * rho;
  return (int)std::ceil(0.5 * (z + q_max) + 2.0 * std::cbrt(z) + 0.5 * margin) + 1;
}

template <class T>
cfft_status tabulate_impl(cfft_ctx* ctx) {
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
  int bp_taps = (int)ctx->opt[CFFT_OPT_BP_TAPS];
  if (bp_taps <= 0) bp_taps = fp64 ? 16 : 12;
  int fill_taps = (int)ctx->opt[CFFT_OPT_FILL_TAPS];
  if (fill_taps <= 0) fill_taps = fp64 ? 16 : 8;
  if (!(bp_taps == 4 || bp_taps == 6 || bp_taps == 8 || bp_taps == 10 || bp_taps == 12 ||
        bp_taps == 16 || bp_taps == 20 || bp_taps == 24) ||
      fill_taps < 2 || fill_taps > 16 || (fill_taps & 1))
    return fail(ctx, CFFT_ERR_ARG,
                "back-projection taps must be one of 4,6,8,10,12,16,20,24; fill taps even, 2..16");
  if (ctx->n_rho < 2 * fill_taps) return fail(ctx, CFFT_ERR_ARG, "n_rho must be >= 2 * fill taps");
  double margin = ctx->opt[CFFT_OPT_ALPHA_MARGIN] > 0 ? ctx->opt[CFFT_OPT_ALPHA_MARGIN] : 24.0;
  int taylor = ctx->taylor_req;
  if (taylor < 0) taylor = auto_taylor(ctx->height * ctx->rho_max, fp64 ? 1e-13 : 1e-7);
  const int64_t P = (int64_t)sigma * n;
  const double ds = 2.0 * kPi / ((double)P * step);
  const int K = (int)std::ceil(ctx->rho_max / ds) + bp_taps / 2 + 2;
  if (2 * (int64_t)K + 1 > P)
    return fail(ctx, CFFT_ERR_ARG, "rho_max exceeds the unaliased range 2 pi / step of the contour");
  // sub-FFT length: power of two dividing P, within shared memory
  const int l_max = fp64 ? 8192 : 16384;
  int L = 1;
  while ((P % (2 * (int64_t)L)) == 0 && 2 * L <= l_max) L *= 2;
  if (L < 64) return fail(ctx, CFFT_ERR_ARG, "sigma * n must be divisible by 64");
  while (L > 256 && (int64_t)series * (P / L) < 2 * 152) L /= 2;
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
  CFFT_CUDA(ctx->bi_rel.ensure(n * sizeof(double)), "alloc contour");
  CFFT_CUDA(ctx->green_p.ensure(n * sizeof(double2)), "alloc contour");
  CFFT_CUDA(ctx->green_r.ensure(n * sizeof(double2)), "alloc contour");
  CFFT_CUDA(ctx->d_y.ensure((size_t)series * n * sizeof(cpx<T>)), "alloc harmonics");
  CFFT_CUDA(ctx->d_grid.ensure((size_t)series * (2 * K + 1) * sizeof(cpx<T>)), "alloc grid");
  const int cls_s = ctx->cls_stored;
  const size_t table_elems = (size_t)cls_s * pairs * nh * ctx->n_rho;
  CFFT_CUDA(ctx->d_table.ensure(table_elems * sizeof(cpx<T>)), "alloc table");
  CFFT_CUDA(ctx->d_flag.ensure(sizeof(int) * 4), "alloc flag");

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
  ContourData cd{ctx->beta_c.as<double2>(), ctx->weight.as<double2>(), ctx->bw.as<double2>(),
                 ctx->bi_rel.as<double>(), ctx->green_p.as<double2>(), ctx->green_r.as<double2>()};
  int launches = 0;
  launch_contour(ca, cd, st);
  ++launches;
  CFFT_CUDA(cudaGetLastError(), "contour kernel");
  CFFT_CUDA(cudaEventRecord(ctx->ev[1], st), "event");

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
  ia.green_p = ctx->green_p.as<double2>();
  ia.green_r = ctx->green_r.as<double2>();
  ia.y = ctx->d_y.as<cpx<T>>();
  CFFT_CUDA(launch_integrand<T>(ia, ctx->n_mbf_pad, st), "integrand kernel");
  ++launches;
  CFFT_CUDA(cudaEventRecord(ctx->ev[2], st), "event");

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
  fa.n_active = n_active;
  fa.sigma = sigma;
  fa.ds_height = ds * ctx->height;
  fa.y = ctx->d_y.as<cpx<T>>();
  fa.bi_rel = ctx->bi_rel.as<double>();
  fa.twiddle = ctx->d_tw.as<cpx<T>>();
  fa.grid = ctx->d_grid.as<cpx<T>>();
  CFFT_CUDA(launch_fft<T>(fa, st), "fft kernel");
  ++launches;
  CFFT_CUDA(cudaEventRecord(ctx->ev[3], st), "event");

  // ---- a5: back-projection to the rho grid
  const int rchunk = 32;
  const int n_chunks = (ctx->n_rho + rchunk - 1) / rchunk;
  const double d_rho = ctx->rho_max / (ctx->n_rho - 1);
  std::vector<int> cn(n_chunks);
  std::vector<int64_t> coff(n_chunks);
  int64_t tot = 0;
  int max_nodes = 0, max_seg = 0;
  double bp_nodes = 0;
  for (int c = 0; c < n_chunks; ++c) {
    int r_top = std::min((c + 1) * rchunk, ctx->n_rho) - 1;
    double rho_top = r_top * d_rho;
    cn[c] = alpha_nodes(beta_abs_max, rho_top, ctx->q_max, margin);
    bp_nodes += (double)cn[c] * (r_top + 1 - c * rchunk) * series;
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
  CFFT_CUDA(launch_chunk_cosines(ctx->d_cnodes.as<int>(), ctx->d_coff.as<int64_t>(), n_chunks,
                                 max_nodes, ctx->d_cos.as<double>(), st), "cosine kernel");
  ++launches;
  int group = 8;
  const size_t smem_cap = 225 * 1024;
  while (group > 1 && backproject_smem<T>(group, max_seg, max_nodes) > smem_cap) --group;
  if (backproject_smem<T>(group, max_seg, max_nodes) > smem_cap)
    return fail(ctx, CFFT_ERR_ARG, "rho_max too large for one shared-memory segment");
  group = std::min(group, series_per_q);
  BackprojArgs<T> ba{};
  ba.series_per_q = series_per_q;
  ba.n_harm = nh;
  ba.q_max = ctx->q_max;
  ba.n_rho = ctx->n_rho;
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
  ba.table = ctx->d_table.as<cpx<T>>();
  CFFT_CUDA(launch_backproject_impl<T>(ba, ctx->d_cnodes.as<int>(), ctx->d_coff.as<int64_t>(),
                                       ctx->d_cos.as<double>(), ctx->d_lag.as<double>(), n_chunks,
                                       max_nodes, max_seg, st), "backprojection kernel");
  ++launches;
  if (cls_s == 4) {
    launch_class_phase<T>(ctx->d_table.as<cpx<T>>(), pairs, nh, ctx->q_max, ctx->n_rho, st);
    ++launches;
    CFFT_CUDA(cudaGetLastError(), "class phase kernel");
  }
  CFFT_CUDA(cudaEventRecord(ctx->ev[4], st), "event");

  // ---- NaN / Inf check (synchronizes)
  bool check = !(ctx->opt[5] < 0);
  if (check) {
    CFFT_CUDA(cudaMemsetAsync(ctx->d_flag.p, 0, sizeof(int), st), "flag");
    launch_nonfinite<T>(ctx->d_table.as<cpx<T>>(), (int64_t)table_elems, ctx->d_flag.as<int>(), st);
    ++launches;
    CFFT_CUDA(cudaGetLastError(), "nonfinite kernel");
  }
  int flag = 0;
  if (check) CFFT_CUDA(cudaMemcpyAsync(&flag, ctx->d_flag.p, sizeof(int), cudaMemcpyDeviceToHost, st), "flag");
  CFFT_CUDA(cudaStreamSynchronize(st), "tabulate");

  cfft_info& in = ctx->info;
  in.taylor_order = taylor;
  in.n_alpha = n_alpha;
  in.sigma = sigma;
  in.fft_len = (int)P;
  in.sub_len = L;
  in.grid_half = K;
  in.bp_taps = bp_taps;
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
  in.work_subffts = (double)series * D * (taylor + 1);
  in.work_bp_nodes = bp_nodes;
  ctx->fill_taps = fill_taps;
  ctx->has_table = true;
  if (flag) return fail(ctx, CFFT_ERR_NUMERIC, "non-finite value in the reaction table");
  return CFFT_OK;
}

template <class T, class TO>
cfft_status fill_impl(cfft_ctx* ctx, int n_el, const double* pos, const int* rot, void* z,
                      int64_t ld) {
  FillArgs<T, TO> fa{};
  fa.n_el = n_el;
  fa.n_mbf = ctx->n_mbf;
  fa.q_max = ctx->q_max;
  fa.n_harm = 2 * ctx->q_max + 1;
  fa.n_rho = ctx->n_rho;
  fa.taps = ctx->fill_taps;
  fa.n_cls = ctx->cls_stored;
  fa.inv_d_rho = (ctx->n_rho - 1) / ctx->rho_max;
  fa.rho_max = ctx->rho_max;
  fa.ld = ld;
  fa.table = ctx->d_table.as<cpx<T>>();
  fa.pos = pos;
  fa.rot = rot;
  fa.z = reinterpret_cast<cpx<TO>*>(z);
  fa.err = ctx->d_flag.as<int>() + 1;
  CFFT_CUDA(cudaMemsetAsync(fa.err, 0, sizeof(int), ctx->stream), "flag");
  cudaError_t le = launch_fill<T, TO>(fa, ctx->stream);
  if (le != cudaSuccess) return cuda_fail(ctx, le, "fill kernel");
  int flag = 0;
  CFFT_CUDA(cudaMemcpyAsync(&flag, fa.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "flag");
  CFFT_CUDA(cudaStreamSynchronize(ctx->stream), "fill");
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
  *out = c;
  return CFFT_OK;
}

void cfft_destroy(cfft_ctx* ctx) {
  if (!ctx) return;
  {
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    DevBuf* bufs[] = {&ctx->beta_c, &ctx->weight, &ctx->bw, &ctx->bi_rel, &ctx->green_p,
                      &ctx->green_r, &ctx->d_shapes, &ctx->d_bx, &ctx->d_by, &ctx->d_q,
                      &ctx->d_y, &ctx->d_grid, &ctx->d_table, &ctx->d_tw, &ctx->d_cnodes,
                      &ctx->d_coff, &ctx->d_cos, &ctx->d_lag, &ctx->d_flag, &ctx->d_pos,
                      &ctx->d_rot, &ctx->d_zbuf};
    for (DevBuf* b : bufs) b->release();
    for (auto& e : ctx->ev)
      if (e) cudaEventDestroy(e);
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
  ctx->elem_radius = 0.5 * std::hypot(length, width);
  ctx->has_el = true;
  ctx->has_table = false;
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
  ctx->n_basis = n_basis;
  ctx->n_mbf = n_mbf;
  ctx->n_mbf_pad = pad;
  ctx->elem_radius = radius;
  ctx->has_el = true;
  ctx->has_table = false;
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

cfft_status cfft_set_option(cfft_ctx* ctx, cfft_option key, double value) {
  if (!ctx) return CFFT_ERR_ARG;
  if ((int)key < 0 || (int)key > 5) return fail(ctx, CFFT_ERR_ARG, "unknown option");
  ctx->opt[(int)key] = value;
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
  if (precision == CFFT_FP64) return tabulate_impl<double>(ctx);
  return tabulate_impl<float>(ctx);
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
