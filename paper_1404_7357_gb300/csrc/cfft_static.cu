// Allocation-free back-projection entry point (cfft_backproject_static).
//
// Some callers cannot call cudaMalloc: plug-ins hosted by an application that
// owns every device allocation through its own pool, and real-time loops
// where a driver-level allocation (which may synchronize the device) is not
// acceptable.  For them
// this entry point runs the back-projection stage on caller-owned input and
// output buffers and keeps its only scratch -- the angular node counts,
// their offsets and the node cosines of every chunk of rows -- in the
// file-scope device array below, which exists once per GPU that loads the
// library, for as long as the library stays loaded.
#include <cmath>
#include <mutex>

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

// 8 MiB: node counts (int32) and offsets (int64) of up to 65536 chunks of
// 32 rows, then the node cosines (float64) of all chunks.
constexpr size_t kScratchBytes = size_t(8) << 20;
constexpr int kMaxChunks = 65536;
constexpr size_t kCountsBytes = kMaxChunks * sizeof(int);
constexpr size_t kOffsetsBytes = kMaxChunks * sizeof(int64_t);
constexpr size_t kMaxCosines = (kScratchBytes - kCountsBytes - kOffsetsBytes) / sizeof(double);
constexpr int kRowChunk = 32;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_bp_scratch[kScratchBytes];

// device address of g_bp_scratch on each device, looked up once per device
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// the angular node rule of the tabulation, per chunk, and the running offsets
// (cbrt_coef: 2 for complex64 tables, 4 for complex128, as in the tabulation)
__global__ void static_chunk_nodes_kernel(int n_chunks, int n_rho, double d_rho,
                                          double beta_abs_max, int q_max, double margin,
                                          double cbrt_coef, int* nodes, int64_t* offsets) {
  for (int c = threadIdx.x; c < n_chunks; c += blockDim.x) {
    int r_top = min((c + 1) * kRowChunk, n_rho) - 1;
    double z = beta_abs_max * (r_top * d_rho);
    nodes[c] = (int)ceil(0.5 * (z + q_max) + cbrt_coef * cbrt(z) + 0.5 * margin) + 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int c = 0; c < n_chunks; ++c) {
      offsets[c] = t;
      t += nodes[c];
    }
  }
}

int host_nodes(double beta_abs_max, double rho, int q_max, double margin, double cbrt_coef) {
  double z = beta_abs_max * rho;
  return (int)std::ceil(0.5 * (z + q_max) + cbrt_coef * std::cbrt(z) + 0.5 * margin) + 1;
}

template <class T>
cfft_status run(cudaStream_t st, unsigned char* scratch, const void* grid, void* table,
                int series_per_q, int q_max, int n_rho, double rho_max, int grid_half,
                double delta_s, int sigma, int taps, double beta_abs_max, double margin) {
  const int n_chunks = (n_rho + kRowChunk - 1) / kRowChunk;
  const double d_rho = rho_max / (n_rho - 1);
  const double cbrt_coef = sizeof(T) == 8 ? 4.0 : 2.0;
  // the grid must reach rho_max plus half a stencil (compared in floating point, so that
  // no huge ratio is converted to an integer)
  if (std::ceil(rho_max / delta_s) + taps / 2 + 2 > (double)grid_half) return CFFT_ERR_ARG;
  // host-side bounds of the scratch and shared-memory use (the device recomputes the
  // same counts; +2 covers a last-bit difference of cbrt between host and device)
  int64_t total = 0;
  int max_nodes = 0, max_seg = 0;
  for (int c = 0; c < n_chunks; ++c) {
    int r_top = std::min((c + 1) * kRowChunk, n_rho) - 1;
    double rho_top = r_top * d_rho;
    int np = host_nodes(beta_abs_max, rho_top, q_max, margin, cbrt_coef) + 2;
    total += np;
    max_nodes = std::max(max_nodes, np);
    int kseg = std::min(grid_half, (int)std::ceil(rho_top / delta_s) + taps / 2 + 2);
    max_seg = std::max(max_seg, 2 * kseg + 1);
  }
  if (n_chunks > kMaxChunks || (size_t)total > kMaxCosines) return CFFT_ERR_ARG;
  int group = 8;
  const size_t cap = 225 * 1024;
  while (group > 1 && backproject_smem<T>(group, max_seg, max_nodes) > cap) --group;
  if (backproject_smem<T>(group, max_seg, max_nodes) > cap) return CFFT_ERR_ARG;
  group = std::min(group, series_per_q);

  int* nodes = reinterpret_cast<int*>(scratch);
  int64_t* offsets = reinterpret_cast<int64_t*>(scratch + kCountsBytes);
  double* cosv = reinterpret_cast<double*>(scratch + kCountsBytes + kOffsetsBytes);
  // every scratch entry the back-projection reads is rewritten here first
  static_chunk_nodes_kernel<<<1, 1024, 0, st>>>(n_chunks, n_rho, d_rho, beta_abs_max, q_max,
                                                margin, cbrt_coef, nodes, offsets);
  if (cudaGetLastError() != cudaSuccess) return CFFT_ERR_CUDA;
  if (launch_chunk_cosines(nodes, offsets, n_chunks, max_nodes, cosv, st) != cudaSuccess)
    return CFFT_ERR_CUDA;
  BackprojArgs<T> ba{};
  ba.series_per_q = series_per_q;
  ba.n_harm = 2 * q_max + 1;
  ba.q_max = q_max;
  ba.n_rho = n_rho;
  ba.grid_half = grid_half;
  ba.sigma = sigma;
  ba.taps = taps;
  ba.group = group;
  ba.rchunk = kRowChunk;
  ba.d_rho = d_rho;
  ba.d_s = delta_s;
  ba.beta_abs_max = beta_abs_max;
  ba.alpha_margin = margin;
  ba.grid = reinterpret_cast<const cpx<T>*>(grid);
  ba.table = reinterpret_cast<cpx<T>*>(table);
  cudaError_t e = launch_backproject_impl<T>(ba, nodes, offsets, cosv, nullptr, n_chunks,
                                             max_nodes, max_seg, st);
  if (e == cudaErrorInvalidValue) return CFFT_ERR_ARG;
  return e == cudaSuccess ? CFFT_OK : CFFT_ERR_CUDA;
}

}  // namespace

extern "C" cfft_status cfft_backproject_static(int device, void* cuda_stream, const void* grid,
                                               void* table, int series_per_q, int q_max,
                                               int n_rho, double rho_max, int grid_half,
                                               double delta_s, int sigma, int taps,
                                               double beta_abs_max, double alpha_margin,
                                               int complex128) {
  if (!grid || !table || device < 0 || device >= kMaxDevices) return CFFT_ERR_ARG;
  if (series_per_q < 1 || q_max < 0 || q_max > 64 || n_rho < 2 || !(rho_max > 0) ||
      grid_half < 1 || !(delta_s > 0) || sigma < 2 || (sigma & (sigma - 1)) ||
      !(beta_abs_max > 0) || !(alpha_margin > 0) ||
      !(taps == 4 || taps == 6 || taps == 8 || taps == 10 || taps == 12 || taps == 16 || taps == 20 ||
        taps == 24))
    return CFFT_ERR_ARG;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return CFFT_ERR_CUDA;
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return CFFT_ERR_CUDA;
  cfft_status status = CFFT_OK;
  void* addr = nullptr;
  {
    // first call on this device: look the array's device address up with the device current
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[device]) {
      if (cudaGetSymbolAddress(&g_scratch_addr[device], g_bp_scratch) != cudaSuccess) {
        g_scratch_addr[device] = nullptr;
        status = CFFT_ERR_CUDA;
      }
    }
    addr = g_scratch_addr[device];
  }
  if (status == CFFT_OK) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    unsigned char* scratch = reinterpret_cast<unsigned char*>(addr);
    status = complex128
                 ? run<double>(st, scratch, grid, table, series_per_q, q_max, n_rho, rho_max,
                               grid_half, delta_s, sigma, taps, beta_abs_max, alpha_margin)
                 : run<float>(st, scratch, grid, table, series_per_q, q_max, n_rho, rho_max,
                              grid_half, delta_s, sigma, taps, beta_abs_max, alpha_margin);
  }
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return status;
}
