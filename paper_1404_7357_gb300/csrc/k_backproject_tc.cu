// Back-projection (Section III-B-3: Z_q(rho) = 1/(2 pi^2) int_0^pi cos(q alpha)
// g_q(rho cos alpha) d alpha by the midpoint rule, g_q interpolated on the s grid)
// in the paired-harmonic, mirror-folded matrix form of k_backproject.cu, with the
// matrix product on the tensor cores (FP32-mixed).
//
// For |q| = p and one chunk of 16 series (both signs of q: 32 series) the rows r
// of a 256-row tile get
//   Z(r) = sum_k A(r, k) G+(k) + i B(r, k) G-(k),   G+-(k) = G(k) +- (-1)^q G(-k),
// A = sum_l c_l L(u_l - k) Re(ph_l), B = sum_l c_l L(u_l - k) Im(ph_l) over the
// nodes alpha_l <= pi/2.  Per K-tile of 16 grid points this is the real product
//   D (256 x 64) = [A B] (K = 32: A(k), B(k) adjacent) x Bop (32 x 64),
//   Bop(A(k), 2c) = Re G+_c(k), Bop(B(k), 2c) = -Im G-_c(k),
//   Bop(A(k), 2c+1) = Im G+_c(k), Bop(B(k), 2c+1) = Re G-_c(k),
// run as three TF32 products (head x head into one tensor-memory accumulator,
// head x tail + tail x head into a second) and added into FP32 registers after
// every K-tile, so the tensor core's truncating accumulation never spans more
// than four MMA steps.
//
// One thread per row: it adds its nodes' stencils into its own row of [A B],
// stored directly in the no-swizzle K-major operand layout (8-row core matrices
// of 16 bytes = two grid points), with 16-byte read-modify-writes that are
// bank-conflict free across the eight rows of a core matrix; then it splits its
// row into TF32 head (in place) and tail.  The G+- tiles are staged in shared
// memory from coalesced global reads and rearranged into Bop.
#include "cfft_common.cuh"
#include "es_weights.cuh"
#include "spectra_tc.cuh"
#include "tc_sm100.cuh"

namespace cfft {

namespace {

constexpr int kTR = 256;              // rows per tile = threads
constexpr int kTK = 16;               // grid points per K-tile
constexpr int kTKK = 2 * kTK;         // K per tile (A and B of each grid point)
constexpr int kTS = 16;               // series per sign per task
constexpr int kTN = 4 * kTS;          // GEMM columns: 32 series x (re, im)
constexpr int kTGPitch = kTK + 2;     // staged G+- rows (complex entries)
constexpr uint32_t kTSbo = (kTKK / 4) * 128;   // 8-row group stride of the operands

struct TcLayout {
  size_t ahi, alo, bhi, blo, gp, gm, nodes;
};

__host__ __device__ constexpr TcLayout tc_layout() {
  return TcLayout{0,
                  (size_t)kTR * kTKK * 4,
                  (size_t)2 * kTR * kTKK * 4,
                  (size_t)2 * kTR * kTKK * 4 + (size_t)kTN * kTKK * 4,
                  (size_t)2 * kTR * kTKK * 4 + (size_t)2 * kTN * kTKK * 4,
                  (size_t)2 * kTR * kTKK * 4 + (size_t)2 * kTN * kTKK * 4 + (size_t)2 * kTS * kTGPitch * 8,
                  (size_t)2 * kTR * kTKK * 4 + (size_t)2 * kTN * kTKK * 4 + (size_t)4 * kTS * kTGPitch * 8};
}

size_t tc_bp_smem_bytes(int n_nodes_max) {
  const int n_half = (n_nodes_max + 1) / 2;
  return tc_layout().nodes + (size_t)n_half * 12 + 128;   // + base alignment slack
}

// tap m of a stencil's weights, zero outside 0..TAPS-1 (m is a constant after unrolling)
template <int TAPS>
__device__ __forceinline__ float wsel(const float* w, int m) {
  return (m >= 0 && m < TAPS) ? w[m < 0 ? 0 : (m >= TAPS ? TAPS - 1 : m)] : 0.f;
}

// byte offset of the 16-byte group (row, k4) of a K-major operand with K = kTKK
__device__ __forceinline__ uint32_t op_off(int row, int k4) {
  return (uint32_t)(row >> 3) * kTSbo + (uint32_t)k4 * 128u + (uint32_t)(row & 7) * 16u;
}

// one (tile, |q| = p, series chunk) task.  n_commit counts the completions of mbar this
// CTA has waited for (the parity of the next one), n_issued (thread 0) the commits it
// made; fail is the CTA's timeout flag: once set, no MMA is issued and no wait is made.
// KERN: the stencil weights, 0 Lagrange (grid of g itself), 1 ES (precorrected grid)
template <int TAPS, int KERN>
__device__ __forceinline__ void bp_tc_task(const BackprojArgs<float>& a, int tile, int p, int chunk,
                                           unsigned char* base, uint64_t* mbar, uint32_t tmem,
                                           uint32_t& n_commit, uint32_t& n_issued, int* fail) {
  constexpr int HALF = TAPS / 2 - 1;
  constexpr TcLayout LY = tc_layout();
  const int S = a.series_per_q;
  const int r0 = tile * kTR;
  const int r1 = min(r0 + kTR, a.n_rho);
  const int np = a.chunk_nodes[tile];
  const int nhalf = (np + 1) / 2;            // nodes with alpha <= pi / 2
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* Ahi = reinterpret_cast<float*>(base + LY.ahi);
  float* Alo = reinterpret_cast<float*>(base + LY.alo);
  float* Bhi = reinterpret_cast<float*>(base + LY.bhi);
  float* Blo = reinterpret_cast<float*>(base + LY.blo);
  cpx<float>* Gp = reinterpret_cast<cpx<float>*>(base + LY.gp);   // G(k) [series][kk]
  cpx<float>* Gm = reinterpret_cast<cpx<float>*>(base + LY.gm);   // G(-k) [series][kk]
  float2* scos = reinterpret_cast<float2*>(base + LY.nodes);      // cos alpha as float hi + lo
  float* scq = reinterpret_cast<float*>(scos + nhalf);             // cos(p alpha), middle node halved
  const int four_np = 4 * np;
  for (int t = tid; t < nhalf; t += blockDim.x) {
    const double c = a.cosv[a.chunk_off[tile] + t];
    const float hi = (float)c;
    scos[t] = make_float2(hi, (float)(c - (double)hi));
    const int e = (int)(((int64_t)p * (2 * t + 1)) % four_np);
    float cq = cospif((float)e / (float)(2 * np));
    if (2 * t + 1 == np) cq *= 0.5f;
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
  const int r = r0 + tid;
  const bool row_ok = r < r1;
  const double arow = (double)r * a.d_rho / a.d_s;
  const float inv_arow = arow > 0.0 ? (float)(1.0 / arow) : 0.f;
  const float ahi = (float)arow, alo = (float)(arow - (double)ahi);
  const float inv_sigma = 1.0f / (float)a.sigma;
  const float scale = (float)np / 3.14159265f;
  const double rho_top = (r1 - 1) * a.d_rho;
  const int kmax = min(a.grid_half - 1, (int)ceil(rho_top / a.d_s) + TAPS);
  const int k_first = -HALF - 1, n_ktiles = (kmax - k_first + kTK) / kTK;
  const int qi_pos = a.q_max + p, qi_neg = a.q_max - p;
  const float par = (p & 1) ? -1.f : 1.f;   // (-1)^q, the same for q and -q
  float acc[kTN];                            // (re, im) of the 32 series of this row
#pragma unroll
  for (int j = 0; j < kTN; ++j) acc[j] = 0.f;
  const uint32_t idesc = tc::idesc_tf32(128, kTN);
  const uint32_t tl = (uint32_t)(32 * (warp & 3)) << 16;     // this warp's TMEM lanes
  const uint32_t tcol = (uint32_t)((warp >> 2) * 2 * kTN);   // its M-tile's accumulators
  __syncthreads();

  // add the finished K-tile's products (tensor memory) into the row's registers
  auto failed = [&]() { return *reinterpret_cast<volatile int*>(fail) != 0; };
  auto drain = [&]() {
    if (lane == 0 && !failed() && !tc::mbar_wait(mbar, n_commit & 1u, kTcPolls)) atomicOr(fail, 1);
    __syncwarp();
    ++n_commit;
    tc::fence_after_sync();
    // warp-uniform decision: the tensor-memory loads are warp-collective
    if (__shfl_sync(0xffffffffu, failed() ? 0 : 1, 0)) {
#pragma unroll
      for (int cb = 0; cb < kTN; cb += 16) {
        float v[16], w[16];
        tc::tmem_ld16x2(tmem + tl + tcol + cb, tmem + tl + tcol + kTN + cb, v, w);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[cb + j] += v[j] + w[j];
      }
    }
    tc::fence_before_sync();
  };

  // this thread's two (series, grid point) entries of the folded grid tiles
  constexpr int kGPer = kTK * 2 * kTS / kTR;
  static_assert(kGPer * kTR == kTK * 2 * kTS, "grid-tile entries per thread");
  for (int kt = 0; kt < n_ktiles; ++kt) {
    const int k0 = k_first + kt * kTK;
    if (kt > 0) drain();
    // grid values G(k), G(-k) of this K-tile into the staging tiles by asynchronous copies
    // (zero-filled outside the grid and for absent series), waited for after the stencils
#pragma unroll
    for (int u = 0; u < kGPer; ++u) {
      const int t = tid + kTR * u;
      const int c = t / kTK, kk = t - c * kTK;
      const int k = k0 + kk;
      const int g = chunk * kTS + (c & (kTS - 1));
      const int qi = c < kTS ? qi_pos : qi_neg;
      const bool have = g < S && (c < kTS || p > 0);
      const cpx<float>* src = a.grid + ((size_t)(have ? g : 0) * a.n_harm + qi) * (2 * a.grid_half + 1) + a.grid_half;
      const bool in_k = have && k >= -a.grid_half && k <= a.grid_half;
      const bool in_n = have && -k >= -a.grid_half && -k <= a.grid_half;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(tc::smem_u32(Gp + c * kTGPitch + kk)),
                   "l"(in_k ? src + k : a.grid), "r"(in_k ? 8 : 0)
                   : "memory");
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(tc::smem_u32(Gm + c * kTGPitch + kk)),
                   "l"(in_n ? src - k : a.grid), "r"(in_n ? 8 : 0)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    // ---- this thread's row of [A B]: zero, add the stencils of its nodes, split
    {
      const uint32_t rowoff = op_off(tid, 0);
#pragma unroll
      for (int k4 = 0; k4 < kTKK / 4; ++k4)
        *reinterpret_cast<float4*>(reinterpret_cast<char*>(Ahi) + rowoff + 128u * k4) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (row_ok) {
      int lo = 0, hi = -1;
      if (!(arow > 0.0)) {
        if (k0 <= TAPS - 1 - HALF && k0 + kTK - 1 >= -HALF) { lo = 0; hi = nhalf - 1; }
      } else {
        // stencil bases b with [b - HALF, b - HALF + TAPS - 1] meeting [k0, k0 + TK),
        // among the nodes with u >= 0
        const float chi = fminf(1.0f, (float)(k0 + kTK + HALF) * inv_arow);
        const float clo = fmaxf(0.0f, (float)(k0 + HALF - TAPS + 1) * inv_arow);
        if (chi >= clo) {
          lo = max((int)floorf(acosf(chi) * scale - 0.5f) - 1, 0);
          hi = min((int)ceilf(acosf(clo) * scale - 0.5f) + 1, nhalf - 1);
        }
      }
      char* arow_p = reinterpret_cast<char*>(Ahi) + op_off(tid, 0);
      for (int l = lo; l <= hi; ++l) {
        const float2 nc = scos[l];
        float pr = ahi * nc.x;
        float e = fmaf(ahi, nc.x, -pr);
        e = fmaf(ahi, nc.y, e);
        e = fmaf(alo, nc.x, e);
        float fl = floorf(pr);
        float f = (pr - fl) + e;
        if (f < 0.f) { f += 1.f; fl -= 1.f; }
        if (f >= 1.f) { f -= 1.f; fl += 1.f; }
        const int kb = (int)fl - HALF - k0;   // tile column of tap 0
        if (kb + TAPS - 1 < 0 || kb >= kTK) continue;
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
        // 16-byte groups (two grid points) kb/2 .. kb/2 + TAPS/2: taps 2j - odd, 2j + 1 - odd
        const int odd = kb & 1;
        const int g0 = (kb - odd) / 2;
#pragma unroll
        for (int j = 0; j <= TAPS / 2; ++j) {
          const int g = g0 + j;
          if (g < 0 || g >= kTK / 2) continue;
          // taps 2j - odd and 2j + 1 - odd (constant indices, the parity selects)
          const float wa = wsel<TAPS>(w, 2 * j - 1), wb = wsel<TAPS>(w, 2 * j), wc = wsel<TAPS>(w, 2 * j + 1);
          const float w0 = odd ? wa : wb, w1 = odd ? wb : wc;
          float4* q = reinterpret_cast<float4*>(arow_p + 128 * g);
          float4 v = *q;
          v.x = fmaf(wr, w0, v.x);
          v.y = fmaf(wi, w0, v.y);
          v.z = fmaf(wr, w1, v.z);
          v.w = fmaf(wi, w1, v.w);
          *q = v;
        }
      }
    }
    {
      // head (in place) and tail of the row
      const uint32_t rowoff = op_off(tid, 0);
#pragma unroll
      for (int k4 = 0; k4 < kTKK / 4; ++k4) {
        float4* ph = reinterpret_cast<float4*>(reinterpret_cast<char*>(Ahi) + rowoff + 128u * k4);
        float4* pl = reinterpret_cast<float4*>(reinterpret_cast<char*>(Alo) + rowoff + 128u * k4);
        const float4 v = *ph;
        float4 h, t;
        tf32_split(v.x, h.x, t.x);
        tf32_split(v.y, h.y, t.y);
        tf32_split(v.z, h.z, t.z);
        tf32_split(v.w, h.w, t.w);
        *ph = h;
        *pl = t;
      }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    // ---- Bop (64 columns x K 32): column n = 2c + part, K group k4 = grid points 2 k4, 2 k4 + 1
    for (int t = tid; t < kTN * (kTKK / 4); t += blockDim.x) {
      const int n = t & (kTN - 1), k4 = t / kTN;
      const int c = n >> 1;
      // G(kk), G(kk + 1) and G(-kk), G(-kk - 1), folded: G+- = G(k) +- (-1)^q G(-k)
      const float4 gk = *reinterpret_cast<const float4*>(Gp + c * kTGPitch + 2 * k4);
      const float4 gn = *reinterpret_cast<const float4*>(Gm + c * kTGPitch + 2 * k4);
      const float4 gp = make_float4(fmaf(par, gn.x, gk.x), fmaf(par, gn.y, gk.y), fmaf(par, gn.z, gk.z),
                                    fmaf(par, gn.w, gk.w));
      const float4 gm = make_float4(fmaf(-par, gn.x, gk.x), fmaf(-par, gn.y, gk.y), fmaf(-par, gn.z, gk.z),
                                    fmaf(-par, gn.w, gk.w));
      float4 v;
      if ((n & 1) == 0) v = make_float4(gp.x, -gm.y, gp.z, -gm.w);   // real part of the series
      else v = make_float4(gp.y, gm.x, gp.w, gm.z);                   // imaginary part
      float4 h, tl4;
      tf32_split(v.x, h.x, tl4.x);
      tf32_split(v.y, h.y, tl4.y);
      tf32_split(v.z, h.z, tl4.z);
      tf32_split(v.w, h.w, tl4.w);
      *reinterpret_cast<float4*>(reinterpret_cast<char*>(Bhi) + op_off(n, k4)) = h;
      *reinterpret_cast<float4*>(reinterpret_cast<char*>(Blo) + op_off(n, k4)) = tl4;
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && !failed()) {
      tc::fence_after_sync();
      const uint32_t bh = tc::smem_u32(Bhi), bl = tc::smem_u32(Blo);
#pragma unroll
      for (int mt = 0; mt < kTR / 128; ++mt) {
        const uint32_t ah = tc::smem_u32(Ahi) + (uint32_t)mt * 16u * kTSbo;
        const uint32_t al = tc::smem_u32(Alo) + (uint32_t)mt * 16u * kTSbo;
        const uint32_t d_big = tmem + (uint32_t)(mt * 2 * kTN), d_small = d_big + (uint32_t)kTN;
#pragma unroll
        for (int s = 0; s < kTKK / 8; ++s) {
          const uint32_t ko = s * 256;
          const uint64_t dah = tc::sdesc(ah + ko, 128, kTSbo), dal = tc::sdesc(al + ko, 128, kTSbo);
          const uint64_t dbh = tc::sdesc(bh + ko, 128, kTSbo), dbl = tc::sdesc(bl + ko, 128, kTSbo);
          const uint32_t accf = s > 0 ? 1u : 0u;
          tc::mma_tf32(d_small, dah, dbl, idesc, accf);
          tc::mma_tf32(d_small, dal, dbh, idesc, 1u);
          tc::mma_tf32(d_big, dah, dbh, idesc, accf);
        }
      }
      tc::mma_commit(mbar);
      ++n_issued;
    }
  }
  drain();
  const float norm = (float)(1.0 / (2.0 * 3.14159265358979323846 * (double)np));
  if (row_ok && !failed()) {
#pragma unroll
    for (int c = 0; c < 2 * kTS; ++c) {
      const int g = chunk * kTS + (c & (kTS - 1));
      if (g >= S || (c >= kTS && p == 0)) continue;
      const int qi = c < kTS ? qi_pos : qi_neg;
      a.table[((size_t)g * a.n_harm + qi) * a.n_rho + r] = mk(acc[2 * c] * norm, acc[2 * c + 1] * norm);
    }
  }
  __syncthreads();   // the next task reuses the shared buffers
}

// CTA setup shared by the one-shot and the persistent kernels: aligned base, mbarrier,
// 256 tensor-memory columns (2 M-tiles x (head x head, corrections) x 64)
struct TcCta {
  unsigned char* base;
  uint64_t* mbar;
  uint32_t tmem;
};

__device__ __forceinline__ TcCta tc_cta_setup(unsigned char* smem_raw, uint64_t* mbar_s, uint32_t* taddr_s) {
  TcCta c;
  c.base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  c.mbar = mbar_s;
  if (threadIdx.x == 0) {
    tc::mbar_init(mbar_s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if ((threadIdx.x >> 5) == 0) {
    tc::tmem_alloc(taddr_s, 256);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  c.tmem = *taddr_s;
  return c;
}

// after a timed-out wait, a bounded wait for the last commit before the tensor memory is freed
__device__ __forceinline__ void tc_cta_teardown(const TcCta& c, int fail, uint32_t n_issued, int* err) {
  if (fail && threadIdx.x == 0) {
    if (err) atomicOr(err, 32);
    if (n_issued > 0) tc::mbar_wait(c.mbar, (n_issued - 1) & 1u, kTcPolls);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(c.tmem, 256);
}

template <int TAPS, int KERN>
__global__ void __launch_bounds__(kTR, 2) backproject_tc_kernel(BackprojArgs<float> a, int n_tiles, int n_p,
                                                                int n_chunk) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t mbar_s;
  __shared__ uint32_t taddr_s;
  __shared__ int s_fail;
  if (threadIdx.x == 0) s_fail = 0;
  const TcCta cta = tc_cta_setup(smem_raw, &mbar_s, &taddr_s);
  const int per_tile = n_p * n_chunk;
  const int t = blockIdx.x;
  const int tile = n_tiles - 1 - t / per_tile;   // larger rho tiles (more work) first
  const int rem = t - (t / per_tile) * per_tile;
  uint32_t n_commit = 0, n_issued = 0;
  bp_tc_task<TAPS, KERN>(a, tile, rem / n_chunk, rem - (rem / n_chunk) * n_chunk, cta.base, cta.mbar,
                         cta.tmem, n_commit, n_issued, &s_fail);
  tc_cta_teardown(cta, s_fail, n_issued, a.err);
}

// persistent form over (item, |q|, tile, series chunk) tasks
template <int TAPS, int KERN>
__global__ void __launch_bounds__(kTR, 2)
backproject_tc_batch_kernel(const BackprojArgs<float>* items, const int4* tasks, int n_tasks, int* counter) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t mbar_s;
  __shared__ uint32_t taddr_s;
  __shared__ int s_fail;
  __shared__ int s_task;
  if (threadIdx.x == 0) s_fail = 0;
  const TcCta cta = tc_cta_setup(smem_raw, &mbar_s, &taddr_s);
  uint32_t n_commit = 0, n_issued = 0;
  int* err = nullptr;
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= n_tasks) break;
    const int4 tk = tasks[t];
    const BackprojArgs<float> a = items[tk.x];
    err = a.err;
    bp_tc_task<TAPS, KERN>(a, tk.z, tk.y, tk.w, cta.base, cta.mbar, cta.tmem, n_commit, n_issued, &s_fail);
  }
  tc_cta_teardown(cta, s_fail, n_issued, err);
}

template <int TAPS, int KERN>
cudaError_t launch_tc_taps(const BackprojArgs<float>& a, int n_tiles, int max_nodes, cudaStream_t s) {
  const size_t smem = tc_bp_smem_bytes(max_nodes);
  cudaError_t e = cudaFuncSetAttribute(backproject_tc_kernel<TAPS, KERN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int n_p = a.q_max + 1;
  const int n_chunk = (a.series_per_q + kTS - 1) / kTS;
  backproject_tc_kernel<TAPS, KERN><<<n_tiles * n_p * n_chunk, kTR, smem, s>>>(a, n_tiles, n_p, n_chunk);
  return cudaGetLastError();
}

template <int TAPS, int KERN>
cudaError_t launch_tc_batch_taps(const BackprojArgs<float>* items, const int4* tasks, int n_tasks, int* counter,
                                 int max_nodes, int n_ctas, cudaStream_t s) {
  const size_t smem = tc_bp_smem_bytes(max_nodes);
  cudaError_t e = cudaFuncSetAttribute(backproject_tc_batch_kernel<TAPS, KERN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // at most two CTAs per SM: their tensor memory (2 x 256 columns) then always fits
  backproject_tc_batch_kernel<TAPS, KERN><<<2 * n_ctas, kTR, smem, s>>>(items, tasks, n_tasks, counter);
  return cudaGetLastError();
}

}  // namespace

size_t backproject_tc_smem(int max_nodes) { return tc_bp_smem_bytes(max_nodes); }
int backproject_tc_ktile() { return kTK; }

cudaError_t launch_backproject_tc(const BackprojArgs<float>& a, int n_tiles, int max_nodes, cudaStream_t s) {
  if (a.rchunk != kTR) return cudaErrorInvalidValue;
  if (a.kern == 1) {
    switch (a.taps) {
      case 6: return launch_tc_taps<6, 1>(a, n_tiles, max_nodes, s);
      case 8: return launch_tc_taps<8, 1>(a, n_tiles, max_nodes, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (a.taps) {
    case 8: return launch_tc_taps<8, 0>(a, n_tiles, max_nodes, s);
    case 12: return launch_tc_taps<12, 0>(a, n_tiles, max_nodes, s);
    case 16: return launch_tc_taps<16, 0>(a, n_tiles, max_nodes, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_backproject_tc_batch(const BackprojArgs<float>* items, const int4* tasks, int n_tasks,
                                        int* counter, int taps, int kern, int max_nodes, int n_ctas,
                                        cudaStream_t s) {
  if (kern == 1) {
    switch (taps) {
      case 6: return launch_tc_batch_taps<6, 1>(items, tasks, n_tasks, counter, max_nodes, n_ctas, s);
      case 8: return launch_tc_batch_taps<8, 1>(items, tasks, n_tasks, counter, max_nodes, n_ctas, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (taps) {
    case 8: return launch_tc_batch_taps<8, 0>(items, tasks, n_tasks, counter, max_nodes, n_ctas, s);
    case 12: return launch_tc_batch_taps<12, 0>(items, tasks, n_tasks, counter, max_nodes, n_ctas, s);
    case 16: return launch_tc_batch_taps<16, 0>(items, tasks, n_tasks, counter, max_nodes, n_ctas, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cfft
