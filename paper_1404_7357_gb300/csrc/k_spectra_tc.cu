// MBF spectra (Eq. 11, and the analytic continuation of the conjugated basis
// spectrum in Eq. 10) as a complex GEMM on the fifth-generation tensor cores.
//
// For wavevector k_p and rooftop i of shape class s(i) (centre r_i):
//   F_i(k) = E_i(k) S_s(k),  E_i = exp(-i k.r_i),  E'_i = exp(+i k.r_i) = F_i(-k) / S_s
// (S_s is even in k).  The per-class sums
//   T_{s,a}(k) = sum_{i in s} conj(Q_ia) E_i,   B_{s,a}(k) = sum_{i in s} Q_ia E'_i
// are one real GEMM: the A operand holds, per point, the four reals
// (Re E_i, Im E_i, Re E'_i, Im E'_i) of every basis function (K = 4 n_basis),
// the B operand holds the matching combinations of Re/Im Q (a constant of the
// element, built on the host), and the N = 4 n_shape M columns are
// (side, class, MBF, re/im).  The epilogue multiplies by S_s(k) and sums the
// classes of each direction:
//   M_a,d(k)    = sum_{s: dir(s) = d} S_s(k) T_{s,a}(k)
//   Mbar_a,d(k) = sum_{s: dir(s) = d} S_s(k) B_{s,a}(k).
//
// Precision: each FP32 operand X is split X ~ X_hi + X_lo, both used at TF32
// precision (|X - X_hi - X_lo| <= 2^-22 |X|), and each product is formed as
// A_hi B_hi + A_hi B_lo + A_lo B_hi with float32 accumulation in tensor memory.
// The tensor core truncates when it adds into an accumulator, so the head x head
// products and the two (small) correction products go to separate accumulators,
// summed in float32 in the epilogue: measured against the oracle this keeps the
// spectra near float32 accuracy instead of a few 1e-6 worse.
//
// Pipeline per 128-point tile: the K dimension runs in chunks of 8 basis
// functions (K = 32).  All 256 threads generate the A chunk (one point and four
// basis functions each) into shared memory in the no-swizzle K-major
// core-matrix layout while the tensor core consumes the previous chunk (two
// buffers); one thread issues the 12 MMAs of a chunk and commits them to the
// chunk buffer's mbarrier; every wait on an mbarrier is bounded.
#include <cstring>
#include <vector>

#include "cfft_common.cuh"
#include "spectra_tc.cuh"
#include "tc_sm100.cuh"

namespace cfft {

namespace {

constexpr int kTcThreads = 256;
constexpr int kTcRows = 128;               // points per tile = MMA M

struct SpectraTcArgs {
  int n_points, n_basis, n_shape, n_mbf, ncol, ncol_alloc, n_chunks;
  const ShapeClass* shapes;  // device
  const float* bx;           // device, basis centres (sorted by class)
  const float* by;
  const float* bmat;         // device, [chunk][hi, lo][ncol x kTcK] core-matrix layout
  const cpx<float>* k;       // device, [n_points][2]
  cpx<float>* out;           // device, [n_points][2 sides][n_mbf][2 comps]
  int* err;                  // device flag: bit 4 = a tensor-core wait timed out
};

size_t tc_smem_bytes(int ncol, int n_basis) {
  const size_t a = (size_t)2 * 2 * kTcRows * kTcK * sizeof(float);
  const size_t b = (size_t)2 * 2 * ncol * kTcK * sizeof(float);
  const size_t kp = (size_t)kTcRows * 2 * sizeof(cpx<float>);
  const size_t basis = (size_t)2 * ((n_basis + kTcBasis - 1) / kTcBasis * kTcBasis) * sizeof(float);
  return 1024 + a + b + kp + basis + 64;
}

template <int MB>
__global__ void __launch_bounds__(kTcThreads, 1) spectra_tc_kernel(SpectraTcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte aligned base for the operand tiles
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  float* A = reinterpret_cast<float*>(base);                       // [2 buf][hi, lo][128 x 32]
  float* B = A + 2 * 2 * kTcRows * kTcK;                           // [2 buf][hi, lo][ncol x 32]
  cpx<float>* kp = reinterpret_cast<cpx<float>*>(B + 2 * 2 * a.ncol * kTcK);  // [128][2]
  const int nb_pad = a.n_chunks * kTcBasis;
  float* sbx = reinterpret_cast<float*>(kp + 2 * kTcRows);
  float* sby = sbx + nb_pad;
  uint64_t* mbar = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(sby + nb_pad) + 7) & ~(uintptr_t)7);
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(mbar + 2);
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < nb_pad; i += kTcThreads) {
    sbx[i] = i < a.n_basis ? a.bx[i] : 0.f;
    sby[i] = i < a.n_basis ? a.by[i] : 0.f;
  }
  if (tid == 0) {
    s_fail = 0;
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tc::tmem_alloc(taddr_s, (uint32_t)a.ncol_alloc);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *taddr_s;
  const uint32_t idesc = tc::idesc_tf32(kTcRows, a.ncol);
  const uint32_t a_bytes = kTcRows * kTcK * sizeof(float);   // one hi or lo block
  const uint32_t b_bytes = (uint32_t)a.ncol * kTcK * sizeof(float);
  const uint32_t sbo = (kTcK / 4) * 128;                      // 8-row group stride
  const int n_tiles = (a.n_points + kTcRows - 1) / kTcRows;
  const int p = tid & (kTcRows - 1), half = tid >> 7;
  uint32_t stage = 0;   // chunks issued by this CTA so far (mbarrier phase bookkeeping)
  bool issued = false;

  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int p0 = tile * kTcRows;
    if (tid < kTcRows) {
      const int pp = p0 + tid;
      kp[2 * tid] = pp < a.n_points ? a.k[2 * (size_t)pp] : mk(0.f, 0.f);
      kp[2 * tid + 1] = pp < a.n_points ? a.k[2 * (size_t)pp + 1] : mk(0.f, 0.f);
    }
    __syncthreads();
    const cpx<float> kx = kp[2 * p], ky = kp[2 * p + 1];
    for (int c = 0; c < a.n_chunks; ++c, ++stage) {
      const int buf = stage & 1;
      if (stage >= 2 && !tc::mbar_wait(&mbar[buf], ((stage - 2) >> 1) & 1, kTcPolls)) atomicOr(&s_fail, 1);
      __syncthreads();
      if (s_fail) break;
      // ---- A chunk: point p, basis functions 4 half .. 4 half + 3 of the chunk
      float* ahi = A + (size_t)buf * 2 * kTcRows * kTcK;
      float* alo = ahi + kTcRows * kTcK;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int iu = 4 * half + u;
        const int i = c * kTcBasis + iu;
        const float x = sbx[i], y = sby[i];
        const float theta = kx.re * x + ky.re * y;   // Re k.r
        const float psi = kx.im * x + ky.im * y;     // Im k.r
        float sn, cs;
        sincosf(theta, &sn, &cs);
        const bool live = i < a.n_basis;
        const float e = live ? expf(psi) : 0.f, ie = live ? expf(-psi) : 0.f;
        const float v0 = cs * e, v1 = -sn * e, v2 = cs * ie, v3 = sn * ie;   // E, E'
        float h0, h1, h2, h3, l0, l1, l2, l3;
        tf32_split(v0, h0, l0);
        tf32_split(v1, h1, l1);
        tf32_split(v2, h2, l2);
        tf32_split(v3, h3, l3);
        const uint32_t off = tc::kmajor_offset(p, 4 * iu, kTcK) / 4;
        *reinterpret_cast<float4*>(ahi + off) = make_float4(h0, h1, h2, h3);
        *reinterpret_cast<float4*>(alo + off) = make_float4(l0, l1, l2, l3);
      }
      // ---- B chunk (prepared on the host): hi and lo blocks, contiguous
      {
        const float4* src = reinterpret_cast<const float4*>(a.bmat + (size_t)c * 2 * a.ncol * kTcK);
        float4* dst = reinterpret_cast<float4*>(B + (size_t)buf * 2 * a.ncol * kTcK);
        for (int t = tid; t < a.ncol * kTcK / 2; t += kTcThreads) dst[t] = src[t];
      }
      tc::fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t a_hi = tc::smem_u32(ahi), a_lo = a_hi + a_bytes;
        const uint32_t b_hi = tc::smem_u32(B + (size_t)buf * 2 * a.ncol * kTcK), b_lo = b_hi + b_bytes;
#pragma unroll
        for (int s = 0; s < kTcK / 8; ++s) {
          const uint32_t ko = s * 256;   // two core matrices (8 tf32) along K per MMA
          const uint64_t dah = tc::sdesc(a_hi + ko, 128, sbo), dal = tc::sdesc(a_lo + ko, 128, sbo);
          const uint64_t dbh = tc::sdesc(b_hi + ko, 128, sbo), dbl = tc::sdesc(b_lo + ko, 128, sbo);
          // head x head products and the two corrections in separate accumulators
          const uint32_t acc = (c > 0 || s > 0) ? 1u : 0u;
          tc::mma_tf32(tmem + (uint32_t)a.ncol, dah, dbl, idesc, acc);
          tc::mma_tf32(tmem + (uint32_t)a.ncol, dal, dbh, idesc, 1u);
          tc::mma_tf32(tmem, dah, dbh, idesc, acc);
        }
        tc::mma_commit(&mbar[buf]);
      }
      issued = true;
    }
    if (s_fail) break;
    // ---- wait for the tile's last chunk (its commit covers every earlier MMA)
    const uint32_t last = stage - 1;
    if (!tc::mbar_wait(&mbar[last & 1], (last >> 1) & 1, kTcPolls)) atomicOr(&s_fail, 1);
    __syncthreads();
    if (s_fail) break;
    tc::fence_after_sync();
    if (warp < 4) {
      constexpr int GC = tc_group_cols(MB);
      const int pl = 32 * warp + lane;
      const int pg = p0 + pl;
      const cpx<float> qx = kp[2 * pl], qy = kp[2 * pl + 1];
      cpx<float> mx[2][MB], my[2][MB];   // [side][MBF] x and y components
#pragma unroll
      for (int sd = 0; sd < 2; ++sd)
#pragma unroll
        for (int m = 0; m < MB; ++m) {
          mx[sd][m] = mk(0.f, 0.f);
          my[sd][m] = mk(0.f, 0.f);
        }
      for (int sc = 0; sc < a.n_shape; ++sc) {
        const ShapeClass shp = a.shapes[sc];
        const cpx<float> sf = rooftop_factor(shp, qx, qy);
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
          const uint32_t col0 = (uint32_t)((sd * a.n_shape + sc) * GC);
#pragma unroll
          for (int cb = 0; cb < GC; cb += 8) {
            float v[8], w8[8];
            tc::tmem_ld8(tmem + ((uint32_t)(32 * warp) << 16) + col0 + cb, v);
            tc::tmem_ld8(tmem + ((uint32_t)(32 * warp) << 16) + col0 + (uint32_t)a.ncol + cb, w8);
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) v[jj] += w8[jj];
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
              const int m = (cb + j) / 2;
              if (m < MB) {
                const cpx<float> t = mk(v[j], v[j + 1]);
                if (shp.dir == 0) cmac(mx[sd][m], sf, t);
                else cmac(my[sd][m], sf, t);
              }
            }
          }
        }
      }
      if (pg < a.n_points) {
        cpx<float>* o = a.out + (size_t)pg * 2 * a.n_mbf * 2;
#pragma unroll
        for (int sd = 0; sd < 2; ++sd)
#pragma unroll
          for (int m = 0; m < MB; ++m)
            if (m < a.n_mbf) {
              o[(sd * a.n_mbf + m) * 2 + 0] = mx[sd][m];
              o[(sd * a.n_mbf + m) * 2 + 1] = my[sd][m];
            }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  // ---- teardown: nothing of ours in flight, then free the tensor memory
  if (s_fail && issued && tid == 0) {
    const uint32_t last = stage - 1;
    tc::mbar_wait(&mbar[last & 1], (last >> 1) & 1, kTcPolls);
  }
  if (s_fail && tid == 0) atomicOr(a.err, 16);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, (uint32_t)a.ncol_alloc);
}

}  // namespace

// GEMM width of an element (0 when the tensor-core form does not apply)
int spectra_tc_columns(int n_shape, int n_mbf) {
  if (n_mbf < 1 || n_mbf > 8) return 0;
  const int ncol = 2 * n_shape * tc_group_cols(tc_mbf_pad(n_mbf));
  return ncol <= 64 ? ncol : 0;
}

// B operand of the element: [chunk][hi, lo][ncol x 32] in the no-swizzle K-major layout.
// mirror: a second block of ncol columns gives the spectra at the opposite wave
// direction alpha + pi from the same A row, whose projections p_i change sign, so
// that E(alpha + pi) = E'(alpha) and E'(alpha + pi) = E(alpha): the side-t
// coefficients move to the E' rows and the side-b ones to the E rows.
void spectra_tc_bmatrix(int n_basis, int n_shape, const int* basis_class, int n_mbf,
                        const double* q_re_im, int q_stride, bool mirror, std::vector<float>* out) {
  const int ncol = spectra_tc_columns(n_shape, n_mbf) * (mirror ? 2 : 1);
  const int half = mirror ? ncol / 2 : 0;
  const int n_chunks = (n_basis + kTcBasis - 1) / kTcBasis;
  out->assign((size_t)n_chunks * 2 * ncol * kTcK, 0.f);
  // nearest TF32 value, ties away from zero (the rounding of cvt.rna.tf32.f32)
  auto rna = [](float v) {
    uint32_t bits;
    std::memcpy(&bits, &v, 4);
    bits = (bits + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &bits, 4);
    return r;
  };
  auto put = [&](int i, int col, int part, double val) {
    const int c = i / kTcBasis, u = i % kTcBasis;
    const float v = (float)val;
    const float hi = rna(v), lo = rna(v - hi);
    const size_t blk = (size_t)c * 2 * ncol * kTcK;
    const uint32_t off = tc::kmajor_offset(col, 4 * u + part, kTcK) / 4;
    (*out)[blk + off] = hi;
    (*out)[blk + (size_t)ncol * kTcK + off] = lo;
  };
  for (int i = 0; i < n_basis; ++i) {
    const int s = basis_class[i];
    for (int m = 0; m < n_mbf; ++m) {
      const double qr = q_re_im[2 * ((size_t)i * q_stride + m)], qi = q_re_im[2 * ((size_t)i * q_stride + m) + 1];
      const int gc = tc_group_cols(tc_mbf_pad(n_mbf));
      const int ct = (0 * n_shape + s) * gc + 2 * m;   // side t: sum conj(Q) E
      const int cb = (1 * n_shape + s) * gc + 2 * m;   // side b: sum Q E'
      // conj(Q) E = (qr er + qi ei) + i (qr ei - qi er)
      put(i, ct, 0, qr);
      put(i, ct, 1, qi);
      put(i, ct + 1, 0, -qi);
      put(i, ct + 1, 1, qr);
      // Q E' = (qr er' - qi ei') + i (qi er' + qr ei')
      put(i, cb, 2, qr);
      put(i, cb, 3, -qi);
      put(i, cb + 1, 2, qi);
      put(i, cb + 1, 3, qr);
      if (mirror) {
        // conj(Q) E(alpha + pi) = conj(Q) E'(alpha), Q E'(alpha + pi) = Q E(alpha)
        put(i, half + ct, 2, qr);
        put(i, half + ct, 3, qi);
        put(i, half + ct + 1, 2, -qi);
        put(i, half + ct + 1, 3, qr);
        put(i, half + cb, 0, qr);
        put(i, half + cb, 1, -qi);
        put(i, half + cb + 1, 0, qi);
        put(i, half + cb + 1, 1, qr);
      }
    }
  }
}

namespace {

// one thread waits, at most `polls` tries, on the phase of an mbarrier that nothing
// completes: the bounded wait of every tensor-core kernel, run out on purpose
__global__ void wait_selftest_kernel(unsigned polls, int* flag) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  tc::mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  *flag = tc::mbar_wait(&bar, 0, polls) ? 1 : 16;
}

}  // namespace

cudaError_t launch_wait_selftest(unsigned polls, int* flag, cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(polls, flag);
  return cudaGetLastError();
}

cudaError_t launch_spectra_tc(int n_points, int n_basis, int n_shape, int n_mbf, const ShapeClass* shapes,
                              const float* bx, const float* by, const float* bmat, const void* k, void* out,
                              int* err, cudaStream_t s) {
  const int ncol = spectra_tc_columns(n_shape, n_mbf);
  if (ncol == 0 || n_points < 1) return cudaErrorInvalidValue;
  SpectraTcArgs a{};
  a.n_points = n_points;
  a.n_basis = n_basis;
  a.n_shape = n_shape;
  a.n_mbf = n_mbf;
  a.ncol = ncol;
  a.ncol_alloc = 2 * ncol <= 64 ? 64 : 128;   // two accumulators (head x head, corrections)
  a.n_chunks = (n_basis + kTcBasis - 1) / kTcBasis;
  a.shapes = shapes;
  a.bx = bx;
  a.by = by;
  a.bmat = bmat;
  a.k = reinterpret_cast<const cpx<float>*>(k);
  a.out = reinterpret_cast<cpx<float>*>(out);
  a.err = err;
  const size_t smem = tc_smem_bytes(ncol, n_basis);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int n_tiles = (n_points + kTcRows - 1) / kTcRows;
  const int grid = n_tiles < sms ? n_tiles : sms;
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kTcThreads, smem, s>>>(a);
    return cudaGetLastError();
  };
  switch (tc_mbf_pad(n_mbf)) {
    case 1: return go(spectra_tc_kernel<1>);
    case 2: return go(spectra_tc_kernel<2>);
    case 4: return go(spectra_tc_kernel<4>);
    default: return go(spectra_tc_kernel<8>);
  }
}

}  // namespace cfft
