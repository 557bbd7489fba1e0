// Fused contour integrand with the MBF spectra on the tensor cores (FP32-mixed,
// rooftop elements, N_alpha = 128): Eq. 11 as a GEMM (see k_spectra_tc.cu for
// the operand layout and the TF32 head/tail products), then the kernel of
// Eq. 10 and its azimuthal harmonics times the contour measure of Eq. 9,
// exactly as the SIMT form in k_integrand.cu computes them.
//
// A CTA owns JT = 4 consecutive contour nodes x 128 angles (4 tiles of 128
// points, one tensor-memory accumulator each).  The basis dimension is the
// outer loop and the nodes the inner one, so a thread keeps, for each of its
// four basis functions, exp(-i beta_R,j p_i) (p_i = x_i cos alpha + y_i sin
// alpha, the projection of the centre on the wave direction) and advances it
// from node j to j + 1 by one complex rotation exp(-i h p_i) (the nodes are
// equally spaced in beta_R); exp(+-beta_I,j p_i) is a short series (|beta_I p|
// is small on the contour) or expf otherwise.  The A chunk of a (chunk, node)
// stage is written while the tensor core consumes the previous stage.
//
// After the GEMM, each point's spectra (both sides, both directions, every
// MBF) go to shared memory component-major; H_ab(j, l) for a chunk of 8 MBF
// pairs follows, folded 4-fold in angle as it is formed, and the angular DFT
// runs over the folded rows (32 terms per harmonic; rows padded to 129
// entries, conflict-free, twiddles broadcast).
#include "cfft_common.cuh"
#include "spectra_tc.cuh"
#include "tc_sm100.cuh"

namespace cfft {

namespace {

constexpr int kIThreads = 256;
constexpr int kJT = 4;          // contour nodes per CTA
constexpr int kNA = 128;        // angles (= MMA M)
constexpr int kPC = 8;          // MBF pairs per H chunk
constexpr int kRow = kNA + 1;   // padded H row

struct ItcLayout {
  size_t a, b, spec, hbuf, tw, bx, node, mbar, total;
};

__host__ __device__ inline ItcLayout itc_layout(int ncol, int mb, int nb_pad) {
  ItcLayout L{};
  // phase 1 (A, B operand buffers) and phases 2-3 (spectra, H rows) share one region
  const size_t p1 = (size_t)2 * 2 * kNA * kTcK * 4 + (size_t)2 * 2 * ncol * kTcK * 4;
  const size_t spec = (size_t)kJT * 4 * mb * kNA * 8;
  const size_t p23 = spec + (size_t)kPC * kJT * kRow * 8;
  L.a = 0;
  L.b = (size_t)2 * 2 * kNA * kTcK * 4;
  L.spec = 0;
  L.hbuf = spec;
  size_t o = (p1 > p23 ? p1 : p23);
  o = (o + 15) & ~(size_t)15;
  L.tw = o;
  o += (size_t)kNA * 8;
  L.bx = o;
  o += (size_t)2 * nb_pad * 4;
  o = (o + 15) & ~(size_t)15;
  L.node = o;                      // per node: beta_R, beta_I, bw (2), P (2), R beta^2 (2) as floats
  o += (size_t)kJT * 8 * 4;
  o = (o + 7) & ~(size_t)7;
  L.mbar = o;
  o += 2 * 8 + 16;
  L.total = o + 1024;              // slack for the 1024-byte alignment of the base
  return L;
}

template <int MB>
__global__ void __launch_bounds__(kIThreads, 2) integrand_tc_kernel(IntegrandArgs<float> a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int ncol = a.tc_ncol;
  const int n_chunks = (a.n_basis + kTcBasis - 1) / kTcBasis;
  const int nb_pad = n_chunks * kTcBasis;
  const ItcLayout L = itc_layout(ncol, MB, nb_pad);
  float* A = reinterpret_cast<float*>(base + L.a);
  float* B = reinterpret_cast<float*>(base + L.b);
  cpx<float>* spec = reinterpret_cast<cpx<float>*>(base + L.spec);   // [t][comp][l]
  cpx<float>* hbuf = reinterpret_cast<cpx<float>*>(base + L.hbuf);   // [pl][t][kRow]
  cpx<float>* tw = reinterpret_cast<cpx<float>*>(base + L.tw);       // exp(-2 pi i l / N)
  float* sbx = reinterpret_cast<float*>(base + L.bx);
  float* sby = sbx + nb_pad;
  float* nd = reinterpret_cast<float*>(base + L.node);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(base + L.mbar);
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(mbar + 2);
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = blockIdx.x * kJT;
  for (int t = tid; t < kNA; t += kIThreads) {
    float s, c;
    sincospif(-2.0f * (float)t / (float)kNA, &s, &c);
    tw[t] = mk(c, s);
  }
  for (int i = tid; i < nb_pad; i += kIThreads) {
    sbx[i] = i < a.n_basis ? a.tc_bx[i] : 0.f;
    sby[i] = i < a.n_basis ? a.tc_by[i] : 0.f;
  }
  if (tid < kJT) {
    const int j = j0 + tid;
    float* o = nd + 8 * tid;
    if (j < a.n) {
      const double2 b = a.beta_c[j], w = a.bw[j], gp = a.green_p[j], gr = a.green_r[j];
      o[0] = (float)b.x; o[1] = (float)b.y;
      o[2] = (float)w.x; o[3] = (float)w.y;
      o[4] = (float)gp.x; o[5] = (float)gp.y;
      o[6] = (float)gr.x; o[7] = (float)gr.y;
    } else {
      for (int k = 0; k < 8; ++k) o[k] = 0.f;
    }
  }
  if (tid == 0) {
    s_fail = 0;
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // per node: head x head products in one accumulator, the two correction products in a
  // second one (the tensor core truncates on every accumulation; splitting the sums
  // keeps the large accumulator's step count and the small one's magnitude low)
  const uint32_t ncol_alloc = 2 * kJT * ncol <= 256 ? 256u : 512u;
  if (warp == 0) {
    tc::tmem_alloc(taddr_s, ncol_alloc);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *taddr_s;
  // node spacing in beta_R (the nodes are the midpoints of equal cells)
  const float h = (float)(a.n > 1 ? a.beta_c[1].x - a.beta_c[0].x : 2.0 * a.beta_c[0].x);
  uint32_t stages_issued = 0;

  // ---------------- phase 1: MBF spectra of the 4 x 128 points on the tensor cores
  {
    const int l = tid & (kNA - 1), half = tid >> 7;
    const float ca = tw[l].re, sa = -tw[l].im;   // cos, sin alpha_l
    const uint32_t idesc = tc::idesc_tf32(kNA, ncol);
    const uint32_t a_bytes = kNA * kTcK * 4, b_bytes = (uint32_t)ncol * kTcK * 4;
    const uint32_t sbo = (kTcK / 4) * 128;
    const int b_vec = ncol * kTcK / 2;           // float4 of one chunk's B operand (hi + lo)
    const float br_pi = nd[0] * 0.31830988618379067f, h_pi = h * 0.31830988618379067f;
    // B operand of chunk 0 (later chunks are prefetched one chunk ahead)
    {
      const float4* src = reinterpret_cast<const float4*>(a.tc_bmat);
      float4* dst = reinterpret_cast<float4*>(B);
      for (int q = tid; q < b_vec; q += kIThreads) dst[q] = src[q];
    }
    uint32_t stage = 0;
    for (int c = 0; c < n_chunks; ++c) {
      // exp(-i beta_R p) of this thread's four basis functions at node j0, and its step
      float pc[4], cs[4], sn[4], cd[4], sd[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = c * kTcBasis + 4 * half + u;
        pc[u] = sbx[i] * ca + sby[i] * sa;
        sincospif(br_pi * pc[u], &sn[u], &cs[u]);
        sincospif(h_pi * pc[u], &sd[u], &cd[u]);
      }
      bool fail = false;
      for (int t = 0; t < kJT; ++t, ++stage) {
        const int buf = stage & 1;
        // the MMAs of stage - 2 have read A[buf] (and, at t = 1, the previous chunk's B)
        if (stage >= 2 && !tc::mbar_wait(&mbar[buf], ((stage - 2) >> 1) & 1, kTcPolls)) atomicOr(&s_fail, 1);
        if (t == 1 && c + 1 < n_chunks) {
          const char* src = reinterpret_cast<const char*>(a.tc_bmat + (size_t)(c + 1) * 2 * ncol * kTcK);
          char* dst = reinterpret_cast<char*>(B + (size_t)((c + 1) & 1) * 2 * ncol * kTcK);
          for (int q = tid; q < b_vec; q += kIThreads)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst + 16 * q)),
                         "l"(src + 16 * q)
                         : "memory");
          asm volatile("cp.async.commit_group;" ::: "memory");
        }
        if (t == 0 && c > 0) asm volatile("cp.async.wait_group 0;" ::: "memory");
        float* ahi = A + (size_t)buf * 2 * kNA * kTcK;
        float* alo = ahi + kNA * kTcK;
        const float bi = nd[8 * t + 1];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int iu = 4 * half + u;
          const bool live = c * kTcBasis + iu < a.n_basis;
          const float psi = bi * pc[u];
          float ep, em;
          if (fabsf(psi) < 0.125f) {
            // exp(+-psi) from its even and odd series parts (error < psi^6 / 720)
            const float p2 = psi * psi;
            const float ev = 1.f + p2 * (0.5f + p2 * (1.f / 24.f));
            const float od = psi * (1.f + p2 * (1.f / 6.f + p2 * (1.f / 120.f)));
            ep = ev + od;
            em = ev - od;
          } else {
            ep = expf(psi);
            em = expf(-psi);
          }
          if (!live) { ep = 0.f; em = 0.f; }
          const float v0 = cs[u] * ep, v1 = -sn[u] * ep, v2 = cs[u] * em, v3 = sn[u] * em;
          float h0, h1, h2, h3, l0, l1, l2, l3;
          tf32_split(v0, h0, l0);
          tf32_split(v1, h1, l1);
          tf32_split(v2, h2, l2);
          tf32_split(v3, h3, l3);
          const uint32_t off = tc::kmajor_offset(l, 4 * iu, kTcK) / 4;
          *reinterpret_cast<float4*>(ahi + off) = make_float4(h0, h1, h2, h3);
          *reinterpret_cast<float4*>(alo + off) = make_float4(l0, l1, l2, l3);
          // advance exp(-i beta_R p) to the next node
          const float c2 = cs[u] * cd[u] - sn[u] * sd[u];
          const float s2 = sn[u] * cd[u] + cs[u] * sd[u];
          cs[u] = c2;
          sn[u] = s2;
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (s_fail) { fail = true; break; }
        if (tid == 0) {
          tc::fence_after_sync();
          const uint32_t a_hi = tc::smem_u32(ahi), a_lo = a_hi + a_bytes;
          const uint32_t b_hi = tc::smem_u32(B + (size_t)(c & 1) * 2 * ncol * kTcK), b_lo = b_hi + b_bytes;
          const uint32_t d_big = tmem + (uint32_t)(2 * t * ncol), d_small = d_big + (uint32_t)ncol;
#pragma unroll
          for (int s = 0; s < kTcK / 8; ++s) {
            const uint32_t ko = s * 256;
            const uint64_t dah = tc::sdesc(a_hi + ko, 128, sbo), dal = tc::sdesc(a_lo + ko, 128, sbo);
            const uint64_t dbh = tc::sdesc(b_hi + ko, 128, sbo), dbl = tc::sdesc(b_lo + ko, 128, sbo);
            const uint32_t acc = (c > 0 || s > 0) ? 1u : 0u;
            tc::mma_tf32(d_small, dah, dbl, idesc, acc);
            tc::mma_tf32(d_small, dal, dbh, idesc, 1u);
            tc::mma_tf32(d_big, dah, dbh, idesc, acc);
          }
          tc::mma_commit(&mbar[buf]);
        }
      }
      if (fail) break;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    stages_issued = stage;
    // the last stage's commit covers every MMA of the CTA
    if (!s_fail && stage > 0) {
      const uint32_t last = stage - 1;
      if (!tc::mbar_wait(&mbar[last & 1], (last >> 1) & 1, kTcPolls)) atomicOr(&s_fail, 1);
    }
    __syncthreads();
    tc::fence_after_sync();
    // ---- epilogue: shape factors, per-direction sums, spectra to shared memory.
    // The A/B region is free now and becomes the spectra buffer.
    if (!s_fail) {
      constexpr int GC = tc_group_cols(MB);
      const int lq = warp & 3;
      const int lp = 32 * lq + lane;                 // angle of this thread's TMEM lane
      const float cl = tw[lp].re, sl = -tw[lp].im;
      for (int t = warp >> 2; t < kJT; t += 2) {
        const cpx<float> bc = mk(nd[8 * t], nd[8 * t + 1]);
        const cpx<float> kx = mk(bc.re * cl, bc.im * cl), ky = mk(bc.re * sl, bc.im * sl);
        cpx<float> mx[2][MB], my[2][MB];
#pragma unroll
        for (int sd2 = 0; sd2 < 2; ++sd2)
#pragma unroll
          for (int m = 0; m < MB; ++m) {
            mx[sd2][m] = mk(0.f, 0.f);
            my[sd2][m] = mk(0.f, 0.f);
          }
        for (int sc = 0; sc < a.n_shape; ++sc) {
          const ShapeClass shp = a.shapes[sc];
          const cpx<float> sf = rooftop_factor(shp, kx, ky);
#pragma unroll
          for (int sd2 = 0; sd2 < 2; ++sd2) {
            const uint32_t col0 = (uint32_t)(2 * t * ncol + (sd2 * a.n_shape + sc) * GC);
#pragma unroll
            for (int cb = 0; cb < GC; cb += 8) {
              float v[8], w8[8];
              tc::tmem_ld8(tmem + ((uint32_t)(32 * lq) << 16) + col0 + cb, v);
              tc::tmem_ld8(tmem + ((uint32_t)(32 * lq) << 16) + col0 + ncol + cb, w8);
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) v[jj] += w8[jj];
#pragma unroll
              for (int jj = 0; jj < 8; jj += 2) {
                const int m = (cb + jj) / 2;
                if (m < MB) {
                  const cpx<float> tv = mk(v[jj], v[jj + 1]);
                  if (shp.dir == 0) cmac(mx[sd2][m], sf, tv);
                  else cmac(my[sd2][m], sf, tv);
                }
              }
            }
          }
        }
        // component-major: comp = (side * MB + m) * 2 + d
#pragma unroll
        for (int sd2 = 0; sd2 < 2; ++sd2)
#pragma unroll
          for (int m = 0; m < MB; ++m) {
            spec[((size_t)t * 4 * MB + (sd2 * MB + m) * 2 + 0) * kNA + lp] = mx[sd2][m];
            spec[((size_t)t * 4 * MB + (sd2 * MB + m) * 2 + 1) * kNA + lp] = my[sd2][m];
          }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }

  if (!s_fail) {
    // ---------------- phases 2-3: kernel of Eq. 10, harmonics, contour measure
    // With w = exp(-2 pi i / 128), sum_l H(l) w^(q l) = sum_{l < 32} w^(q l) G_r(l) where
    // r = q mod 4 and G_r(l) = sum_k H(l + 32 k) (-i)^(r k) (the angles folded 4-fold,
    // a 4-point DFT per l): every harmonic then costs 32 terms instead of 128.
    const int mr = a.n_mbf;
    const int n_pairs = mr * mr;
    const int nh = 2 * a.q_max + 1;
    const int quarter = kNA / 4;
    const float inv_na = 1.0f / (float)kNA;
    for (int cls = 0; cls < a.n_cls; ++cls)
      for (int pair0 = 0; pair0 < n_pairs; pair0 += kPC) {
        const int npc = min(kPC, n_pairs - pair0);
        const bool rot_t = (cls == 2), rot_b = (cls == 1);
        for (int idx = tid; idx < npc * kJT * 32; idx += kIThreads) {
          const int l0 = idx & 31;
          const int rest = idx >> 5;
          const int t = rest % kJT, pl = rest / kJT;
          const int pair = pair0 + pl;
          const int ia = pair / mr, ib = pair - ia * mr;
          const cpx<float>* st = spec + (size_t)t * 4 * MB * kNA;
          const float* o = nd + 8 * t;
          const cpx<float> gp = mk(o[4], o[5]), gr = mk(o[6], o[7]);
          cpx<float> hk[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int l = l0 + 32 * k;
            const int lt = rot_t ? (l - quarter + kNA) & (kNA - 1) : l;
            const int lb = rot_b ? (l - quarter + kNA) & (kNA - 1) : l;
            cpx<float> tx = st[((0 * MB + ia) * 2 + 0) * kNA + lt], ty = st[((0 * MB + ia) * 2 + 1) * kNA + lt];
            cpx<float> bx = st[((1 * MB + ib) * 2 + 0) * kNA + lb], by = st[((1 * MB + ib) * 2 + 1) * kNA + lb];
            if (rot_t) { const cpx<float> q = tx; tx = mk(-ty.re, -ty.im); ty = q; }   // R90 (x,y) = (-y, x)
            if (rot_b) { const cpx<float> q = bx; bx = mk(-by.re, -by.im); by = q; }
            const float ua = tw[l].re, ub = -tw[l].im;
            const cpx<float> dot = tx * bx + ty * by;
            const cpx<float> et = ua * tx + ub * ty;
            const cpx<float> eb = ua * bx + ub * by;
            hk[k] = gp * dot - gr * (et * eb);
          }
          // G_0..G_3 at l0: the 4-point DFT of (H(l0), H(l0+32), H(l0+64), H(l0+96))
          const cpx<float> s02 = hk[0] + hk[2], d02 = hk[0] - hk[2];
          const cpx<float> s13 = hk[1] + hk[3], d13 = hk[1] - hk[3];
          const cpx<float> mid = mk(d13.im, -d13.re);        // -i (h1 - h3)
          cpx<float>* row = hbuf + (size_t)(pl * kJT + t) * kRow;
          row[0 * 32 + l0] = s02 + s13;
          row[1 * 32 + l0] = d02 + mid;
          row[2 * 32 + l0] = s02 - s13;
          row[3 * 32 + l0] = d02 - mid;
        }
        __syncthreads();
        // warp w: harmonics of class r = w mod 4 (every fourth q), half w / 4 of them;
        // lanes: the 32 (pair, node) rows
        const int rowi = lane;
        const int pl = rowi / kJT, t = rowi - pl * kJT;
        const bool row_ok = pl < npc && j0 + t < a.n;
        const int r = warp & 3;
        // harmonic indices qi = q + q_max with q = r (mod 4), split between the two warps of r
        const int q_first = -a.q_max + ((r - (-a.q_max)) % 4 + 4) % 4;
        const int n_r = q_first > a.q_max ? 0 : (a.q_max - q_first) / 4 + 1;
        const int k_lo = (warp >> 2) ? (n_r + 1) / 2 : 0, k_hi = (warp >> 2) ? n_r : (n_r + 1) / 2;
        if (row_ok) {
          const cpx<float>* g = hbuf + (size_t)rowi * kRow + r * 32;
          const float* o = nd + 8 * t;
          const cpx<float> w = mk(o[2], o[3]);
          const int j = j0 + t;
          for (int kq = k_lo; kq < k_hi; kq += 3) {
            // up to three harmonics of this class at once, sharing each G load
            int qv[3], e[3], mq[3];
            cpx<float> acc[3];
#pragma unroll
            for (int u = 0; u < 3; ++u) {
              const int kk = min(kq + u, k_hi - 1);
              qv[u] = q_first + 4 * kk;
              mq[u] = ((qv[u] % kNA) + kNA) % kNA;
              e[u] = 0;
              acc[u] = mk(0.f, 0.f);
            }
#pragma unroll 4
            for (int l = 0; l < 32; ++l) {
              const cpx<float> gv = g[l];
#pragma unroll
              for (int u = 0; u < 3; ++u) {
                cmac(acc[u], gv, tw[e[u]]);
                e[u] = (e[u] + mq[u]) & (kNA - 1);
              }
            }
#pragma unroll
            for (int u = 0; u < 3; ++u) {
              if (kq + u < k_hi) {
                const size_t series = ((size_t)cls * n_pairs + pair0 + pl) * nh + (qv[u] + a.q_max);
                a.y[series * a.n + j] = w * (inv_na * acc[u]);
              }
            }
          }
        }
        __syncthreads();
      }
  }
  // ---- teardown: after a timed-out wait, give the tensor core a bounded time to finish
  if (s_fail && tid == 0) {
    atomicOr(a.err, 16);
    if (stages_issued > 0) {
      const uint32_t last = stages_issued - 1;
      tc::mbar_wait(&mbar[last & 1], (last >> 1) & 1, kTcPolls);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, ncol_alloc);
}

}  // namespace

bool integrand_tc_applies(const IntegrandArgs<float>& a) {
  if (a.n_alpha != kNA || a.tc_bmat == nullptr || a.tc_ncol <= 0 || a.n_mbf > 4) return false;
  if (2 * kJT * a.tc_ncol > 512) return false;
  const int nb_pad = (a.n_basis + kTcBasis - 1) / kTcBasis * kTcBasis;
  return itc_layout(a.tc_ncol, tc_mbf_pad(a.n_mbf), nb_pad).total <= 220 * 1024;
}

cudaError_t launch_integrand_tc(const IntegrandArgs<float>& a, cudaStream_t s) {
  if (!integrand_tc_applies(a)) return cudaErrorInvalidValue;
  const int mb = tc_mbf_pad(a.n_mbf);
  const int nb_pad = (a.n_basis + kTcBasis - 1) / kTcBasis * kTcBasis;
  const size_t smem = itc_layout(a.tc_ncol, mb, nb_pad).total;
  const int grid = (a.n + kJT - 1) / kJT;
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kIThreads, smem, s>>>(a);
    return cudaGetLastError();
  };
  switch (mb) {
    case 1: return go(integrand_tc_kernel<1>);
    case 2: return go(integrand_tc_kernel<2>);
    default: return go(integrand_tc_kernel<4>);
  }
}

}  // namespace cfft
