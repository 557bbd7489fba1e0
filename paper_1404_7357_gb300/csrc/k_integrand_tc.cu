// Fused contour integrand with the MBF spectra on the tensor cores (FP32-mixed,
// rooftop elements, N_alpha = 128 or 256): Eq. 11 as a GEMM (see k_spectra_tc.cu for
// the operand layout and the TF32 head/tail products), then the kernel of
// Eq. 10 and its azimuthal harmonics times the contour measure of Eq. 9,
// exactly as the SIMT form in k_integrand.cu computes them.
//
// A CTA owns 512 points: JT = 512 / N_alpha consecutive contour nodes x N_alpha
// angles.  The wave directions alpha and alpha + pi have opposite projections
// p_i = x_i cos alpha + y_i sin alpha of every basis centre, so one A row (the
// exponentials exp(-+i beta_c,j p_i) of direction alpha) serves both: the B
// operand carries a second block of columns with the two sides' coefficients
// exchanged (k_spectra_tc.cu), and the rows are the JT x N_alpha / 2 (node,
// alpha < pi) pairs, as 2 tiles of 128 (one tensor-memory accumulator pair
// each).  The basis dimension is the outer loop and the tiles the inner one, so
// a thread keeps, for each of its four basis functions, exp(-i beta_R,j p_i)
// and advances it from its node in one tile to its node in the next by one
// complex rotation (the nodes are equally spaced in beta_R); exp(+-beta_I,j p_i)
// is a short series (|beta_I p| is small on the contour) or expf otherwise.
// The A chunk of a (chunk, tile) stage is written while the tensor core
// consumes the previous stage.
//
// After the GEMM, each point's spectra (both sides, both directions, every
// MBF) go to shared memory component-major; H_ab(j, l) for a chunk of MBF pairs
// (32 or 16 (pair, node) rows) follows, folded F = N_alpha / 32 -fold in angle as it is formed
// (an F-point DFT per angle), and the angular DFT runs over the folded rows
// (32 terms per harmonic; rows padded by one entry, conflict-free, twiddles
// broadcast).
#include "cfft_common.cuh"
#include "dft_small.cuh"
#include "spectra_tc.cuh"
#include "tc_sm100.cuh"

namespace cfft {

namespace {

constexpr int kIThreads = 256;
constexpr int kTiles = 2;       // 128-row tiles (tensor-core M = 128) per CTA

template <int NA>
struct ItcShape {
  static constexpr int HA = NA / 2;        // directions alpha < pi (A rows per node)
  static constexpr int NPT = 128 / HA;     // contour nodes per tile
  static constexpr int JT = kTiles * NPT;  // contour nodes per CTA
  static constexpr int F = NA / 32;        // angular fold of the DFT
  static constexpr int ROWS = NA == 256 ? 16 : 32;   // H rows (pairs x nodes) per chunk
  static constexpr int PC = ROWS / JT;     // MBF pairs per H chunk
  static constexpr int ROW = NA + 1;       // padded H row
};

struct ItcLayout {
  size_t a, b, spec, hbuf, tw, bx, node, mbar, total;
};

template <int NA>
__host__ __device__ inline ItcLayout itc_layout(int ncol, int mb, int nb_pad) {
  using S = ItcShape<NA>;
  ItcLayout L{};
  // phase 1 (A, B operand buffers) and phases 2-3 (spectra, H rows) share one region
  const size_t p1 = (size_t)2 * 2 * 128 * kTcK * 4 + (size_t)2 * 2 * ncol * kTcK * 4;
  const size_t spec = (size_t)S::JT * 4 * mb * NA * 8;
  const size_t p23 = spec + (size_t)S::ROWS * S::ROW * 8;
  L.a = 0;
  L.b = (size_t)2 * 2 * 128 * kTcK * 4;
  L.spec = 0;
  L.hbuf = spec;
  size_t o = (p1 > p23 ? p1 : p23);
  o = (o + 15) & ~(size_t)15;
  L.tw = o;
  o += (size_t)NA * 8;
  L.bx = o;
  o += (size_t)2 * nb_pad * 4;
  o = (o + 15) & ~(size_t)15;
  L.node = o;                      // per node: beta_R, beta_I, bw (2), P (2), R beta^2 (2) as floats
  o += (size_t)S::JT * 8 * 4;
  o = (o + 7) & ~(size_t)7;
  L.mbar = o;
  o += 2 * 8 + 16;
  L.total = o + 1024;              // slack for the 1024-byte alignment of the base
  return L;
}

size_t itc_smem(int na, int ncol, int mb, int nb_pad) {
  return na == 256 ? itc_layout<256>(ncol, mb, nb_pad).total : itc_layout<128>(ncol, mb, nb_pad).total;
}

template <int MB, int NA>
__device__ __forceinline__ void integrand_tc_body(const IntegrandArgs<float>& a, const int j0,
                                                  unsigned char* smem_raw) {
  using S = ItcShape<NA>;
  constexpr int HA = S::HA, NPT = S::NPT, JT = S::JT, F = S::F, PC = S::PC, ROW = S::ROW;
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int ncol = a.tc_ncol;
  const int n_chunks = (a.n_basis + kTcBasis - 1) / kTcBasis;
  const int nb_pad = n_chunks * kTcBasis;
  const ItcLayout L = itc_layout<NA>(ncol, MB, nb_pad);
  float* A = reinterpret_cast<float*>(base + L.a);
  float* B = reinterpret_cast<float*>(base + L.b);
  cpx<float>* spec = reinterpret_cast<cpx<float>*>(base + L.spec);   // [t][comp][angle]
  cpx<float>* hbuf = reinterpret_cast<cpx<float>*>(base + L.hbuf);   // [pl][t][ROW]
  cpx<float>* tw = reinterpret_cast<cpx<float>*>(base + L.tw);       // exp(-2 pi i l / N_alpha)
  float* sbx = reinterpret_cast<float*>(base + L.bx);
  float* sby = sbx + nb_pad;
  float* nd = reinterpret_cast<float*>(base + L.node);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(base + L.mbar);
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(mbar + 2);
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int t = tid; t < NA; t += kIThreads) {
    float s, c;
    sincospif(-2.0f * (float)t / (float)NA, &s, &c);
    tw[t] = mk(c, s);
  }
  for (int i = tid; i < nb_pad; i += kIThreads) {
    sbx[i] = i < a.n_basis ? a.tc_bx[i] : 0.f;
    sby[i] = i < a.n_basis ? a.tc_by[i] : 0.f;
  }
  if (tid < JT) {
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
  // per tile: head x head products in one accumulator, the two correction products in a
  // second one (the tensor core truncates on every accumulation; splitting the sums
  // keeps the large accumulator's step count and the small one's magnitude low)
  const uint32_t ncol_alloc = 2 * kTiles * ncol <= 256 ? 256u : 512u;
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

  // ---------------- phase 1: MBF spectra of the 512 points on the tensor cores
  {
    // A row r of tile T: node T NPT + r / HA, direction alpha_(r mod HA) (and its mirror)
    const int r = tid & 127, half = tid >> 7;
    const int tn = r / HA, ang = r - tn * HA;
    const uint32_t idesc = tc::idesc_tf32(128, ncol);
    const uint32_t a_bytes = 128 * kTcK * 4, b_bytes = (uint32_t)ncol * kTcK * 4;
    const uint32_t sbo = (kTcK / 4) * 128;
    const int b_vec = ncol * kTcK / 2;           // float4 of one chunk's B operand (hi + lo)
    const float br_pi = nd[8 * tn] * 0.31830988618379067f;
    const float hs = (float)NPT * h, hs_pi = hs * 0.31830988618379067f;   // node step between tiles
    const bool small_step = hs * a.tc_rmax < 0.0625f;
    const float ca = tw[ang].re, sa = -tw[ang].im;   // cos, sin alpha
    // B operand of chunk 0 (later chunks are prefetched one chunk ahead)
    {
      const float4* src = reinterpret_cast<const float4*>(a.tc_bmat);
      float4* dst = reinterpret_cast<float4*>(B);
      for (int q = tid; q < b_vec; q += kIThreads) dst[q] = src[q];
    }
    uint32_t stage = 0;
    for (int c = 0; c < n_chunks; ++c) {
      // exp(-i beta_R p) at this thread's node of tile 0 for its four basis functions,
      // and the rotation to its node of the next tile
      float pc[4], cs[4], sn[4], cd[4], sd[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = c * kTcBasis + 4 * half + u;
        pc[u] = sbx[i] * ca + sby[i] * sa;
        sincospif(br_pi * pc[u], &sn[u], &cs[u]);
        if (small_step) {
          // |hs p| <= hs r_max < 1/16: short series (truncation below 1e-14)
          const float x = hs * pc[u], x2 = x * x;
          sd[u] = x * (1.f - x2 * (1.f / 6.f) * (1.f - x2 * (1.f / 20.f)));
          cd[u] = 1.f - x2 * 0.5f * (1.f - x2 * (1.f / 12.f) * (1.f - x2 * (1.f / 30.f)));
        } else {
          sincospif(hs_pi * pc[u], &sd[u], &cd[u]);
        }
      }
      bool fail = false;
#pragma unroll
      for (int tile = 0; tile < kTiles; ++tile) {
        const int t = tile * NPT + tn;
        const int buf = stage & 1;
        // the MMAs of stage - 2 have read A[buf] (and, at tile 1, the previous chunk's B):
        // one lane per warp polls the mbarrier, the others wait at the warp barrier
        if (stage >= 2) {
          if (lane == 0 && !tc::mbar_wait(&mbar[buf], ((stage - 2) >> 1) & 1, kTcPolls)) atomicOr(&s_fail, 1);
          __syncwarp();
        }
        if (tile == 1 && c + 1 < n_chunks) {
          const char* src = reinterpret_cast<const char*>(a.tc_bmat + (size_t)(c + 1) * 2 * ncol * kTcK);
          char* dst = reinterpret_cast<char*>(B + (size_t)((c + 1) & 1) * 2 * ncol * kTcK);
          for (int q = tid; q < b_vec; q += kIThreads)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst + 16 * q)),
                         "l"(src + 16 * q)
                         : "memory");
          asm volatile("cp.async.commit_group;" ::: "memory");
        }
        if (tile == 0 && c > 0) asm volatile("cp.async.wait_group 0;" ::: "memory");
        float* ahi = A + (size_t)buf * 2 * 128 * kTcK;
        float* alo = ahi + 128 * kTcK;
        const float bi = nd[8 * t + 1];
        // |beta_I p| <= beta_I r_max: the short series when that bound is small (uniform
        // per warp: a warp's rows share one node); basis functions past n_basis meet
        // zero rows of B
        const bool series = bi * a.tc_rmax < 0.125f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int iu = 4 * half + u;
          const float psi = bi * pc[u];
          float ep, em;
          if (series) {
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
          const float v0 = cs[u] * ep, v1 = -sn[u] * ep, v2 = cs[u] * em, v3 = sn[u] * em;
          float h0, h1, h2, h3, l0, l1, l2, l3;
          tf32_split(v0, h0, l0);
          tf32_split(v1, h1, l1);
          tf32_split(v2, h2, l2);
          tf32_split(v3, h3, l3);
          const uint32_t off = tc::kmajor_offset(r, 4 * iu, kTcK) / 4;
          *reinterpret_cast<float4*>(ahi + off) = make_float4(h0, h1, h2, h3);
          *reinterpret_cast<float4*>(alo + off) = make_float4(l0, l1, l2, l3);
          if (tile + 1 < kTiles) {
            // advance exp(-i beta_R p) to this thread's node of the next tile
            const float c2 = cs[u] * cd[u] - sn[u] * sd[u];
            const float s2 = sn[u] * cd[u] + cs[u] * sd[u];
            cs[u] = c2;
            sn[u] = s2;
          }
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (s_fail) { fail = true; break; }
        if (tid == 0) {
          tc::fence_after_sync();
          const uint32_t a_hi = tc::smem_u32(ahi), a_lo = a_hi + a_bytes;
          const uint32_t b_hi = tc::smem_u32(B + (size_t)(c & 1) * 2 * ncol * kTcK), b_lo = b_hi + b_bytes;
          const uint32_t d_big = tmem + (uint32_t)(2 * tile * ncol), d_small = d_big + (uint32_t)ncol;
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
        ++stage;
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
      const int hcol = ncol / 2;                       // columns of one direction block
      const int lq = warp & 3, tile = warp >> 2;       // kTiles = 2: one tile per warp
      const int r = 32 * lq + lane;                    // this thread's TMEM lane = A row
      const int tn = r / HA, ang = r - tn * HA;
      const int t = tile * NPT + tn;
      const float cl = tw[ang].re, sl = -tw[ang].im;
      const cpx<float> bc = mk(nd[8 * t], nd[8 * t + 1]);
      const cpx<float> kx = mk(bc.re * cl, bc.im * cl), ky = mk(bc.re * sl, bc.im * sl);
      // mir = 0: direction alpha; 1: alpha + pi (k -> -k; the rooftop factor is even)
#pragma unroll 1
      for (int mir = 0; mir < 2; ++mir) {
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
            const uint32_t col0 = (uint32_t)(2 * tile * ncol + mir * hcol + (sd2 * a.n_shape + sc) * GC);
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
        const int al = ang + mir * HA;
#pragma unroll
        for (int sd2 = 0; sd2 < 2; ++sd2)
#pragma unroll
          for (int m = 0; m < MB; ++m) {
            spec[((size_t)t * 4 * MB + (sd2 * MB + m) * 2 + 0) * NA + al] = mx[sd2][m];
            spec[((size_t)t * 4 * MB + (sd2 * MB + m) * 2 + 1) * NA + al] = my[sd2][m];
          }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }

  if (!s_fail) {
    // ---------------- phases 2-3: kernel of Eq. 10, harmonics, contour measure
    // With w = exp(-2 pi i / N_alpha), sum_l H(l) w^(q l) = sum_{l < 32} w^(q l) G_r(l) where
    // r = q mod F and G_r(l) = sum_k H(l + 32 k) W_F^(r k) (the angles folded F-fold, an
    // F-point DFT per l): every harmonic then costs 32 terms instead of N_alpha.
    const int mr = a.n_mbf;
    const int n_pairs = mr * mr;
    const int nh = 2 * a.q_max + 1;
    const int quarter = NA / 4;
    const float inv_na = 1.0f / (float)NA;
    for (int cls = 0; cls < a.n_cls; ++cls)
      for (int pair0 = 0; pair0 < n_pairs; pair0 += PC) {
        const int npc = min(PC, n_pairs - pair0);
        const bool rot_t = (cls == 2), rot_b = (cls == 1);
        for (int idx = tid; idx < npc * JT * 32; idx += kIThreads) {
          const int l0 = idx & 31;
          const int rest = idx >> 5;
          const int t = rest % JT, pl = rest / JT;
          const int pair = pair0 + pl;
          const int ia = pair / mr, ib = pair - ia * mr;
          const cpx<float>* st = spec + (size_t)t * 4 * MB * NA;
          const float* o = nd + 8 * t;
          const cpx<float> gp = mk(o[4], o[5]), gr = mk(o[6], o[7]);
          cpx<float> hk[F];
#pragma unroll
          for (int k = 0; k < F; ++k) {
            const int l = l0 + 32 * k;
            const int lt = rot_t ? (l - quarter + NA) & (NA - 1) : l;
            const int lb = rot_b ? (l - quarter + NA) & (NA - 1) : l;
            cpx<float> tx = st[((0 * MB + ia) * 2 + 0) * NA + lt], ty = st[((0 * MB + ia) * 2 + 1) * NA + lt];
            cpx<float> bx = st[((1 * MB + ib) * 2 + 0) * NA + lb], by = st[((1 * MB + ib) * 2 + 1) * NA + lb];
            if (rot_t) { const cpx<float> q = tx; tx = mk(-ty.re, -ty.im); ty = q; }   // R90 (x,y) = (-y, x)
            if (rot_b) { const cpx<float> q = bx; bx = mk(-by.re, -by.im); by = q; }
            const float ua = tw[l].re, ub = -tw[l].im;
            const cpx<float> dot = tx * bx + ty * by;
            const cpx<float> et = ua * tx + ub * ty;
            const cpx<float> eb = ua * bx + ub * by;
            hk[k] = gp * dot - gr * (et * eb);
          }
          // G_0..G_{F-1} at l0: the F-point DFT of (H(l0 + 32 k))_k
          if constexpr (F == 4) dft4(hk[0], hk[1], hk[2], hk[3]);
          else dft8(hk);
          cpx<float>* row = hbuf + (size_t)(pl * JT + t) * ROW;
#pragma unroll
          for (int k = 0; k < F; ++k) row[k * 32 + l0] = hk[k];
        }
        __syncthreads();
        // warp w: harmonics of class r = w mod F (every F-th q); lanes: the ROWS (pair,
        // node) rows, each row served by 32 / ROWS lanes that split the class's harmonics
        constexpr int ROWS = S::ROWS;
        const int rowi = lane % ROWS;
        const int pl = rowi / JT, t = rowi - pl * JT;
        const bool row_ok = pl < npc && j0 + t < a.n;
        const int r = warp % F;
        constexpr int WPC = (8 / F) * (32 / ROWS);   // shares per class
        const int share = (warp / F) * (32 / ROWS) + lane / ROWS;
        // harmonic indices qi = q + q_max with q = r (mod F), split between the warps of r
        const int q_first = -a.q_max + ((r + a.q_max) % F + F) % F;
        const int n_r = q_first > a.q_max ? 0 : (a.q_max - q_first) / F + 1;
        const int k_lo = (n_r * share) / WPC, k_hi = (n_r * (share + 1)) / WPC;
        if (row_ok) {
          const cpx<float>* g = hbuf + (size_t)rowi * ROW + r * 32;
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
              qv[u] = q_first + F * kk;
              mq[u] = ((qv[u] % NA) + NA) % NA;
              e[u] = 0;
              acc[u] = mk(0.f, 0.f);
            }
#pragma unroll 4
            for (int l = 0; l < 32; ++l) {
              const cpx<float> gv = g[l];
#pragma unroll
              for (int u = 0; u < 3; ++u) {
                cmac(acc[u], gv, tw[e[u]]);
                e[u] = (e[u] + mq[u]) & (NA - 1);
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

template <int MB, int NA>
__global__ void __launch_bounds__(kIThreads, 2) integrand_tc_kernel(IntegrandArgs<float> a) {
  extern __shared__ unsigned char smem_raw[];
  integrand_tc_body<MB, NA>(a, blockIdx.x * ItcShape<NA>::JT, smem_raw);
}

// batched form: block b processes the nodes from map[b].y of item map[b].x
template <int MB, int NA>
__global__ void __launch_bounds__(kIThreads, 2)
integrand_tc_batch_kernel(const IntegrandArgs<float>* items, const int2* map) {
  extern __shared__ unsigned char smem_raw[];
  const int2 bm = map[blockIdx.x];
  const IntegrandArgs<float> a = items[bm.x];
  integrand_tc_body<MB, NA>(a, bm.y, smem_raw);
}

template <template <int, int> class K, class Go>
cudaError_t dispatch_tc(int mb, int na, Go go) {
  if (na == 256) {
    switch (mb) {
      case 1: return go(K<1, 256>::fn());
      case 2: return go(K<2, 256>::fn());
      default: return go(K<4, 256>::fn());
    }
  }
  switch (mb) {
    case 1: return go(K<1, 128>::fn());
    case 2: return go(K<2, 128>::fn());
    default: return go(K<4, 128>::fn());
  }
}

template <int MB, int NA>
struct SingleK {
  static auto fn() { return integrand_tc_kernel<MB, NA>; }
};
template <int MB, int NA>
struct BatchK {
  static auto fn() { return integrand_tc_batch_kernel<MB, NA>; }
};

}  // namespace

bool integrand_tc_applies(const IntegrandArgs<float>& a) {
  if ((a.n_alpha != 128 && a.n_alpha != 256) || a.tc_bmat == nullptr || a.tc_ncol <= 0 || a.n_mbf > 4)
    return false;
  if (2 * kTiles * a.tc_ncol > 512) return false;
  const int nb_pad = (a.n_basis + kTcBasis - 1) / kTcBasis * kTcBasis;
  return itc_smem(a.n_alpha, a.tc_ncol, tc_mbf_pad(a.n_mbf), nb_pad) <= 220 * 1024;
}

// contour nodes per CTA of the tensor-core integrand for n_alpha angles
int integrand_tc_nodes(int n_alpha) { return n_alpha == 256 ? ItcShape<256>::JT : ItcShape<128>::JT; }

cudaError_t launch_integrand_tc(const IntegrandArgs<float>& a, cudaStream_t s) {
  if (!integrand_tc_applies(a)) return cudaErrorInvalidValue;
  const int mb = tc_mbf_pad(a.n_mbf);
  const int nb_pad = (a.n_basis + kTcBasis - 1) / kTcBasis * kTcBasis;
  const size_t smem = itc_smem(a.n_alpha, a.tc_ncol, mb, nb_pad);
  const int jt = integrand_tc_nodes(a.n_alpha);
  const int grid = (a.n + jt - 1) / jt;
  return dispatch_tc<SingleK>(mb, a.n_alpha, [&](auto kern) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kIThreads, smem, s>>>(a);
    return cudaGetLastError();
  });
}

cudaError_t launch_integrand_tc_batch(const IntegrandArgs<float>& shape_args, const IntegrandArgs<float>* items,
                                      const int2* map, int n_blocks, cudaStream_t s) {
  if (!integrand_tc_applies(shape_args)) return cudaErrorInvalidValue;
  const int mb = tc_mbf_pad(shape_args.n_mbf);
  const int nb_pad = (shape_args.n_basis + kTcBasis - 1) / kTcBasis * kTcBasis;
  const size_t smem = itc_smem(shape_args.n_alpha, shape_args.tc_ncol, mb, nb_pad);
  return dispatch_tc<BatchK>(mb, shape_args.n_alpha, [&](auto kern) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<n_blocks, kIThreads, smem, s>>>(items, map);
    return cudaGetLastError();
  });
}

}  // namespace cfft
