// Reduced MBF system on the GPU (Section II): the reduced excitation V' = Q^H V
// (Eq. 4), the direct solution of Z' I' = V' by a blocked LU factorization with
// partial pivoting, and the port currents (Q I'_m)[port].  The paper solves the
// reduced system directly because the MBF reduction makes it small (Table II,
// "Solving time"); this is that step, dense, on one GPU.
//
// LU (right-looking, row-major, panels of kNb columns):
//   panel    one launch over the panel's rows: per column, every CTA proposes its
//            largest |re| + |im| among the rows not yet chosen (compared on the
//            leading 32 bits of the double, ties: lowest row), a barrier, every
//            CTA takes the same pivot, reads the pivot row and
//            eliminates the column from its own rows.  Pivoting is logical: rows
//            stay where they are and the chosen rows are recorded; one barrier per
//            column.  A panel of at most 2048 rows (that fits the shared memory
//            of one thread-block cluster, 16 CTAs, else 8) runs on the cluster:
//            the CTAs exchange candidates and the pivot row through distributed
//            shared memory with the cluster's hardware barrier.  Longer panels
//            run cooperatively over the grid: each CTA publishes its candidate's
//            key with a column tag in global memory, and polling the keys (with
//            a bound) is the grid barrier.
//   moves    the panel's pivot rows go to rows k..k+kb-1 and the rows they
//            displace to the vacated places, as a list of (source, destination)
//            row moves applied to every column of the matrix.
//   trsm     U12 = L11^-1 A12 (unit lower L11), one thread per column.
//   gemm     A22 -= L21 U12, K = the panel: in complex64 on the tensor cores (the
//            complex product as a real GEMM, three TF32 products), otherwise
//            64 x 64 tiles of complex entries on the FP32 / FP64 pipe.
// The solve applies every panel's moves to the right-hand side, then blocked
// forward (unit L) and backward (U) substitution: per panel one launch whose
// CTAs each solve the small diagonal block (one warp) and update their rows.
//
// Every poll of the grid panel is bounded: a poll that runs out sets an error bit,
// and every CTA leaves the panel (the host then returns CFFT_ERR_TIMEOUT).  The
// cluster barrier is the hardware's own: every CTA of the cluster is resident by
// construction, and every CTA takes every barrier (the pivot, and so any early
// stop, is the same decision in all of them).
#include <algorithm>

#include "cfft_common.cuh"
#include "spectra_tc.cuh"
#include "tc_sm100.cuh"

namespace cfft {

namespace {

constexpr int kNb = 64;                 // panel width
constexpr int kPanelThreads = 256;
constexpr unsigned kBarrierPolls = 1u << 22;

template <class T>
__device__ __forceinline__ cpx<T> ldcg(const cpx<T>* p);
template <>
__device__ __forceinline__ cpx<float> ldcg(const cpx<float>* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return mk(v.x, v.y);
}
template <>
__device__ __forceinline__ cpx<double> ldcg(const cpx<double>* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return mk(v.x, v.y);
}

template <class T>
__device__ __forceinline__ cpx<T> crecip(cpx<T> z) {
  return cdiv(mk((T)1, (T)0), z);
}

template <class T>
struct PanelArgs {
  cpx<T>* a;
  int64_t ld;
  int n, k, kb;
  unsigned long long* slot;  // [2][grid] per-CTA pivot key | column tag, by column parity
  cpx<T>* cand_data;  // [2][grid][kNb] the candidate rows' remaining panel entries
  int2* moves;        // (source row, destination row), at most 2 kb
  int* n_moves;
  int* err;           // bit 1: a barrier wait ran out; bit 2: zero pivot
};

// pivot key of row `row` with |re| + |im| = metric: the leading 32 bits of the metric (a
// non-negative double, so its bits order like its value: exponent and 20 mantissa bits),
// then the lower row (rows below 65535); the low 16 bits stay free for a column tag.  The
// largest key is the pivot, so the choice does not depend on how the rows are split
// between CTAs; 0 stands for no candidate.
__device__ __forceinline__ unsigned long long pivot_key(double metric, int row) {
  return (((unsigned long long)__double_as_longlong(metric) >> 32) << 32) |
         ((unsigned long long)(0xFFFFu - (unsigned)row) << 16);
}
__device__ __forceinline__ int key_row(unsigned long long key) { return 0xFFFF - (int)((key >> 16) & 0xFFFFu); }
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}

// the largest key of this CTA's rows not chosen yet in column j (every thread gets it)
template <class T, int kWarps>
__device__ __forceinline__ unsigned long long cta_best_key(const cpx<T>* rows, const unsigned char* chosen,
                                                           int nr, int kb, int j, int lo,
                                                           unsigned long long* wk) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned long long best = 0;
  for (int i = tid; i < nr; i += blockDim.x) {
    if (chosen[i]) continue;
    const cpx<T> v = rows[i * kb + j];
    best = umax64(best, pivot_key(fabs((double)v.re) + fabs((double)v.im), lo + i));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) best = umax64(best, __shfl_xor_sync(0xffffffffu, best, off));
  if (lane == 0) wk[warp] = best;
  __syncthreads();
  unsigned long long b = wk[0];
#pragma unroll
  for (int w = 1; w < kWarps; ++w) b = umax64(b, wk[w]);
  __syncthreads();   // wk is rewritten at the next column
  return b;
}

// the panel's row moves from its pivots (one thread): rows k+j <- pivot j; the rows of
// [k, k+kb) that were not chosen go to the places the chosen rows outside that range
// leave free, both in increasing order
template <class T>
__device__ void panel_record_moves(const PanelArgs<T>& p, const int* s_piv) {
  const int kb = p.kb;
  int nm = 0, nd = 0, nv = 0;
  int displaced[kNb], vacated[kNb];
  for (int j = 0; j < kb; ++j) {
    if (s_piv[j] != p.k + j) p.moves[nm++] = make_int2(s_piv[j], p.k + j);
    if (s_piv[j] >= p.k + kb) vacated[nv++] = s_piv[j];
  }
  for (int r = p.k; r < p.k + kb; ++r) {
    bool taken = false;
    for (int j = 0; j < kb; ++j) taken = taken || s_piv[j] == r;
    if (!taken) displaced[nd++] = r;
  }
  // nd == nv: both count the pivots from outside [k, k+kb)
  for (int t = 0; t < nd && t < nv; ++t) {
    int m = t;
    for (int u = t + 1; u < nv; ++u)
      if (vacated[u] < vacated[m]) m = u;
    const int tmp = vacated[t];
    vacated[t] = vacated[m];
    vacated[m] = tmp;
    p.moves[nm++] = make_int2(displaced[t], vacated[t]);
  }
  *p.n_moves = nm;
}

// One panel of kb columns on rows k..n-1, cooperative over the grid.  Each CTA holds its
// slice of rows in shared memory for the whole panel.  Per column it stages its best
// candidate's remaining entries in global memory, then publishes its pivot key tagged with
// the column (one 64-bit store after a fence); warp 0 of every CTA polls the G keys of the
// column until all carry the tag (the poll is the grid barrier, and it delivers the
// candidates), every CTA takes the largest key as the pivot and reads that row's entries.
// Keys and entries are double-buffered by column parity: a CTA publishes column j + 2 only
// after it has seen every key of column j + 1, which each CTA publishes after its reads of
// column j.  Every poll is bounded; a CTA whose poll runs out leaves the panel, and the
// others then run out on its missing keys.
template <class T>
__global__ void __launch_bounds__(kPanelThreads) lu_panel_kernel(PanelArgs<T> p) {
  constexpr int kWarps = kPanelThreads / 32;
  const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int R = p.n - p.k, kb = p.kb;
  const int per = (R + G - 1) / G;
  const int lo = p.k + min(g * per, R), hi = p.k + min((g + 1) * per, R), nr = hi - lo;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* rows = reinterpret_cast<cpx<T>*>(smem_raw);                       // [per][kb]
  unsigned char* chosen = smem_raw + (size_t)per * kb * sizeof(cpx<T>);     // [per]
  __shared__ cpx<T> prow[kNb];
  __shared__ unsigned long long wk[kWarps];
  __shared__ unsigned long long s_win;
  __shared__ int s_piv[kNb];
  __shared__ int s_fail;
  for (int e = tid; e < nr * kb; e += blockDim.x)
    rows[e] = p.a[(int64_t)(lo + e / kb) * p.ld + p.k + e % kb];
  for (int i = tid; i < per; i += blockDim.x) chosen[i] = 0;
  if (tid == 0) s_fail = 0;
  __syncthreads();
  bool ok = true;
  for (int j = 0; j < kb; ++j) {
    const int buf = (p.k + j) & 1;
    const unsigned long long tag = (unsigned long long)((p.k + j) & 0xFFFF);
    const unsigned long long mine = cta_best_key<T, kWarps>(rows, chosen, nr, kb, j, lo, wk);
    if (mine != 0) {
      const int bl = key_row(mine) - lo;
      for (int t = tid; t < kb - j; t += blockDim.x)
        p.cand_data[((size_t)buf * G + g) * kNb + t] = rows[bl * kb + j + t];
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();   // the entries before the key
      *reinterpret_cast<volatile unsigned long long*>(p.slot + buf * G + g) = mine | tag;
    }
    if (warp == 0) {
      unsigned long long kmax = 0;
      bool fine = true;
      for (int t = lane; t < G && fine; t += 32) {
        const volatile unsigned long long* sp = reinterpret_cast<const volatile unsigned long long*>(p.slot + buf * G + t);
        unsigned polls = 0;
        unsigned long long x = *sp;
        while ((x & 0xFFFFull) != tag) {
          if (++polls > kBarrierPolls) {
            fine = false;
            break;
          }
          if (polls > 256) __nanosleep(32);
          x = *sp;
        }
        kmax = umax64(kmax, x & ~0xFFFFull);
      }
      const bool all_fine = __all_sync(0xffffffffu, fine);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) kmax = umax64(kmax, __shfl_xor_sync(0xffffffffu, kmax, off));
      __threadfence();   // the winner's entries after its key
      if (lane == 0) {
        s_win = kmax;
        if (!all_fine) s_fail = 1;
      }
    }
    __syncthreads();
    if (s_fail) {
      ok = false;
      break;
    }
    const unsigned long long win = s_win;
    const int pr = win != 0 ? key_row(win) : -1;
    if (!(pr >= p.k && pr < p.n)) {   // no row left (cannot happen with n - k >= kb)
      if (tid == 0 && g == 0) atomicOr(p.err, 4);
      ok = false;
      break;
    }
    if ((win >> 32) == 0 && tid == 0 && g == 0) atomicOr(p.err, 4);   // a zero pivot
    const int w = (pr - p.k) / per;   // the CTA whose candidate it is
    for (int t = tid; t < kb - j; t += blockDim.x) prow[t] = ldcg(p.cand_data + ((size_t)buf * G + w) * kNb + t);
    if (tid == 0) {
      if (pr >= lo && pr < hi) chosen[pr - lo] = 1;
      s_piv[j] = pr;
    }
    __syncthreads();
    const cpx<T> inv = crecip(prow[0]);
    // eliminate column j from this CTA's other rows: the multipliers first (one thread per
    // row), then the updates (one warp per row, lanes over columns; rows independent)
    for (int i = tid; i < nr; i += blockDim.x)
      if (!chosen[i]) rows[i * kb + j] = rows[i * kb + j] * inv;
    __syncthreads();
#pragma unroll 4
    for (int i = warp; i < nr; i += kWarps) {
      if (chosen[i]) continue;
      cpx<T>* row = rows + i * kb + j;
      const cpx<T> l = row[0];
      const cpx<T> ml = mk(-l.re, -l.im);
      for (int t = 1 + lane; t < kb - j; t += 32) cmac(row[t], ml, prow[t]);
    }
    __syncthreads();
  }
  if (!ok) {
    // the panel stopped (a zero pivot or a wait that ran out): no row moves for it
    if (tid == 0 && s_fail) atomicOr(p.err, 2);
    if (tid == 0 && g == 0) *p.n_moves = 0;
    return;
  }
  for (int e = tid; e < nr * kb; e += blockDim.x)
    p.a[(int64_t)(lo + e / kb) * p.ld + p.k + e % kb] = rows[e];
  if (g == 0 && tid == 0) panel_record_moves(p, s_piv);
}

// ---- the panel inside one thread-block cluster (distributed shared memory)
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// all threads of all CTAs of the cluster; orders this CTA's shared-memory writes before
// the peers' reads after the barrier
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// the address of `p` (this CTA's shared memory) in the shared memory of cluster CTA `rank`
__device__ __forceinline__ uint32_t cluster_addr(const void* p, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(tc::smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ unsigned long long ld_cluster_u64(uint32_t a) {
  unsigned long long v;
  asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ cpx<float> ld_cluster_cpx(const cpx<float>*, uint32_t a) {
  float x, y;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(a) : "memory");
  return mk(x, y);
}
__device__ __forceinline__ cpx<double> ld_cluster_cpx(const cpx<double>*, uint32_t a) {
  double x, y;
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(x), "=d"(y) : "r"(a) : "memory");
  return mk(x, y);
}

// One panel of kb columns on rows k..n-1, the grid being one cluster of G CTAs.  Each CTA
// holds its slice of rows in shared memory for the whole panel.  Per column it posts its
// best pivot key in its own shared memory, the cluster barrier, then every CTA reads the
// G keys and takes the largest (the same pivot as the grid form), and reads the pivot row
// from the owner's shared memory.  The candidate slots are double-buffered by column: a CTA writes
// the slot of column j + 2 only after the barrier of column j + 1, which every CTA passes
// after its reads of column j.  A chosen row is never written again in the panel, so the
// pivot row is read while its owner eliminates its other rows.  A last cluster barrier
// keeps every CTA's shared memory in place until no peer reads it.
template <class T>
__global__ void __launch_bounds__(kPanelThreads) lu_panel_cluster_kernel(PanelArgs<T> p) {
  constexpr int kWarps = kPanelThreads / 32;
  const int G = gridDim.x, g = (int)cluster_rank(), tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int R = p.n - p.k, kb = p.kb;
  const int per = (R + G - 1) / G;
  const int lo = p.k + min(g * per, R), hi = p.k + min((g + 1) * per, R), nr = hi - lo;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* rows = reinterpret_cast<cpx<T>*>(smem_raw);                       // [per][kb]
  unsigned char* chosen = smem_raw + (size_t)per * kb * sizeof(cpx<T>);     // [per]
  __shared__ cpx<T> prow[kNb];
  __shared__ unsigned long long wk[kWarps];
  __shared__ int s_piv[kNb];
  __shared__ unsigned long long s_ck[2];   // this CTA's key of the column, by column parity
  __shared__ unsigned long long s_win;
  for (int e = tid; e < nr * kb; e += blockDim.x)
    rows[e] = p.a[(int64_t)(lo + e / kb) * p.ld + p.k + e % kb];
  for (int i = tid; i < per; i += blockDim.x) chosen[i] = 0;
  __syncthreads();
  bool ok = true;
  for (int j = 0; j < kb; ++j) {
    const int buf = j & 1;
    const unsigned long long mine = cta_best_key<T, kWarps>(rows, chosen, nr, kb, j, lo, wk);
    if (tid == 0) s_ck[buf] = mine;
    cluster_sync_all();
    // the pivot: the largest key over the cluster (the same choice in every CTA)
    if (warp == 0) {
      unsigned long long kmax = lane < G ? ld_cluster_u64(cluster_addr(&s_ck[buf], lane)) : 0ull;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) kmax = umax64(kmax, __shfl_xor_sync(0xffffffffu, kmax, off));
      if (lane == 0) s_win = kmax;
    }
    __syncthreads();
    const unsigned long long win = s_win;
    const int pr = win != 0 ? key_row(win) : -1;
    if (!(pr >= p.k && pr < p.n)) {   // no row left (cannot happen with n - k >= kb): every CTA stops here
      if (tid == 0 && g == 0) atomicOr(p.err, 4);
      ok = false;
      break;
    }
    if ((win >> 32) == 0 && tid == 0 && g == 0) atomicOr(p.err, 4);   // a zero pivot
    {
      // the pivot row's entries j.. from its owner (its local row pr - lo_w, lo_w = k + w per)
      const int w = (pr - p.k) / per;
      const int lrow = pr - (p.k + w * per);
      const cpx<T>* src = rows + (size_t)lrow * kb + j;
      for (int t = tid; t < kb - j; t += blockDim.x) prow[t] = ld_cluster_cpx(src, cluster_addr(src + t, w));
    }
    if (tid == 0) {
      if (pr >= lo && pr < hi) chosen[pr - lo] = 1;
      s_piv[j] = pr;
    }
    __syncthreads();
    const cpx<T> inv = crecip(prow[0]);
    for (int i = tid; i < nr; i += blockDim.x)
      if (!chosen[i]) rows[i * kb + j] = rows[i * kb + j] * inv;
    __syncthreads();
#pragma unroll 4
    for (int i = warp; i < nr; i += kWarps) {
      if (chosen[i]) continue;
      cpx<T>* row = rows + i * kb + j;
      const cpx<T> l = row[0];
      const cpx<T> ml = mk(-l.re, -l.im);
      for (int t = 1 + lane; t < kb - j; t += 32) cmac(row[t], ml, prow[t]);
    }
    __syncthreads();
  }
  if (ok) {
    for (int e = tid; e < nr * kb; e += blockDim.x)
      p.a[(int64_t)(lo + e / kb) * p.ld + p.k + e % kb] = rows[e];
    if (g == 0 && tid == 0) panel_record_moves(p, s_piv);
  } else if (tid == 0 && g == 0) {
    *p.n_moves = 0;   // the panel stopped: no row moves for it
  }
  cluster_sync_all();
}

// the panel's row moves on columns [0, n_cols): all sources read before any destination
// is written (16 columns per block, every move)
template <class T>
__global__ void __launch_bounds__(256) lu_moves_kernel(cpx<T>* a, int64_t ld, int n_cols, const int2* moves,
                                                       const int* n_moves) {
  __shared__ cpx<T> buf[2 * kNb][16];
  __shared__ int2 mv[2 * kNb];
  const int nm = max(0, min(*n_moves, 2 * kNb));
  const int tid = threadIdx.x, cl = tid & 15, mr = tid >> 4;
  const int col = blockIdx.x * 16 + cl;
  // a move outside the matrix (none is written; checked all the same) is dropped
  for (int m = tid; m < nm; m += blockDim.x) {
    const int2 v = moves[m];
    mv[m] = (v.x >= 0 && v.x < n_cols && v.y >= 0 && v.y < n_cols) ? v : make_int2(-1, -1);
  }
  __syncthreads();
  for (int m = mr; m < nm; m += 16)
    if (col < n_cols && mv[m].x >= 0) buf[m][cl] = a[(int64_t)mv[m].x * ld + col];
  __syncthreads();
  for (int m = mr; m < nm; m += 16)
    if (col < n_cols && mv[m].x >= 0) a[(int64_t)mv[m].y * ld + col] = buf[m][cl];
}

// Column-oriented substitution with one warp: the right-hand side's entries of rows
// lane and lane + 32 stay in the lane's registers; at step j the solved entry x_j is
// shuffled to every lane, and the rows below (lower) or above (upper) subtract their
// coefficient times x_j.  M: the kb x kb diagonal block in shared memory (row stride ms).
template <class T, bool UPPER>
__device__ __forceinline__ void warp_substitute(const cpx<T>* M, int ms, int kb, cpx<T>& x0, cpx<T>& x1) {
  const int lane = threadIdx.x & 31;
  for (int s = 0; s < kb; ++s) {
    const int j = UPPER ? kb - 1 - s : s;
    if (UPPER) {   // x_j /= U_jj by the lane that holds row j
      if (j < 32 && lane == j) x0 = cdiv(x0, M[j * ms + j]);
      if (j >= 32 && lane == j - 32) x1 = cdiv(x1, M[j * ms + j]);
    }
    const T r0 = __shfl_sync(0xffffffffu, j < 32 ? x0.re : x1.re, j & 31);
    const T i0 = __shfl_sync(0xffffffffu, j < 32 ? x0.im : x1.im, j & 31);
    const cpx<T> xj = mk(-r0, -i0);
    const bool t0 = UPPER ? lane < j : (lane > j && lane < kb);
    const bool t1 = UPPER ? lane + 32 < j : (lane + 32 > j && lane + 32 < kb);
    if (t0) cmac(x0, M[lane * ms + j], xj);
    if (t1) cmac(x1, M[(lane + 32) * ms + j], xj);
  }
}

// U12 = L11^-1 A12 on rows k..k+kb-1: L11 and a tile of 32 columns in shared memory,
// one warp per column (lanes over rows), the tile stored back coalesced
template <class T>
__global__ void __launch_bounds__(256) lu_trsm_kernel(cpx<T>* a, int64_t ld, int n, int k, int kb) {
  constexpr int TC = 32, LS = kNb + 1;
  extern __shared__ __align__(16) unsigned char sm[];
  cpx<T>* L = reinterpret_cast<cpx<T>*>(sm);          // [kb][LS]
  cpx<T>* X = L + kNb * LS;                            // [kNb][TC]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c0 = k + kb + blockIdx.x * TC;
  for (int e = tid; e < kb * kb; e += blockDim.x) L[(e / kb) * LS + e % kb] = a[(int64_t)(k + e / kb) * ld + k + e % kb];
  for (int e = tid; e < kb * TC; e += blockDim.x) {
    const int r = e / TC, c = e % TC;
    X[r * TC + c] = c0 + c < n ? a[(int64_t)(k + r) * ld + c0 + c] : mk((T)0, (T)0);
  }
  __syncthreads();
  for (int c = warp; c < TC; c += blockDim.x / 32) {
    cpx<T> x0 = lane < kb ? X[lane * TC + c] : mk((T)0, (T)0);
    cpx<T> x1 = lane + 32 < kb ? X[(lane + 32) * TC + c] : mk((T)0, (T)0);
    warp_substitute<T, false>(L, LS, kb, x0, x1);
    if (lane < kb) X[lane * TC + c] = x0;
    if (lane + 32 < kb) X[(lane + 32) * TC + c] = x1;
  }
  __syncthreads();
  for (int e = tid; e < kb * TC; e += blockDim.x) {
    const int r = e / TC, c = e % TC;
    if (c0 + c < n) a[(int64_t)(k + r) * ld + c0 + c] = X[r * TC + c];
  }
}

// A22 -= L21 U12: a 64 x 64 tile of complex entries per block, 256 threads with 4 x 4 each,
// the whole K (the panel width) staged in shared memory (A transposed, padded)
template <class T>
__global__ void __launch_bounds__(256) lu_gemm_kernel(cpx<T>* a, int64_t ld, int n, int k, int kb) {
  constexpr int BM = 64, BN = 64, PA = BM + 1;
  extern __shared__ unsigned char sm[];
  cpx<T>* As = reinterpret_cast<cpx<T>*>(sm);   // [kb][PA]
  cpx<T>* Bs = As + kb * PA;                    // [kb][BN]
  const int tid = threadIdx.x;
  const int r0 = k + kb + blockIdx.y * BM, c0 = k + kb + blockIdx.x * BN;
  for (int e = tid; e < BM * kb; e += 256) {
    const int row = e / kb, kk = e % kb;
    As[kk * PA + row] = r0 + row < n ? a[(int64_t)(r0 + row) * ld + k + kk] : mk((T)0, (T)0);
  }
  for (int e = tid; e < kb * BN; e += 256) {
    const int kk = e / BN, col = e % BN;
    Bs[kk * BN + col] = c0 + col < n ? a[(int64_t)(k + kk) * ld + c0 + col] : mk((T)0, (T)0);
  }
  __syncthreads();
  const int ty = tid >> 4, tx = tid & 15;
  cpx<T> acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mk((T)0, (T)0);
  for (int kk = 0; kk < kb; ++kk) {
    cpx<T> av[4], bv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) av[i] = As[kk * PA + ty * 4 + i];
#pragma unroll
    for (int j = 0; j < 4; ++j) bv[j] = Bs[kk * BN + tx * 4 + j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) cmac(acc[i][j], av[i], bv[j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty * 4 + i;
    if (r >= n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int cc = c0 + tx * 4 + j;
      if (cc < n) {
        cpx<T>& z = a[(int64_t)r * ld + cc];
        z = z - acc[i][j];
      }
    }
  }
}

// ---- A22 -= L21 U12 on the tensor cores (complex64).  With the rows of L21 and of A22
// stored interleaved (re, im), one tile
//   D (128 rows x 128 reals = 64 complex columns) = A' (128 x 2 kb) B' (2 kb x 128)
// with A' the rows of L21 as stored (k' = 2 c + part) and
//   B'^T[2j][2c] = Re U_cj, B'^T[2j][2c+1] = -Im U_cj,
//   B'^T[2j+1][2c] = Im U_cj, B'^T[2j+1][2c+1] = Re U_cj
// holds (Re, Im) of (L21 U12)_ij in columns 2j, 2j+1: the layout of A22 itself.  Three
// TF32 products (head x head into one tensor-memory accumulator, the two corrections
// into a second, added in FP32 registers), K staged 16 reals (8 panel columns) at a time
// in two buffers, so the threads build one stage while the tensor core consumes the
// other.  Every mbarrier wait is bounded; a wait that runs out sets bit 3 of err and the
// CTA issues nothing more.
constexpr int kUM = 128, kUN = 128, kUK = 16;   // tile rows, tile real columns, reals per stage
constexpr uint32_t kUSbo = (kUK / 4) * 128;      // 8-row group stride of the K-major operands
constexpr size_t kUStage = (size_t)2 * kUM * kUK * 4 + (size_t)2 * kUN * kUK * 4;
// shared bytes per CTA: two stages, padded so that at most two CTAs share an SM (their
// 2 x 256 tensor-memory columns then always fit)
constexpr size_t kUSmem = 96 * 1024;
static_assert(2 * kUStage + 128 <= kUSmem, "update stages");
constexpr int kUPitch = kUN + 4;                 // row pitch (floats) of the staged product tile
static_assert((size_t)kUM * kUPitch * 4 + 128 <= kUSmem, "staged product tile");

__global__ void __launch_bounds__(256, 2) lu_gemm_tc_kernel(cpx<float>* a, int64_t ld, int n, int k, int kb, int* err) {
  extern __shared__ __align__(128) unsigned char sm_raw[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t taddr_s;
  __shared__ int s_fail;
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(sm_raw) + 127) & ~(uintptr_t)127);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r0 = k + kb + blockIdx.y * kUM;          // first row of the tile
  const int c0 = k + kb + blockIdx.x * (kUN / 2);    // first complex column of the tile
  float* af = reinterpret_cast<float*>(a);
  const int64_t ldf = 2 * ld;
  if (tid == 0) {
    s_fail = 0;
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tc::tmem_alloc(&taddr_s, 256);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = taddr_s;
  const uint32_t idesc = tc::idesc_tf32(kUM, kUN);
  const int n_stages = (2 * kb + kUK - 1) / kUK;
  // A: rows (tid >> 3) + 32 q, q < 4, reals 2 p, 2 p + 1 of the stage's 16 (p = tid & 7): the
  // eight lanes of a row read its 64 bytes of the stage together
  const int arow = tid >> 3, apiece = tid & 7;
  const int brow = tid >> 5, bcol = tid & 31;   // B: panel row of the stage, columns bcol, bcol + 32
  auto failed = [&]() { return *reinterpret_cast<volatile int*>(&s_fail) != 0; };
  // a stage's global values, loaded one stage ahead (in flight across the barrier and the
  // MMA issue of the stage before)
  float2 av[4];
  cpx<float> bv[2];
  auto load_stage = [&](int st) {
    const int f = kUK * st + 2 * apiece;   // even, as is 2 kb: both reals are in range or neither
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int R = r0 + arow + 32 * q;
      av[q] = (R < n && f < 2 * kb) ? __ldcg(reinterpret_cast<const float2*>(af + (int64_t)R * ldf + 2 * (int64_t)k + f))
                                    : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int j = bcol + 32 * u, c = (kUK / 2) * st + brow;
      float2 x = make_float2(0.f, 0.f);
      if (c < kb && c0 + j < n) x = __ldcg(reinterpret_cast<const float2*>(a + (int64_t)(k + c) * ld + c0 + j));
      bv[u] = mk(x.x, x.y);
    }
  };
  load_stage(0);
  uint32_t n_issued = 0;
  for (int st = 0; st < n_stages; ++st) {
    const int buf = st & 1;
    float* Ahi = reinterpret_cast<float*>(base + buf * kUStage);
    float* Alo = Ahi + kUM * kUK;
    float* Bhi = Alo + kUM * kUK;
    float* Blo = Bhi + kUN * kUK;
    if (st >= 2) {
      // the MMAs of stage st - 2 read this buffer: one lane per warp polls, the others wait
      if (lane == 0 && !failed() && !tc::mbar_wait(&mbar[buf], ((st - 2) >> 1) & 1, kTcPolls)) atomicOr(&s_fail, 1);
      __syncwarp();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      // A: reals 16 st + 2 apiece, + 1 of row r0 + arow + 32 q of L21 (zero outside)
      float h0, l0, h1, l1;
      tf32_split(av[q].x, h0, l0);
      tf32_split(av[q].y, h1, l1);
      const uint32_t off = tc::kmajor_offset(arow + 32 * q, 2 * apiece, kUK) / 4;
      *reinterpret_cast<float2*>(Ahi + off) = make_float2(h0, h1);
      *reinterpret_cast<float2*>(Alo + off) = make_float2(l0, l1);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      // B: U12 entry (panel column 8 st + brow, tile column bcol + 32 u), four reals of B'^T
      const int j = bcol + 32 * u;
      float h0, l0, h1, l1;
      tf32_split(bv[u].re, h0, l0);
      tf32_split(bv[u].im, h1, l1);
      const uint32_t o0 = tc::kmajor_offset(2 * j, 2 * brow, kUK) / 4;
      const uint32_t o1 = tc::kmajor_offset(2 * j + 1, 2 * brow, kUK) / 4;
      *reinterpret_cast<float2*>(Bhi + o0) = make_float2(h0, -h1);
      *reinterpret_cast<float2*>(Blo + o0) = make_float2(l0, -l1);
      *reinterpret_cast<float2*>(Bhi + o1) = make_float2(h1, h0);
      *reinterpret_cast<float2*>(Blo + o1) = make_float2(l1, l0);
    }
    if (st + 1 < n_stages) load_stage(st + 1);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && !failed()) {
      tc::fence_after_sync();
      const uint32_t ah = tc::smem_u32(Ahi), al = tc::smem_u32(Alo), bh = tc::smem_u32(Bhi), bl = tc::smem_u32(Blo);
#pragma unroll
      for (int s2 = 0; s2 < kUK / 8; ++s2) {
        const uint32_t ko = s2 * 256;
        const uint64_t dah = tc::sdesc(ah + ko, 128, kUSbo), dal = tc::sdesc(al + ko, 128, kUSbo);
        const uint64_t dbh = tc::sdesc(bh + ko, 128, kUSbo), dbl = tc::sdesc(bl + ko, 128, kUSbo);
        const uint32_t accf = (st > 0 || s2 > 0) ? 1u : 0u;
        tc::mma_tf32(tmem + kUN, dah, dbl, idesc, accf);
        tc::mma_tf32(tmem + kUN, dal, dbh, idesc, 1u);
        tc::mma_tf32(tmem, dah, dbh, idesc, accf);
      }
      tc::mma_commit(&mbar[buf]);
      ++n_issued;
    }
  }
  // A22's tile, read while the last products run (the tile is this CTA's alone): warp w
  // takes tile rows 16 w .. 16 w + 15, its lanes consecutive complex columns (two
  // 256-byte halves of each row)
  float2 cz[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int R = r0 + 16 * warp + (i >> 1), jc = c0 + 32 * (i & 1) + lane;
    cz[i] = (R < n && jc < n) ? __ldcg(reinterpret_cast<const float2*>(af + (int64_t)R * ldf + 2 * (int64_t)jc))
                              : make_float2(0.f, 0.f);
  }
  // the last commit covers every MMA of the CTA
  if (tid == 0 && !failed() && n_stages > 0) {
    const int last = n_stages - 1;
    if (!tc::mbar_wait(&mbar[last & 1], (last >> 1) & 1, kTcPolls)) atomicOr(&s_fail, 1);
  }
  __syncthreads();
  tc::fence_after_sync();
  const bool ok = !failed();   // no writer is left: the same value in every thread
  if (ok) {
    // the products (tensor-memory lane = tile row; warp w: lanes 32 (w mod 4).., real columns
    // 64 (w / 4)..) into a shared tile over the stage buffers, which the finished MMAs no
    // longer read
    float* T = reinterpret_cast<float*>(base);
    const int lq = warp & 3, ch = warp >> 2;
    const int r = 32 * lq + lane;
    const uint32_t tl = (uint32_t)(32 * lq) << 16;
#pragma unroll
    for (int cb = 0; cb < 64; cb += 16) {
      const int col = 64 * ch + cb;
      float v[16], w[16];
      tc::tmem_ld16x2(tmem + tl + (uint32_t)col, tmem + tl + (uint32_t)(kUN + col), v, w);
#pragma unroll
      for (int i = 0; i < 16; i += 4)
        *reinterpret_cast<float4*>(T + r * kUPitch + col + i) =
            make_float4(v[i] + w[i], v[i + 1] + w[i + 1], v[i + 2] + w[i + 2], v[i + 3] + w[i + 3]);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const int rr = 16 * warp + (i >> 1), h = i & 1;
      const int R = r0 + rr, jc = c0 + 32 * h + lane;
      const float2 d = *reinterpret_cast<const float2*>(T + rr * kUPitch + 64 * h + 2 * lane);
      if (R < n && jc < n)
        *reinterpret_cast<float2*>(af + (int64_t)R * ldf + 2 * (int64_t)jc) = make_float2(cz[i].x - d.x, cz[i].y - d.y);
    }
  } else if (tid == 0) {
    atomicOr(err, 8);
    // a bounded wait for the MMAs in flight before their tensor memory is freed
    if (n_issued > 0) tc::mbar_wait(&mbar[(n_issued - 1) & 1], ((n_issued - 1) >> 1) & 1, kTcPolls);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// every panel's row moves on the right-hand side, in panel order (one block)
template <class T>
__global__ void lu_vector_moves_kernel(cpx<T>* x, int n, int n_panels, const int2* moves, const int* n_moves) {
  __shared__ cpx<T> buf[2 * kNb];
  for (int pnl = 0; pnl < n_panels; ++pnl) {
    const int nm = max(0, min(n_moves[pnl], 2 * kNb));
    const int2* mv = moves + (size_t)pnl * 2 * kNb;
    auto valid = [&](int2 v) { return v.x >= 0 && v.x < n && v.y >= 0 && v.y < n; };
    for (int m = threadIdx.x; m < nm; m += blockDim.x)
      if (valid(mv[m])) buf[m] = x[mv[m].x];
    __syncthreads();
    for (int m = threadIdx.x; m < nm; m += blockDim.x)
      if (valid(mv[m])) x[mv[m].y] = buf[m];
    __syncthreads();
  }
}

// the diagonal block of rows k..k+kb-1 into shared memory (coalesced), then one warp
// solves it against src[k..k+kb) (unit lower: forward; upper: backward) into xb
template <class T, bool UPPER>
__device__ void block_solve(const cpx<T>* a, int64_t ld, int k, int kb, const cpx<T>* src, cpx<T>* D,
                            cpx<T>* xb) {
  constexpr int LS = kNb + 1;
  for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) D[(e / kb) * LS + e % kb] = a[(int64_t)(k + e / kb) * ld + k + e % kb];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    cpx<T> x0 = lane < kb ? src[k + lane] : mk((T)0, (T)0);
    cpx<T> x1 = lane + 32 < kb ? src[k + lane + 32] : mk((T)0, (T)0);
    warp_substitute<T, UPPER>(D, LS, kb, x0, x1);
    if (lane < kb) xb[lane] = x0;
    if (lane + 32 < kb) xb[lane + 32] = x1;
  }
  __syncthreads();
}

// forward step of panel k: y_b = L11^-1 x_b (written to y), x[r] -= L[r][k..] y_b for the
// rows below (one warp per row)
template <class T>
__global__ void __launch_bounds__(256) lu_forward_kernel(const cpx<T>* a, int64_t ld, int n, int k, int kb,
                                                         cpx<T>* x, cpx<T>* y) {
  __shared__ cpx<T> yb[kNb];
  extern __shared__ __align__(16) unsigned char sm[];
  block_solve<T, false>(a, ld, k, kb, x, reinterpret_cast<cpx<T>*>(sm), yb);
  if (blockIdx.x == 0)
    for (int t = threadIdx.x; t < kb; t += blockDim.x) y[k + t] = yb[t];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = k + kb + blockIdx.x * nw + warp; r < n; r += gridDim.x * nw) {
    cpx<T> acc = mk((T)0, (T)0);
    for (int j = lane; j < kb; j += 32) cmac(acc, a[(int64_t)r * ld + k + j], yb[j]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      acc.re += __shfl_xor_sync(0xffffffffu, acc.re, off);
      acc.im += __shfl_xor_sync(0xffffffffu, acc.im, off);
    }
    if (lane == 0) x[r] = x[r] - acc;
  }
}

// backward step of panel k: x_b = U11^-1 y_b (written to x), y[r] -= U[r][k..] x_b for the
// rows above
template <class T>
__global__ void __launch_bounds__(256) lu_backward_kernel(const cpx<T>* a, int64_t ld, int k, int kb,
                                                          cpx<T>* y, cpx<T>* x) {
  __shared__ cpx<T> xb[kNb];
  extern __shared__ __align__(16) unsigned char sm[];
  block_solve<T, true>(a, ld, k, kb, y, reinterpret_cast<cpx<T>*>(sm), xb);
  if (blockIdx.x == 0)
    for (int t = threadIdx.x; t < kb; t += blockDim.x) x[k + t] = xb[t];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = blockIdx.x * nw + warp; r < k; r += gridDim.x * nw) {
    cpx<T> acc = mk((T)0, (T)0);
    for (int j = lane; j < kb; j += 32) cmac(acc, a[(int64_t)r * ld + k + j], xb[j]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      acc.re += __shfl_xor_sync(0xffffffffu, acc.re, off);
      acc.im += __shfl_xor_sync(0xffffffffu, acc.im, off);
    }
    if (lane == 0) y[r] = y[r] - acc;
  }
}

// r = b - Z x in float64 from the float64 matrix (one warp per row), and |r|^2, |b|^2 sums
__global__ void __launch_bounds__(256) residual_kernel(const cpx<double>* z, int64_t ld, int n, const cpx<double>* x,
                                                       const cpx<double>* b, cpx<double>* r, double* sums) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double rr = 0.0, bb = 0.0;
  for (int i = blockIdx.x * nw + warp; i < n; i += gridDim.x * nw) {
    cpx<double> acc = mk(0.0, 0.0);
    for (int j = lane; j < n; j += 32) cmac(acc, z[(int64_t)i * ld + j], x[j]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      acc.re += __shfl_xor_sync(0xffffffffu, acc.re, off);
      acc.im += __shfl_xor_sync(0xffffffffu, acc.im, off);
    }
    if (lane == 0) {
      const cpx<double> v = b[i] - acc;
      if (r) r[i] = v;
      rr += v.re * v.re + v.im * v.im;
      bb += b[i].re * b[i].re + b[i].im * b[i].im;
    }
  }
  if (lane == 0) {
    atomicAdd(sums, rr);
    atomicAdd(sums + 1, bb);
  }
}

// the same residual from a complex64 matrix and vectors (accumulated in float64)
__global__ void __launch_bounds__(256) residual32_kernel(const cpx<float>* z, int64_t ld, int n, const cpx<float>* x,
                                                         const cpx<float>* b, double* sums) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double rr = 0.0, bb = 0.0;
  for (int i = blockIdx.x * nw + warp; i < n; i += gridDim.x * nw) {
    cpx<double> acc = mk(0.0, 0.0);
    for (int j = lane; j < n; j += 32) cmac(acc, ccast<double>(z[(int64_t)i * ld + j]), ccast<double>(x[j]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      acc.re += __shfl_xor_sync(0xffffffffu, acc.re, off);
      acc.im += __shfl_xor_sync(0xffffffffu, acc.im, off);
    }
    if (lane == 0) {
      const cpx<double> v = ccast<double>(b[i]) - acc;
      rr += v.re * v.re + v.im * v.im;
      bb += (double)b[i].re * b[i].re + (double)b[i].im * b[i].im;
    }
  }
  if (lane == 0) {
    atomicAdd(sums, rr);
    atomicAdd(sums + 1, bb);
  }
}

// copy an n x n block (row stride ld_src) into a dense n x n buffer, changing precision
template <class TD, class TS>
__global__ void copy_matrix_kernel(const cpx<TS>* src, int64_t ld, int n, cpx<TD>* dst) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    dst[e] = ccast<TD>(src[i * ld + j]);
  }
}

template <class TD, class TS>
__global__ void copy_vector_kernel(const cpx<TS>* src, int n, cpx<TD>* dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = ccast<TD>(src[i]);
}

// x += d (float64 + float32 correction); sums[0] += |d|^2, sums[1] += |x|^2
__global__ void add_correction_kernel(cpx<double>* x, const cpx<float>* d, int n, double* sums) {
  double dd = 0.0, xx = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const cpx<double> di = ccast<double>(d[i]);
    const cpx<double> v = x[i] + di;
    x[i] = v;
    dd += di.re * di.re + di.im * di.im;
    xx += v.re * v.re + v.im * v.im;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    dd += __shfl_xor_sync(0xffffffffu, dd, off);
    xx += __shfl_xor_sync(0xffffffffu, xx, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(sums, dd);
    atomicAdd(sums + 1, xx);
  }
}

// V'_{e,a} = sum_i conj(Q_ia) V_{e,i}  (Eq. 4), one thread per (element, MBF)
template <class T>
__global__ void reduced_excitation_kernel(int n_el, int n_basis, int m, const cpx<T>* v, const cpx<double>* q,
                                          cpx<T>* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_el * m) return;
  const int e = t / m, a = t % m;
  cpx<double> acc = mk(0.0, 0.0);
  for (int i = 0; i < n_basis; ++i) cmac_conj(acc, q[(size_t)i * m + a], ccast<double>(v[(size_t)e * n_basis + i]));
  out[t] = ccast<T>(acc);
}

// delta-gap port across basis function `port`: V'_{e,a} = amp_e conj(Q_port,a)
template <class T>
__global__ void port_excitation_kernel(int n_el, int m, int port, const cpx<T>* amp, const cpx<double>* q,
                                       cpx<T>* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_el * m) return;
  const int e = t / m, a = t % m;
  out[t] = ccast<T>(conj(q[(size_t)port * m + a]) * ccast<double>(amp[e]));
}

// port current of element e: (Q I'_e)[port] = sum_a Q_port,a I'_{e,a}
template <class T>
__global__ void port_currents_kernel(int n_el, int m, int port, const cpx<T>* ired, const cpx<double>* q,
                                     cpx<T>* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_el) return;
  cpx<double> acc = mk(0.0, 0.0);
  for (int a = 0; a < m; ++a) cmac(acc, q[(size_t)port * m + a], ccast<double>(ired[(size_t)e * m + a]));
  out[e] = ccast<T>(acc);
}

int grid_for(int64_t items, int per_block, int cap) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((items + per_block - 1) / per_block, cap));
}

}  // namespace

int lu_panel_width() { return kNb; }

// panel CTAs: enough that each CTA's rows fit kPanelSmem bytes of shared memory, and about
// kPanelRows rows each (the per-column elimination is short; the grid barrier's cost grows
// slowly with the CTA count), at most one per SM
constexpr size_t kPanelSmem = 160 * 1024;
constexpr int kPanelRows = 64;

template <class T>
int lu_panel_grid(int rows, int sms) {
  const int64_t row_bytes = (int64_t)kNb * sizeof(cpx<T>);
  const int64_t need = (rows * row_bytes + (int64_t)kPanelSmem - 1) / (int64_t)kPanelSmem;
  const int64_t g = std::max<int64_t>(need, std::min<int64_t>(sms, (rows + kPanelRows - 1) / kPanelRows));
  return (int)std::max<int64_t>(1, g);
}

// the most rows of a panel of kb columns that one cluster of cs CTAs holds in shared
// memory (the opt-in limit per CTA less room for the kernel's static words)
template <class T>
int cluster_panel_rows(int cs, int kb, int smem_optin) {
  const int64_t avail = std::max<int64_t>(0, (int64_t)smem_optin - 4096);
  return (int)std::min<int64_t>((int64_t)cs * (avail / ((int64_t)kb * (int64_t)sizeof(cpx<T>) + 1)), 1 << 30);
}

// panels of at most this many rows run on the cluster: there its cheaper barrier wins
// (GB300, 16 CTAs: 12.2 ms against 15.0 for the whole 2,000^2 complex64 factorization);
// on longer panels the elimination work of its 16 CTAs outweighs it (8,000^2 with every
// panel that fits on the cluster: 90.3 ms against 83.6 on the grid)
constexpr int kClusterPanelRows = 2048;

// cluster size of the cluster panels on this device: 16 CTAs where the device schedules
// such a cluster with the shared memory it needs, else 8, else 0 (grid panels only)
template <class T>
int choose_panel_cluster(int smem_optin, cudaStream_t s) {
  const int dyn = std::max(0, smem_optin - 4096);
  if (cudaFuncSetAttribute(lu_panel_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) !=
          cudaSuccess ||
      cudaFuncSetAttribute(lu_panel_cluster_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  for (int c : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kPanelThreads);
    cfg.dynamicSmemBytes = (size_t)dyn;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, lu_panel_cluster_kernel<T>, &cfg) == cudaSuccess && nc >= 1) return c;
    cudaGetLastError();
  }
  return 0;
}

template <class T>
int lu_max_order(int sms) {
  return (int)((int64_t)sms * (int64_t)kPanelSmem / ((int64_t)kNb * sizeof(cpx<T>)));
}

template <class T>
cudaError_t lu_factor(cpx<T>* a, int64_t ld, int n, const LuWork& w, cudaStream_t s) {
  const int sms = current_sm_count();
  const int n_panels = (n + kNb - 1) / kNb;
  if (lu_panel_grid<T>(n, sms) > sms) return cudaErrorInvalidValue;
  if (n > 65535) return cudaErrorInvalidValue;   // rows and column tags are 16-bit fields of the pivot keys
  // every panel CTA's key slots start with a tag no column has (0xFFFF)
  cudaError_t e = cudaMemsetAsync(w.cand_val, 0xFF, (size_t)2 * sms * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(w.err, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  // no row moves until a panel records its own (a panel that stops early records none)
  e = cudaMemsetAsync(w.n_moves, 0, (size_t)n_panels * sizeof(int), s);
  if (e != cudaSuccess) return e;
  const size_t trsm_smem = (size_t)kNb * (kNb + 1 + 32) * sizeof(cpx<T>);
  const size_t gemm_smem = (size_t)kNb * (65 + 64) * sizeof(cpx<T>);
  // the most shared memory any panel's CTAs take (the grid shrinks in steps as the rows do)
  size_t panel_smem0 = 0;
  for (int pnl = 0; pnl < n_panels; ++pnl) {
    const int R = n - pnl * kNb, G = lu_panel_grid<T>(R, sms), per = (R + G - 1) / G;
    panel_smem0 = std::max(panel_smem0, (size_t)per * kNb * sizeof(cpx<T>) + (size_t)per + 16);
  }
  if ((e = cudaFuncSetAttribute(lu_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)panel_smem0)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(lu_panel_kernel<T>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(lu_trsm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trsm_smem)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(lu_gemm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem)) !=
      cudaSuccess)
    return e;
  const bool tc_update = sizeof(T) == 4 && w.tc_update;
  if (tc_update && (e = cudaFuncSetAttribute(lu_gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kUSmem)) != cudaSuccess)
    return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lu_panel_kernel<T>, kPanelThreads,
                                                         panel_smem0)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int smem_optin = 0, dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
    return e;
  const int cs = w.panel_cluster ? choose_panel_cluster<T>(smem_optin, s) : 0;
  w.diag[3] = 0;
  w.diag[4] = cs;
  for (int pnl = 0; pnl < n_panels; ++pnl) {
    const int k = pnl * kNb, kb = std::min(kNb, n - k), R = n - k;
    PanelArgs<T> pa{a, ld, n, k, kb, reinterpret_cast<unsigned long long*>(w.cand_val),
                    reinterpret_cast<cpx<T>*>(w.cand_data), w.moves + (size_t)pnl * 2 * kNb, w.n_moves + pnl,
                    w.err};
    if (cs > 0 && R <= std::min(kClusterPanelRows, cluster_panel_rows<T>(cs, kb, smem_optin))) {
      const int per = (R + cs - 1) / cs;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cs);
      cfg.blockDim = dim3(kPanelThreads);
      cfg.dynamicSmemBytes = (size_t)per * kb * sizeof(cpx<T>) + (size_t)per + 16;
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cs;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      if ((e = cudaLaunchKernelEx(&cfg, lu_panel_cluster_kernel<T>, pa)) != cudaSuccess) return e;
      ++w.diag[3];
    } else {
      const int G = std::min(lu_panel_grid<T>(R, sms), per_sm * sms);   // all CTAs resident
      const int per = (R + G - 1) / G;
      const size_t psmem = (size_t)per * kb * sizeof(cpx<T>) + (size_t)per + 16;
      void* args[] = {&pa};
      w.diag[0] = G;
      w.diag[1] = per_sm;
      w.diag[2] = (int)psmem;
      if ((e = cudaLaunchCooperativeKernel((const void*)lu_panel_kernel<T>, dim3(G), dim3(kPanelThreads), args,
                                           psmem, s)) != cudaSuccess)
        return e;
    }
    lu_moves_kernel<T><<<(n + 15) / 16, 256, 0, s>>>(a, ld, n, w.moves + (size_t)pnl * 2 * kNb, w.n_moves + pnl);
    const int rest = n - k - kb;
    if (rest > 0) {
      lu_trsm_kernel<T><<<(rest + 31) / 32, 256, trsm_smem, s>>>(a, ld, n, k, kb);
      if constexpr (sizeof(T) == 4) {
        if (tc_update)
          lu_gemm_tc_kernel<<<dim3((rest + kUN / 2 - 1) / (kUN / 2), (rest + kUM - 1) / kUM), 256, kUSmem, s>>>(
              a, ld, n, k, kb, w.err);
        else
          lu_gemm_kernel<T><<<dim3((rest + 63) / 64, (rest + 63) / 64), 256, gemm_smem, s>>>(a, ld, n, k, kb);
      } else {
        lu_gemm_kernel<T><<<dim3((rest + 63) / 64, (rest + 63) / 64), 256, gemm_smem, s>>>(a, ld, n, k, kb);
      }
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <class T>
cudaError_t lu_solve(const cpx<T>* a, int64_t ld, int n, const LuWork& w, cpx<T>* x, cpx<T>* y, cudaStream_t s) {
  const int sms = current_sm_count();
  const int n_panels = (n + kNb - 1) / kNb;
  const size_t dsm = (size_t)kNb * (kNb + 1) * sizeof(cpx<T>);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(lu_forward_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(lu_backward_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm)) !=
      cudaSuccess)
    return e;
  lu_vector_moves_kernel<T><<<1, 128, 0, s>>>(x, n, n_panels, w.moves, w.n_moves);
  for (int pnl = 0; pnl < n_panels; ++pnl) {
    const int k = pnl * kNb, kb = std::min(kNb, n - k);
    lu_forward_kernel<T><<<grid_for(n - k - kb, 8, 2 * sms), 256, dsm, s>>>(a, ld, n, k, kb, x, y);
  }
  for (int pnl = n_panels - 1; pnl >= 0; --pnl) {
    const int k = pnl * kNb, kb = std::min(kNb, n - k);
    lu_backward_kernel<T><<<grid_for(k, 8, 2 * sms), 256, dsm, s>>>(a, ld, k, kb, y, x);
  }
  return cudaGetLastError();
}

cudaError_t residual_f64(const void* z, int64_t ld, int n, const void* x, const void* b, void* r, double* sums,
                         cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(sums, 0, 2 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  residual_kernel<<<grid_for(n, 8, 8 * current_sm_count()), 256, 0, s>>>(
      reinterpret_cast<const cpx<double>*>(z), ld, n, reinterpret_cast<const cpx<double>*>(x),
      reinterpret_cast<const cpx<double>*>(b), reinterpret_cast<cpx<double>*>(r), sums);
  return cudaGetLastError();
}

cudaError_t residual_f32(const void* z, int64_t ld, int n, const void* x, const void* b, double* sums,
                         cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(sums, 0, 2 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  residual32_kernel<<<grid_for(n, 8, 8 * current_sm_count()), 256, 0, s>>>(
      reinterpret_cast<const cpx<float>*>(z), ld, n, reinterpret_cast<const cpx<float>*>(x),
      reinterpret_cast<const cpx<float>*>(b), sums);
  return cudaGetLastError();
}

template <class TD, class TS>
cudaError_t copy_matrix(const void* src, int64_t ld, int n, void* dst, cudaStream_t s) {
  copy_matrix_kernel<TD, TS><<<grid_for((int64_t)n * n, 256, 16 * current_sm_count()), 256, 0, s>>>(
      reinterpret_cast<const cpx<TS>*>(src), ld, n, reinterpret_cast<cpx<TD>*>(dst));
  return cudaGetLastError();
}

template <class TD, class TS>
cudaError_t copy_vector(const void* src, int n, void* dst, cudaStream_t s) {
  copy_vector_kernel<TD, TS><<<grid_for(n, 256, 4 * current_sm_count()), 256, 0, s>>>(
      reinterpret_cast<const cpx<TS>*>(src), n, reinterpret_cast<cpx<TD>*>(dst));
  return cudaGetLastError();
}

cudaError_t add_correction(void* x, const void* d, int n, double* sums, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(sums, 0, 2 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  add_correction_kernel<<<grid_for(n, 256, 4 * current_sm_count()), 256, 0, s>>>(
      reinterpret_cast<cpx<double>*>(x), reinterpret_cast<const cpx<float>*>(d), n, sums);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_excitation(int kind, int n_el, int n_basis, int m, int port, const void* in, const double* q,
                              void* out, cudaStream_t s) {
  const cpx<double>* qd = reinterpret_cast<const cpx<double>*>(q);
  const int items = kind == 2 ? n_el : n_el * m;
  const int blocks = (items + 255) / 256;
  if (kind == 0)
    reduced_excitation_kernel<T><<<blocks, 256, 0, s>>>(n_el, n_basis, m, reinterpret_cast<const cpx<T>*>(in), qd,
                                                        reinterpret_cast<cpx<T>*>(out));
  else if (kind == 1)
    port_excitation_kernel<T><<<blocks, 256, 0, s>>>(n_el, m, port, reinterpret_cast<const cpx<T>*>(in), qd,
                                                     reinterpret_cast<cpx<T>*>(out));
  else
    port_currents_kernel<T><<<blocks, 256, 0, s>>>(n_el, m, port, reinterpret_cast<const cpx<T>*>(in), qd,
                                                   reinterpret_cast<cpx<T>*>(out));
  return cudaGetLastError();
}

template int lu_max_order<float>(int);
template int lu_max_order<double>(int);
template cudaError_t lu_factor<float>(cpx<float>*, int64_t, int, const LuWork&, cudaStream_t);
template cudaError_t lu_factor<double>(cpx<double>*, int64_t, int, const LuWork&, cudaStream_t);
template cudaError_t lu_solve<float>(const cpx<float>*, int64_t, int, const LuWork&, cpx<float>*, cpx<float>*,
                                     cudaStream_t);
template cudaError_t lu_solve<double>(const cpx<double>*, int64_t, int, const LuWork&, cpx<double>*, cpx<double>*,
                                      cudaStream_t);
template cudaError_t copy_matrix<float, double>(const void*, int64_t, int, void*, cudaStream_t);
template cudaError_t copy_matrix<float, float>(const void*, int64_t, int, void*, cudaStream_t);
template cudaError_t copy_matrix<double, double>(const void*, int64_t, int, void*, cudaStream_t);
template cudaError_t copy_vector<float, double>(const void*, int, void*, cudaStream_t);
template cudaError_t copy_vector<double, float>(const void*, int, void*, cudaStream_t);
template cudaError_t copy_vector<float, float>(const void*, int, void*, cudaStream_t);
template cudaError_t copy_vector<double, double>(const void*, int, void*, cudaStream_t);
template cudaError_t launch_excitation<float>(int, int, int, int, int, const void*, const double*, void*,
                                              cudaStream_t);
template cudaError_t launch_excitation<double>(int, int, int, int, int, const void*, const double*, void*,
                                               cudaStream_t);

}  // namespace cfft
