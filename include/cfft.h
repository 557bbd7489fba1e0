/*
 * cfft.h -- C ABI of the GB300 Contour-FFT (C-FFT) MBF reaction library.
 *
 * The library tabulates the substrate-related reaction terms between the
 * Macro Basis Functions (MBFs) of one printed element on a grounded slab for
 * all relative positions (Jha & Craeye, "Contour-FFT based spectral domain MBF
 * analysis of large printed antenna arrays", Section III), and fills the
 * reduced MoM matrix of an array of identical elements by interpolating that
 * table (Section III-B-1 and III-B-3).
 *
 * The problem statement it follows (Section III-B-1): once the table exists
 * for a given substrate and element, the reduced matrix of any array layout
 * follows by low-order interpolation at every element pair's relative
 * position (rho, phi).  Calls therefore follow the order
 *     set_substrate -> set_mbf_spectra* -> build_contour -> tabulate_reactions
 *     -> fill_reduced_matrix (any number of times, any layout)
 * and a call out of this order returns CFFT_ERR_STATE.
 *
 * Conventions for every entry point:
 *   - Lengths in any unit consistent with k0 (the tests use free-space
 *     wavelengths, k0 = 2 pi).  Spectral variables are in 1/length.
 *   - Time convention exp(+j omega t); the spectral kernel of Eq. 5 carries
 *     exp(-i k . Delta) with Delta = r_test - r_basis = rho (cos phi, sin phi).
 *   - Complex arrays are interleaved (re, im) pairs of the stated real type.
 *   - "host" pointers are read during the call only and never retained.
 *     "device" pointers must be CUDA device memory of the context's device;
 *     the library reads/writes them in stream order on the context stream and
 *     never frees them.  Buffers the library allocates itself (contour,
 *     spectra, scratch, table) are owned by the context and released by
 *     cfft_destroy.
 *   - Every call is stream-ordered on the context's stream; the calls that
 *     return results to the host (cfft_copy_table to host memory,
 *     cfft_synchronize, the NaN/Inf check in cfft_tabulate_reactions)
 *     synchronize that stream.
 *   - No C++ exception crosses this boundary.  On failure a call returns a
 *     non-zero cfft_status and cfft_last_error() describes it; the context
 *     stays usable unless the status is CFFT_ERR_CUDA from a sticky device
 *     error.
 *   - Threads: a context is not safe for concurrent calls (its buffers,
 *     scratch, error message and captured graph are shared); use one context
 *     per host thread, or serialise the calls.  Distinct contexts are
 *     independent, except that cfft_backproject_static shares one scratch
 *     array per device (see there).
 */
#ifndef CFFT_H
#define CFFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cfft_ctx cfft_ctx; /* opaque, library-owned */

typedef enum {
  CFFT_OK = 0,
  CFFT_ERR_ARG = 1,      /* invalid argument (null pointer, size, range) */
  CFFT_ERR_STATE = 2,    /* call out of order (e.g. tabulate before contour) */
  CFFT_ERR_OOM = 3,      /* device allocation failed */
  CFFT_ERR_CUDA = 4,     /* a CUDA runtime call failed */
  CFFT_ERR_NUMERIC = 5,  /* NaN or Inf in a produced table */
  CFFT_ERR_TIMEOUT = 6   /* a bounded device-side wait gave up */
} cfft_status;

typedef enum {
  CFFT_FP64 = 0,        /* all arithmetic in float64, table complex128 */
  CFFT_FP32_MIXED = 1   /* float32 spectra/FFT/back-projection, float64 contour,
                           Green's function denominators and branch-point
                           square roots; table complex64 */
} cfft_precision;

/* Tunables of the tabulation and the fill (cfft_set_option).  A value <= 0
 * restores the automatic choice, which depends on precision and element size,
 * except where an option below gives negative values a meaning of their own
 * (CHECK_FINITE, FILL_BLOCK, FILL_SIMT):
 *   N_ALPHA     angular samples for the azimuthal harmonics (multiple of 4)
 *   SIGMA       zero-padding factor of the beta FFT (power of two >= 2)
 *   BP_TAPS     taps of the back-projection interpolation: Lagrange one
 *               of 4, 6, 8, 10, 12, 16, 20, 24 (default 16 in FP64, 12 in
 *               FP32-mixed), ES 6 or 8 (default 6)
 *   FILL_TAPS   Lagrange taps of the fill interpolation in rho (even)
 *   ALPHA_MARGIN extra angular nodes of the back-projection quadrature
 *   CHECK_FINITE a value < 0 skips the NaN/Inf scan (and its stream sync)
 *                at the end of cfft_tabulate_reactions
 *   DERIVATIVES  a value > 0 makes cfft_tabulate_reactions also tabulate
 *                d Z_ab,q / d eps_r and d Z_ab,q / d h with the contour held
 *                fixed (three times the work; see cfft_get_derivative_table)
 *   BP_GATHER    a value > 0 selects the direct gather form of the
 *                back-projection instead of its matrix form (both evaluate
 *                the same quadrature; the matrix form needs at most 64 series
 *                per harmonic and 8, 12 or 16 taps)
 *   FILL_BLOCK   test elements per row block of the bucketed fill and of
 *                its adjoint (default 1024); a value < 0 selects the per-row
 *                kernels, which also serve the cases the bucketed forms do
 *                not cover (M other than 1, 2, 4; fill taps other than 8, 12,
 *                16; an output or gradient precision different from the
 *                table's)
 *   SPECTRA_SIMT a value > 0 evaluates the MBF spectra of the FP32-mixed
 *                tabulation with SIMT FP32 arithmetic instead of the tensor
 *                cores (which need a rooftop element, N_ALPHA = 128, M <= 4
 *                and the GEMM width limit of cfft_mbf_spectra)
 *   BP_SIMT      a value > 0 runs the FP32-mixed back-projection's matrix
 *                products on the FP32 pipe (paired-harmonic form) instead of
 *                the tensor cores (same quadrature; three TF32 products)
 *   FILL_SIMT    a value > 0 runs the FP32 fill of M = 4 with 8 taps and its
 *                adjoint on the FP32 pipe (bucketed form) instead of the
 *                tensor cores (the interpolation as one contraction per
 *                stencil cell); 0 (default): the fill on the tensor cores,
 *                the adjoint there from 512 element pairs per stencil cell;
 *                a value < 0: both on the tensor cores whenever they apply
 *   FILL_REFINE  grid of the table the fill interpolates.  Default (< 1):
 *                automatic, see cfft_fill_reduced_matrix; a value k >= 1
 *                fixes it at k times finer than the tabulated grid, without
 *                the accuracy check (k = 1: the tabulated table as it is)
 *   CONTOUR_SERIES  the series of the contour factor exp(beta_I s) that
 *                separates the transform into FFTs.  1: the Taylor series of
 *                Eq. 22 (term n: weight (beta_I/H)^n, coefficient
 *                (H s)^n / n!).  2: its Chebyshev series about the middle
 *                of the range of beta_I / H: exp(H s b) = exp(a) exp(a z),
 *                a = H s / 2, z = 2 b - 1, exp(a z) = I_0(a) + 2 sum_m
 *                I_m(a) T_m(z); the nodes beyond beta_p (b = 0) form one
 *                extra FFT with weight 1.  Default (<= 0): an explicit
 *                taylor_order keeps the Taylor series; the automatic order
 *                takes the series with fewer FFTs for the precision's
 *                remainder bound (Taylor on a tie)
 *   BP_KERNEL    interpolation kernel of the back-projection.  1: Lagrange
 *                polynomials on the transform grid g(s_k).  2: the ES
 *                kernel exp(beta (sqrt(1 - (2x/w)^2) - 1)) of width w = taps
 *                on the grid precorrected in the spectral domain (every
 *                contour sample divided by the kernel's Fourier transform at
 *                its frequency, so the "grid" debug buffer then holds the
 *                precorrected grid); FP32-mixed, matrix forms, 6 or 8 taps:
 *                6 ES taps reach the accuracy of 12 Lagrange taps at sigma 4
 *                (aliasing below 2e-6; 8 taps: 1e-8).  Default (<= 0): ES
 *                in FP32-mixed when the taps allow it, Lagrange otherwise;
 *                2 where ES cannot run is CFFT_ERR_ARG
 *   SOLVE_SIMT   a value > 0 runs the complex64 LU's trailing matrix
 *                products (cfft_solve_reduced) on the FP32 pipe instead of
 *                the tensor cores
 *   FFT_SUB_LEN  length L of the sub-FFTs of cfft_tabulate_reactions (the
 *                transform of length P = sigma n is split into P / L
 *                residue classes of its outputs, Eq. 23): a power of two in
 *                64..16384 (64..8192 in FP64) dividing P, else CFFT_ERR_ARG
 *                at the tabulation.  Default (<= 0): automatic
 *   SOLVE_GRID_PANEL  a value > 0 runs every LU panel of cfft_solve_reduced
 *                as a cooperative launch over the grid (pivot keys
 *                published and polled in global memory per column) instead
 *                of on one
 *                thread-block cluster for panels of at most 2048 rows */
typedef enum {
  CFFT_OPT_N_ALPHA = 0,
  CFFT_OPT_SIGMA = 1,
  CFFT_OPT_BP_TAPS = 2,
  CFFT_OPT_FILL_TAPS = 3,
  CFFT_OPT_ALPHA_MARGIN = 4,
  CFFT_OPT_CHECK_FINITE = 5,
  CFFT_OPT_DERIVATIVES = 6,
  CFFT_OPT_BP_GATHER = 7,
  CFFT_OPT_FILL_BLOCK = 8,
  CFFT_OPT_SPECTRA_SIMT = 9,
  CFFT_OPT_BP_SIMT = 10,
  CFFT_OPT_FILL_SIMT = 11,
  CFFT_OPT_FILL_REFINE = 12,
  CFFT_OPT_CONTOUR_SERIES = 13,
  CFFT_OPT_BP_KERNEL = 14,
  CFFT_OPT_SOLVE_SIMT = 15,
  CFFT_OPT_FFT_SUB_LEN = 16,
  CFFT_OPT_SOLVE_GRID_PANEL = 17
} cfft_option;

/* Create a context on CUDA device `device`, issuing all work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * context.  Errors: CFFT_ERR_ARG (out == NULL), CFFT_ERR_CUDA (bad device). */
cfft_status cfft_create(cfft_ctx** out, int device, void* cuda_stream);

/* Release every buffer the context owns.  NULL is ignored. */
void cfft_destroy(cfft_ctx* ctx);

/* Message of the last failing call on this context (never NULL). */
const char* cfft_last_error(const cfft_ctx* ctx);

/* Grounded dielectric slab (Section II, Eq. 2: the layered medium of Z^l):
 * relative permittivity eps_r > 0, thickness h >= 0, free-space wavenumber
 * k0 > 0.  Invalidates any contour and table. */
cfft_status cfft_set_substrate(cfft_ctx* ctx, double eps_r, double h, double k0);

/* Green's function of the tabulation (Sections II and III-A: the paper tabulates Z^l,
 * the layered-medium part from which an effective homogeneous medium and its image
 * through the ground plane have been extracted, and treats that extracted part, Z^h, in
 * the space domain).  extract = 0 (default): the full grounded-slab dyadic; extract = 1:
 * the slab dyadic minus the dyadic of a current sheet in a homogeneous medium of
 * permittivity eps_eff with the ground plane h below it (the matched line of the medium
 * in parallel with its shorted line: Z_TE = k0 Z0 (1 - e^{-2j kz h}) / (2 kz),
 * Z_TM = Z0 kz (1 - e^{-2j kz h}) / (2 k0 eps_eff), kz = -j sqrt(beta^2 - eps_eff k0^2)),
 * so that the tables, fills and the Cartesian tabulation hold Z^l.  eps_eff <= 0 takes
 * (eps_r + 1) / 2, which removes the slab's large-beta charge term; the substrate
 * derivatives then include d eps_eff / d eps_r = 1/2.  For eps_r = 1 the extracted part
 * is the whole slab (free space above a ground plane) and Z^l vanishes.  The space-domain
 * evaluation of Z^h (multipoles in the paper) is not part of this library.  Invalidates
 * the table.  CFFT_ERR_ARG for extract other than 0 or 1. */
cfft_status cfft_set_green_extraction(cfft_ctx* ctx, int extract, double eps_eff);

/* Element made of one x-directed cosine strip dipole of length `length` and
 * width `width` centred at the origin (one MBF, M = 1).  Its spectrum is
 * analytic (Section III-A).  Invalidates contour-independent caches. */
cfft_status cfft_set_mbf_spectra_strip(cfft_ctx* ctx, double length, double width);

/* Element made of n_basis rooftop basis functions combined into n_mbf MBFs
 * by the coefficient matrix Q (Eq. 3 and Eq. 11, M~ = sum_j q_j^* F~_j):
 *   centers  host, float64[2 * n_basis]: (x, y) of each rooftop centre,
 *            relative to the element centre
 *   dir      host, int32[n_basis]: 0 = x-directed, 1 = y-directed
 *   half_len host, float64[n_basis]: half-length a of the triangle
 *   width    host, float64[n_basis]: width w across the current
 *   q        host, float64[2 * n_basis * n_mbf]: complex Q, row-major
 *            [basis i][mbf a], interleaved (re, im)
 * Limits: 1 <= n_basis <= 4096, 1 <= n_mbf <= 8.
 * Errors: CFFT_ERR_ARG on null pointers or sizes out of range. */
cfft_status cfft_set_mbf_spectra(cfft_ctx* ctx, int n_basis, const double* centers,
                                 const int* dir, const double* half_len,
                                 const double* width, int n_mbf, const double* q);

/* Deformed contour of Eq. 8 (Fig. 1): n rectangle-rule samples (Eq. 23) at
 * beta_R = (j + 1/2) beta_max / n, j = 0..n-1, with the parabola
 * beta_I = 4 height beta_R (beta_p - beta_R) / beta_p^2 on [0, beta_p] and
 * the real axis beyond; weight (1 + i d beta_I / d beta_R) beta_max / n.
 * beta_max bounds the spectral integration (5 k_d in Section III-A);
 * beta_p must exceed every surface-wave pole (> k0 sqrt(eps_r)).
 * taylor_order is the highest power N_t kept in the Taylor expansion of the
 * contour factor (Eq. 22); -1 chooses the series (see CONTOUR_SERIES) and its
 * order from the precision's tolerance and the largest rho of the table at
 * tabulation time.
 * Accuracy: the samples enter the transform weighted by up to
 * exp(height * rho_max), so their rounding grows by that factor; for the
 * 1e-5 target of CFFT_FP32_MIXED keep height * rho_max <= 3 (and height a few
 * node spacings beta_max / n, so that the rectangle rule stays accurate next
 * to the poles).
 * Limits: 16 <= n <= 1048576; 0 < beta_p < beta_max; height >= 0;
 * -1 <= taylor_order <= 64.  Requires a substrate (else CFFT_ERR_STATE). */
cfft_status cfft_build_contour(cfft_ctx* ctx, int n, double beta_max, double beta_p,
                               double height, int taylor_order);

/* Override a tunable (see cfft_option; values <= 0 restore the automatic
 * choice unless the option says otherwise).  CFFT_ERR_ARG for an unknown key.
 * Takes effect at the next tabulation or fill. */
cfft_status cfft_set_option(cfft_ctx* ctx, cfft_option key, double value);

/* The series and order of the contour factor exp(beta_I s) that the automatic
 * choice of cfft_tabulate_reactions takes for x = height * rho_max (Eq. 22 and
 * its Chebyshev form, option CONTOUR_SERIES): the smallest order N whose
 * remainder bound, relative to the summed magnitudes of the transform's
 * inputs, is at most 1e-13 (CFFT_FP64) or 2^-22 (CFFT_FP32_MIXED); Taylor:
 * x^(N+1) / (N+1)! e^x, Chebyshev: e^a 2 sum_{m>N} I_m(a) with a = x / 2.
 * series_opt as the option CONTOUR_SERIES (<= 0: the series with fewer
 * transforms, Taylor on a tie; 1 Taylor; 2 Chebyshev).  Out: *series 0
 * Taylor, 1 Chebyshev; *order N; *n_ffts the transforms per (pair, harmonic,
 * residue class of the outputs): N + 1 for Taylor, N + 2 for Chebyshev (the
 * nodes beyond beta_p form one of them).  Host only: needs no context and no
 * device.  CFFT_ERR_ARG for x < 0 or not finite, a bad precision, a NULL
 * output, or no order up to 64 that reaches the bound. */
cfft_status cfft_contour_series_order(double x, cfft_precision precision, int series_opt, int* series,
                                      int* order, int* n_ffts);

/* Tabulate Z_ab,q(rho_r) for all MBF pairs (a, b), harmonics q = -q_max..q_max
 * and rho_r = r * rho_max / (n_rho - 1), r = 0..n_rho-1:
 *   Z'_ab(rho, phi) = sum_q Z_ab,q(rho) exp(i q phi)               (Eq. 9)
 * computed by the C-FFT: MBF spectra along the contour (Eq. 11), the kernel
 * H = M_t . G . M_b^* (Eq. 10), azimuthal harmonics, the Taylor expansion of
 * the contour factor (Eq. 22), one zero-padded FFT per (pair, harmonic,
 * Taylor term) (Eq. 23-24) and a back-projection over the angle to the
 * uniform rho grid.  The back-projection's midpoint rule in the angle takes,
 * for the rows of each chunk up to rho, ceil((z + q_max)/2 + c z^(1/3) +
 * margin/2) + 1 nodes with z = |beta_c|max rho, margin = ALPHA_MARGIN (24)
 * and c = 4 in FP64, 2 in FP32-mixed: the first aliased angular harmonic
 * then lies far enough beyond z that its Bessel factor is below the
 * precision's target at every rho.
 * rotation_classes = 1: elements unrotated (one class);
 * rotation_classes = 4: element rotations in {0, 90 deg}; the table holds the
 * classes (test, basis) = (0,0), (0,90), (90,0), (90,90) in that order.
 * Limits: 0 <= q_max <= 64; 2 <= n_rho <= 1048576; rho_max > 0.
 * Errors: CFFT_ERR_STATE (no substrate/element/contour), CFFT_ERR_ARG (also
 * when taylor_order is -1 and no order up to 64 meets the precision's
 * tolerance: height * rho_max beyond about 13 in FP64, 16 in FP32-mixed),
 * CFFT_ERR_OOM, CFFT_ERR_NUMERIC (NaN/Inf produced). */
cfft_status cfft_tabulate_reactions(cfft_ctx* ctx, int q_max, double rho_max, int n_rho,
                                    cfft_precision precision, int rotation_classes);

/* Borrow the table: *dev_ptr = device address (owned by ctx, valid until the
 * next tabulate or destroy), shape = {classes, M*M, 2*q_max+1, n_rho}, row-
 * major with pair index a*M + b, element type complex128 (precision FP64) or
 * complex64 (FP32_MIXED) as *is_complex128 says.  CFFT_ERR_STATE if no table. */
cfft_status cfft_get_table(const cfft_ctx* ctx, const void** dev_ptr, int64_t shape[4],
                           int* is_complex128);

/* Copy the table into caller memory `dst` (bytes must equal the table size);
 * dst_is_host != 0: dst is host memory and the call synchronizes the stream;
 * dst_is_host == 0: dst is device memory (stream-ordered copy). */
cfft_status cfft_copy_table(const cfft_ctx* ctx, void* dst, int64_t bytes, int dst_is_host);

/* Fill the dense reduced matrix of n_elements identical elements (Eq. 3 per
 * block, Eq. 9 per entry, interpolated in the table; Section III-B-3):
 *   Z_out[(m*M + a) * ld + n*M + b] = sum_q exp(i q phi_mn) Z^{cls}_ab,q(rho_mn)
 * with (rho_mn, phi_mn) the polar form of r_m - r_n (m = test element,
 * n = basis element) and cls the rotation class of (rot[m], rot[n]).  The
 * diagonal blocks (m = n) take the table at rho = 0.
 *   pos_xy  device, float64[2 * n_elements]: element centres (x, y)
 *   rot     device, int32[n_elements]: 0 or 1 (0 or 90 deg); may be NULL when
 *           the table has one class (all elements unrotated)
 *   z_out   device, caller-owned: complex128 (out_complex128 != 0) or
 *           complex64, at least n_elements*M rows of ld entries
 *   ld      row stride in complex entries, >= n_elements * M
 * Requires a table (CFFT_ERR_STATE).  A pair farther apart than the table's
 * rho_max makes the call return CFFT_ERR_ARG (after the kernel ran; the
 * affected entries are zero).  Stream-ordered; synchronizes for that check.
 * The element pairs of each block of test elements are counting-sorted by
 * (rotation class, stencil row) before the interpolation, so that pairs that
 * share table rows run together on one copy of those rows in shared memory;
 * the context owns that scratch (4 bytes per element pair of up to 2^27 pairs
 * at a time, 8 bytes per (row block, class, table row), 16 bytes per element)
 * and keeps it for the next fill.
 * Accuracy: the fill's interpolation keeps within a quarter of the table
 * precision's target (1e-10 of the table maximum per (class, pair) for FP64,
 * 1e-5 for FP32-mixed) at every distance up to rho_max.  The first fill or
 * adjoint after a tabulation estimates the interpolation error on the
 * tabulated rho grid from the table's p-th differences (the Lagrange
 * remainder; p = fill taps), for the interior stencils and for the stencil
 * shifted inward at rho_max.  When the estimate misses that share, the
 * context tabulates the same reactions once more, with the options in force
 * at the tabulation, on a grid finer by an integer factor r >= 1 that
 * reaches p/2 rows beyond rho_max (so that every stencil is centred), and
 * the fill and its adjoint interpolate that table from then on;
 * cfft_get_table keeps returning the tabulated grid.  cfft_get_info reports
 * the estimate, r and the grid used (fill_err_est, fill_refine,
 * fill_n_rho).  A loaded table (cfft_load_table) cannot be tabulated again:
 * when its grid misses the share the fill returns CFFT_ERR_ARG
 * (CFFT_OPT_FILL_REFINE set to 1 accepts the grid as it is). */
cfft_status cfft_fill_reduced_matrix(cfft_ctx* ctx, int n_elements, const double* pos_xy,
                                     const int* rot, void* z_out, int64_t ld,
                                     int out_complex128);

/* Same as cfft_fill_reduced_matrix with HOST arrays: pos_xy, rot and z_out
 * are host memory; the call copies them to and from the device through
 * context-owned buffers and synchronizes. */
cfft_status cfft_fill_reduced_matrix_host(cfft_ctx* ctx, int n_elements, const double* pos_xy,
                                          const int* rot, void* z_out, int64_t ld,
                                          int out_complex128);

/* One item of a batched sweep: substrate (eps_r, h), free-space wavenumber k0
 * (the frequency, with lengths in fixed units) and its own contour (n samples,
 * beta_max, beta_p, height as in cfft_build_contour; taylor_order -1 = auto). */
typedef struct {
  double eps_r, h, k0;
  int n;
  double beta_max, beta_p, height;
  int taylor_order;
} cfft_batch_item;

/* Batched sweep (the paper fixes one substrate and frequency; sweeping many is
 * the same Section III-B tabulation repeated): tabulate the element set by
 * cfft_set_mbf_spectra for n_items (substrate, frequency, contour) items with
 * uneven contour lengths, one rotation class, harmonics -q_max..q_max and
 * n_rho points to rho_max, into
 *   tables  device, caller-owned: n_items consecutive tables of
 *           M*M * (2*q_max+1) * n_rho entries (layout of cfft_get_table),
 *           complex128 (precision FP64) or complex64.
 * Every stage runs as one launch over all items of a wave (items are split
 * into waves only when their scratch would exceed 24 GiB): contour and
 * integrand as multi-item grids, the FFTs and the back-projection as
 * persistent kernels that pull (item, series, residue) and (item, group,
 * harmonic, row chunk) tasks from a counter, largest first.
 * flags bit 0: capture the launch sequence into a CUDA graph on the first
 *              call with a given structure (items' n and Taylor orders,
 *              sizes, output buffer) and replay it on later calls, which only
 *              refresh the per-item parameters.  A call whose plan moved
 *              anything the graph holds by value (grid widths and angular
 *              node counts that follow the contours, launch shapes, the
 *              library's buffer addresses) captures again instead of
 *              replaying.  The batch runs on a
 *              library-owned stream ordered after the context's stream, so
 *              any context stream (also the legacy default one) works.
 * flags bit 1: autotune the sub-FFT length, and in FP32-mixed whether the
 *              back-projection's products run on the tensor cores or the
 *              FP32 pipe, by timing the candidates on this batch (cached per
 *              structure).
 * Each n must be a multiple of 256 (sigma * n divisible by 1024).  Requires
 * cfft_set_mbf_spectra* (CFFT_ERR_STATE).  Synchronizes. */
cfft_status cfft_tabulate_batch(cfft_ctx* ctx, int n_items, const cfft_batch_item* items,
                                int q_max, double rho_max, int n_rho, cfft_precision precision,
                                void* tables, int flags);

/* Diagnostics of the last batch: stage times of the first wave (contour +
 * integrand, FFT, back-projection), the whole graph replay, work counts,
 * chosen sub-FFT length and row chunk, waves, kernel launches, bp_tc = 1
 * when the back-projection's products ran on the tensor cores, and the number
 * of graph captures the context has made (a replayed call leaves it unchanged). */
typedef struct {
  double ms_integrand, ms_fft, ms_backproject, ms_graph;
  double work_subffts, work_bp_nodes;
  int sub_len, rchunk, waves, launches, bp_tc, captures;
} cfft_batch_info;
cfft_status cfft_get_batch_info(const cfft_ctx* ctx, cfft_batch_info* info);

/* Substrate derivatives of the table (forward mode; no counterpart in the
 * paper, which fixes the substrate).  The table is linear in the Green's
 * function, G = P(beta) I - R(beta) k k^T, so d Z / d theta is the same C-FFT
 * applied to dP/dtheta and dR/dtheta (analytic derivatives of the TE/TM
 * expressions, float64) with the contour, Taylor order and grids unchanged.
 * which = 0: the table itself; 1: d/d eps_r; 2: d/d h.  Same layout and
 * element type as cfft_get_table; borrowed.  For which = 1 or 2 the call
 * returns CFFT_ERR_STATE unless the last tabulation ran with
 * CFFT_OPT_DERIVATIVES > 0. */
cfft_status cfft_get_derivative_table(const cfft_ctx* ctx, int which, const void** dev_ptr,
                                      int64_t shape[4]);

/* Adjoint of cfft_fill_reduced_matrix (no counterpart in the paper): given
 * grad_z = dL/dZ' of a real objective L in the convention
 * dL = Re sum_ij conj(grad_z_ij) dZ'_ij (the one PyTorch uses for complex
 * tensors), write
 *   grad_pos[2m + {0,1}] = dL / d(x_m, y_m)      (device float64[2 * n_elements])
 *   grad_eps_h[{0,1}]    = dL / d(eps_r, h)      (device float64[2], optional)
 * through the interpolated table: d rho and d phi of every element pair
 * (the Lagrange stencil's slope and i q exp(i q phi)), and the derivative
 * tables for the substrate (requires CFFT_OPT_DERIVATIVES at tabulation,
 * else CFFT_ERR_STATE when grad_eps_h is not NULL).  grad_z: device,
 * complex128 (grad_complex128 != 0) or complex64, rows of ld entries, layout
 * of Z_out.  Outputs are overwritten.  Pairs are bucketed as in the fill
 * (the fill's scratch is reused); a pair's contribution is formed in the
 * table precision and accumulated with float64 atomics (results can differ in
 * the last bits from run to run).  Synchronizes the stream. */
cfft_status cfft_fill_backward(cfft_ctx* ctx, int n_elements, const double* pos_xy,
                               const int* rot, const void* grad_z, int64_t ld,
                               int grad_complex128, double* grad_pos, double* grad_eps_h);

/* The same adjoint for the array objective L = sum_i |(Z' v - t)_i|^2 (no
 * counterpart in the paper): given the excitation v and the residual
 * r = Z' v - t (device, A*M entries each, complex128 when complex128 != 0,
 * else complex64), dL/dZ' = 2 r v^H is formed in context-owned scratch
 * ((A*M)^2 entries, kept for the next call) and cfft_fill_backward runs on it;
 * outputs and errors as there (CFFT_ERR_OOM when the scratch does not fit). */
cfft_status cfft_fill_backward_residual(cfft_ctx* ctx, int n_elements, const double* pos_xy,
                                        const int* rot, const void* v, const void* resid,
                                        int complex128, double* grad_pos, double* grad_eps_h);

/* Diagnostics of the last tabulation (host values): highest term index of
 * the contour-factor series used (taylor_order; contour_series 0: Taylor,
 * 1: Chebyshev; the FFTs per (pair, harmonic) are taylor_order + 1, or + 2
 * for Chebyshev),
 * n_alpha, sigma, FFT length, sub-FFT length, grid half-width K, back-
 * projection taps, fill taps, series count, the device time of each stage in
 * milliseconds (contour, integrand, fft, backproject; CUDA events on the
 * context stream), the number of kernels launched, and the work of each
 * stage: integrand points (nodes x angles), sub-FFTs run (each of length
 * sub_len), and back-projection node evaluations (series x rows x angles).
 * spectra_tc: 1 when the MBF spectra ran on the tensor cores; bp_form: 0 the
 * gather form of the back-projection, 1 the matrix form, 2 the paired-
 * harmonic matrix form, 3 the paired-harmonic form with its products on the
 * tensor cores; for the matrix forms work_bp_macs counts the complex
 * multiply-adds of the interpolation-matrix products (rows x grid columns x
 * series, every harmonic) and work_bp_stencils the node stencils added into
 * the matrices (rows x angular nodes x matrices).  fill_form: the form of the
 * last cfft_fill_reduced_matrix: 1 per-row, 2 bucketed on the FP32 pipe, 3 on
 * the tensor cores (0: no fill yet).  fill_err_est: the estimated
 * interpolation error of the fill on the tabulated grid, relative to the
 * table maximum (-1: not estimated); fill_refine: the factor r of the grid
 * the fill interpolates (0: no fill since the last tabulation); fill_n_rho:
 * that grid's points (n_rho when the fill uses the tabulated table, else
 * (n_rho - 1) r + 1 + fill_taps / 2, reaching beyond rho_max).
 * bp_kernel: the back-projection's interpolation kernel (0 Lagrange, 1 ES).
 * tc_flops_integrand, tc_flops_backproject: the tensor-core flops the
 * integrand's spectra GEMM and the back-projection's products executed in the
 * tabulation (three TF32 products per term, padding included; 0 when that
 * stage ran on the FP32 pipe). */
typedef struct {
  int taylor_order, n_alpha, sigma, fft_len, sub_len, grid_half, bp_taps, fill_taps;
  int series, classes, n_pairs, n_harm;
  double delta_s, ms_contour, ms_integrand, ms_fft, ms_backproject;
  int launches, n_basis;
  double work_points, work_subffts, work_bp_nodes;
  int spectra_tc, bp_form;
  double work_bp_macs, work_bp_stencils;
  int fill_form;
  double fill_err_est;
  int fill_refine, fill_n_rho;
  double tc_flops_integrand, tc_flops_backproject;
  int contour_series, bp_kernel;
} cfft_info;
cfft_status cfft_get_info(const cfft_ctx* ctx, cfft_info* info);

/* Device address of an intermediate buffer of the last tabulation, for
 * stage-by-stage verification:
 *   "harmonics": the contour integrand H_ab,q(beta_j) beta_c,j w_j,
 *                shape {computed classes, M*M, 2*q_max+1, n}
 *   "grid":      the series-summed transform on s_k = k delta_s, k = -K..K,
 *                demodulated: g_ab,q(s_k) exp(i beta_max s_k / 2) (with the
 *                ES kernel: of the precorrected samples, see BP_KERNEL),
 *                shape {computed classes, M*M, 2*q_max+1, 2K+1}
 *   "contour":   the nodes beta_c,j (complex128), shape {1, n, 1, 1}
 * "computed classes" is 1, or 3 with four rotation classes (the (90, 90)
 * class is derived from (0, 0)).  Element type as the table's except
 * "contour".  Borrowed; valid until the next tabulate. */
cfft_status cfft_debug_buffer(const cfft_ctx* ctx, const char* name, const void** dev_ptr,
                              int64_t shape[4]);

/* Wait for all work issued on the context stream. */
cfft_status cfft_synchronize(cfft_ctx* ctx);

/* Allocation-free back-projection.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- plug-ins whose host
 * application owns every device allocation, real-time loops that cannot
 * afford an allocation that may synchronize the device.  It runs the
 * back-projection stage of
 * cfft_tabulate_reactions on caller-owned buffers and allocates nothing:
 * its scratch (angular node counts, offsets and cosines for every chunk of
 * 32 rho rows) lives in one 8 MiB device array inside the library, present
 * on every GPU that loads the library until the process exits.
 *   grid    device, input: [series][2*grid_half+1] with series =
 *           g * (2*q_max+1) + (q + q_max), g < series_per_q -- the layout of
 *           cfft_debug_buffer("grid"): the transform in beta on s_k =
 *           k * delta_s, k = -grid_half..grid_half, demodulated by
 *           exp(i pi k / sigma), as the FFT stage writes it
 *   table   device, output: [series][n_rho], rho_r = r * rho_max / (n_rho-1)
 *   complex128 != 0: both buffers complex128, else complex64
 *   sigma, taps, delta_s, grid_half: the transform grid's zero padding,
 *           Lagrange taps (4, 6, 8, 10, 12, 16, 20 or 24), step and half-width
 *           (cfft_get_info reports them for a tabulation); beta_abs_max is
 *           |beta_c| at the end of the contour, alpha_margin the angular node
 *           margin (24 is the default of cfft_tabulate_reactions; the node
 *           rule's cube-root term follows the element type as there).  The
 *           angular node counts are computed on the device here and on the
 *           host in the tabulation, so the result matches the tabulation's
 *           table within its precision's tolerance, not bit for bit
 * Limits: at most 65536 chunks (n_rho <= 2097152) and at most 950,272
 * angular nodes summed over the chunks (about n_rho * beta_abs_max * rho_max
 * / 128; 8192 rows to rho 50 at beta 66 use about 2.1e5); a request beyond
 * them, or whose rho_max needs more grid than grid_half, returns
 * CFFT_ERR_ARG before any work is queued.
 * The first call on a device looks the scratch array's device address up
 * (with `device` made current for the call).  Every call reuses the same array and rewrites the
 * entries it reads before reading them, so no call depends on what an
 * earlier one left there -- but two calls whose work overlaps on the GPU
 * (different streams, no ordering between them) race on the array.
 * Work is queued on cuda_stream; the call does not synchronize. */
cfft_status cfft_backproject_static(int device, void* cuda_stream, const void* grid,
                                    void* table, int series_per_q, int q_max, int n_rho,
                                    double rho_max, int grid_half, double delta_s, int sigma,
                                    int taps, double beta_abs_max, double alpha_margin,
                                    int complex128);

/* MBF spectra (Eq. 11) of the element set by cfft_set_mbf_spectra at n_points
 * complex wavevectors, as a complex GEMM on the tensor cores:
 *   out[p][0][a][d] = M_a,d(k_p)    = sum_i conj(Q_ia) F_i(k_p) d_i
 *   out[p][1][a][d] = Mbar_a,d(k_p) = sum_i Q_ia F_i(-k_p) d_i
 * (d = x, y: the basis directions; the second side is the analytic
 * continuation of the conjugated basis spectrum of Eq. 10).
 *   k    device, complex64 [n_points][2]: (kx, ky), any complex values
 *   out  device, complex64 [n_points][2][M][2], caller-owned
 * Arithmetic: FP32 operands split into TF32 head + tail, three tensor-core
 * products per term, FP32 accumulation (float32 accuracy).  Applies to
 * rooftop elements with 2 * classes * max(2 M, 8) <= 64, where classes counts
 * the distinct (direction, half-length, width) rooftop shapes: CFFT_ERR_ARG
 * otherwise, CFFT_ERR_STATE without an element.  A tensor-core wait that
 * runs past its bound returns CFFT_ERR_TIMEOUT.  Stream-ordered on the
 * context stream; synchronizes to read the error flag. */
cfft_status cfft_mbf_spectra(cfft_ctx* ctx, int n_points, const void* k, void* out);

/* Failure-detection self-test (no counterpart in the paper).  One device
 * thread waits, with at most `polls` tries (1 .. 2^20), on an mbarrier phase
 * that nothing completes -- the bounded wait every tensor-core kernel uses
 * for its asynchronous products -- and records that it gave up.  Returns
 * CFFT_ERR_TIMEOUT (the designed outcome; the context stays usable),
 * CFFT_ERR_ARG for a bad bound, CFFT_ERR_CUDA on a launch failure.  No
 * trap, fault or unbounded wait is involved.  Synchronizes the stream. */
cfft_status cfft_selftest_bounded_wait(cfft_ctx* ctx, unsigned polls);

/* Failure-injection hook for tests (host side only; no device fault): the next
 * `after` device allocations the library makes succeed and the one after them
 * fails as if the device were out of memory -- no allocation is attempted, the
 * call in progress returns CFFT_ERR_OOM, and the hook disarms itself.
 * after < 0 disarms it.  Process-wide, for single-threaded tests only.  The
 * context stays usable: a later call allocates what it needs again. */
void cfft_test_fail_allocation(int after);

/* Reduced excitation of an array of identical elements (Section II, Eq. 4):
 *   v_red[m M + a] = sum_i conj(Q_ia) v[m][i]
 * for every element m and MBF a, with Q the coefficient matrix given to
 * cfft_set_mbf_spectra (basis functions in the caller's order; the strip
 * element has Q = [1]).  The order m M + a is the row order of the reduced
 * matrix Z' of cfft_fill_reduced_matrix.
 *   v      device, [n_elements][n_basis] elementary excitation vectors
 *   v_red  device, [n_elements * M]
 * complex128 != 0: both complex128, else complex64 (accumulated in float64).
 * CFFT_ERR_STATE without an element.  Synchronizes the context stream. */
cfft_status cfft_reduced_excitation(cfft_ctx* ctx, int n_elements, const void* v, void* v_red,
                                    int complex128);

/* Delta-gap ports (Section IV: the arrays are excited at a port of each
 * element): a voltage amplitudes[m] across basis function `port` of element m,
 * V_m = amplitudes[m] e_port, so v_red[m M + a] = amplitudes[m] conj(Q_port,a).
 *   amplitudes  device, [n_elements]; v_red device, [n_elements * M]
 * CFFT_ERR_ARG for a port outside 0..n_basis-1.  Synchronizes. */
cfft_status cfft_port_excitation(cfft_ctx* ctx, int n_elements, int port, const void* amplitudes,
                                 void* v_red, int complex128);

/* Port currents from the reduced solution: the current of element m on its port
 * basis function, (Q I'_m)[port] = sum_a Q_port,a i_red[m M + a] (the elementary
 * currents of Section II are I_m = Q I'_m).
 *   i_red  device, [n_elements * M]; i_port device, [n_elements]
 * Synchronizes. */
cfft_status cfft_port_currents(cfft_ctx* ctx, int n_elements, int port, const void* i_red,
                               void* i_port, int complex128);

/* Direct solution of the reduced system Z' I' = V' (Section II: the MBF
 * reduction makes the system small enough to solve directly; Table II,
 * "Solving time").  z: device, n rows of ld >= n entries, row-major as
 * cfft_fill_reduced_matrix writes it; not modified (the context factors a copy
 * of n x n entries, kept until the next solve or destroy).  v: device, [n]
 * right-hand side; i_out: device, [n] solution.  Element types: complex128
 * when complex128 != 0, else complex64.  n is at most the order whose panel
 * rows fit the panel CTAs' shared memory (48,640 in complex64 and 24,320 in
 * complex128 on 152 SMs) and at most 65535; beyond, CFFT_ERR_ARG.
 * mode 0: LU with partial pivoting (|re| + |im| of the column, compared on
 *         the leading 32 bits of its double, ties to the lowest row) in the
 *         matrix's own precision.
 * mode 1 (complex128 only): the LU of a complex64 copy, then iterative
 *         refinement in float64 against z: x += LU^-1 (v - z x) until the
 *         correction falls below float64 resolution or the residual stops
 *         falling (at most 30 steps).
 * The factorization runs in panels of 64 columns: one launch per panel (pivot
 * search and elimination, one barrier per column: the hardware barrier of one
 * thread-block cluster of 16 or 8 CTAs, candidates and pivot rows read from
 * the peers' shared memory, for panels of at most 2048 rows that fit that
 * cluster's shared memory; otherwise a cooperative launch over the grid whose
 * CTAs publish their candidates' pivot keys, tagged with the column, in
 * global memory and poll them with a bound), the panel's row moves applied to
 * the whole matrix, a
 * triangular solve for
 * the panel's rows and a complex matrix product for the trailing matrix.  In
 * complex64 that product runs on the tensor cores (three TF32 products, FP32
 * accumulation) unless the option SOLVE_SIMT is > 0, which keeps it on the
 * FP32 pipe.
 * cfft_get_solve_info reports the times and the relative residual
 * |v - z x| / |v| computed in float64 from z.  Errors: CFFT_ERR_ARG,
 * CFFT_ERR_OOM, CFFT_ERR_NUMERIC (a zero pivot: z singular), CFFT_ERR_TIMEOUT
 * (a grid-barrier or tensor-core wait gave up).  Synchronizes. */
cfft_status cfft_solve_reduced(cfft_ctx* ctx, int n, const void* z, int64_t ld, const void* v,
                               void* i_out, int complex128, int mode);

/* Diagnostics of the last cfft_solve_reduced: factorization and solve times
 * (ms, CUDA events on the context stream; the solve includes refinement),
 * relative residual, order n, mode, refinement steps (mode 1), panel width,
 * update_tc = 1 when the trailing updates ran on the tensor cores, the number
 * of panels that ran on one thread-block cluster and its CTA count (0: none). */
typedef struct {
  double ms_factor, ms_solve, residual;
  int n, mode, refinements, panel_width, update_tc, cluster_panels, panel_cluster;
} cfft_solve_info;
cfft_status cfft_get_solve_info(const cfft_ctx* ctx, cfft_solve_info* info);

/* The paper's own 2-D Cartesian C-FFT (Section III-B-2 and III-B-3, Eq. 21-24,
 * Appendix I), beside the harmonic tabulation.  On the real grid
 * kx, ky = -beta_max + n dk (n < n_grid, dk = 2 beta_max / n_grid) the contour of
 * cfft_build_contour enters through the extension k (1 + i gamma), gamma =
 * beta_I(|k|) / |k| (Eq. 20), with the Jacobian (1 + i d beta_I/d beta_R)
 * (1 + i gamma) (Eq. 21); samples outside |k| <= beta_max are zero (the polar
 * integral's limit).  The contour factor exp(gamma k.Delta) is expanded in
 * Taylor monomials (Eq. 22), each an FFT2 with the signs of Appendix I, the
 * spectrum zero-padded to twice the size (the Whittaker-Shannon refinement at
 * the end of Section III-B-3).  The table holds, for every MBF pair (a, b),
 *   Z'_ab(x0 + i step, x0 + j step),  i, j < 2 n_grid,
 *   x0 = -n_grid pi / (2 beta_max), step = pi / (2 beta_max)
 * (row-major [pair a*M+b][i: dx][j: dy]; complex128 for CFFT_FP64, else
 * complex64).  rho_max: the largest element distance the fill will ask for;
 * it must lie inside the table by two steps (else CFFT_ERR_ARG: raise
 * n_grid), and sets the automatic Taylor order (taylor_order = -1: from
 * height * rho_max as for cfft_tabulate_reactions; a fixed order 0..40
 * otherwise).  n_grid: a power of two in 16..2048.  The slope of the contour
 * is discontinuous on the circle |k| = beta_p and the integrand is cut on
 * |k| = beta_max; no Cartesian grid follows either, so the rectangle rule is
 * first to second order in dk there (the harmonic tabulation integrates the
 * same contour along beta to spectral accuracy).  One rotation class
 * (unrotated elements).  Requires substrate, element and contour
 * (CFFT_ERR_STATE).  Synchronizes. */
cfft_status cfft_tabulate_cartesian(cfft_ctx* ctx, int n_grid, double rho_max, int taylor_order,
                                    cfft_precision precision);

/* Description of the Cartesian table: grid size, table size (2 n_grid), Taylor
 * order, number of monomials (FFT2s per pair), element type, lattice origin
 * and step, rho_max, and the device time of the tabulation in ms. */
typedef struct {
  int n_grid, n_table, taylor_order, monomials, complex128;
  double x0, step, rho_max, ms;
} cfft_cartesian_info;
/* Borrow the Cartesian table (device, context-owned, valid until the next
 * Cartesian tabulation or destroy) and its description.  CFFT_ERR_STATE if
 * none. */
cfft_status cfft_get_cartesian_table(const cfft_ctx* ctx, const void** dev_ptr, cfft_cartesian_info* info);

/* Reduced matrix of unrotated elements from the Cartesian table by second-order
 * (three-point) Lagrange interpolation in dx and dy around the nearest lattice
 * node (the end of Section III-B-3):
 *   Z_out[(m M + a) ld + n M + b] = Z'_ab(r_m - r_n)
 * pos_xy, z_out, ld, out_complex128 as in cfft_fill_reduced_matrix.  A pair
 * farther apart than the table's rho_max returns CFFT_ERR_ARG (its entries
 * zero).  Synchronizes. */
cfft_status cfft_fill_cartesian(cfft_ctx* ctx, int n_elements, const double* pos_xy, void* z_out,
                                int64_t ld, int out_complex128);

/* Arithmetic peak microbenchmark (no counterpart in the paper; the roofline
 * fractions of the measurement divide by its results).  which:
 *   0  FP32 FMA pipe: independent fused multiply-add chains on every SM
 *      (2 flops per FMA)
 *   1  FP64 FMA pipe: the same in float64
 *   2  tensor cores, tcgen05.mma kind::tf32: M 128 x N 256 x K 8 products from
 *      shared memory into fp32 accumulators in tensor memory, one CTA per SM
 *   3  tensor cores, kind::f16 with bf16 operands (K 16), the same shape
 * One untimed launch, then `reps` (1..100) launches timed with CUDA events on
 * a stream of the call's own; *tflops = flops of a launch / the shortest
 * launch time, *best_ms = that time (may be NULL).  Allocates and frees a
 * small output buffer; synchronizes its stream.  Errors: CFFT_ERR_ARG (bad
 * which, reps, device or pointer), CFFT_ERR_CUDA, CFFT_ERR_TIMEOUT (a bounded
 * tensor-core wait gave up). */
cfft_status cfft_measure_peak(int device, int which, int reps, double* tflops, double* best_ms);

/* Checkpoint / resume of a table (the paper's tables are reusable across array
 * layouts for a fixed substrate and element, Section IV-F): installs a table
 * saved from cfft_copy_table (layout [class][pair][q][r] of cfft_get_table,
 * complex128 for CFFT_FP64, complex64 otherwise) with its description: MBF
 * count (1..8), harmonics |q| <= q_max (0..64), n_rho points (at most 2^20)
 * on [0, rho_max] (rho_max finite, > 0), rotation classes (1 or 4), fill taps
 * (even, 2..16, n_rho >= 2 taps).  Afterwards the fill and
 * its position adjoint run without a tabulation (the substrate adjoint needs
 * the derivative tables of a tabulation).  table: host (src_is_host != 0) or
 * device memory, copied; the context keeps no reference.  CFFT_ERR_ARG for a
 * bad description or an MBF count that differs from the context's element. */
cfft_status cfft_load_table(cfft_ctx* ctx, int n_mbf, int q_max, double rho_max, int n_rho,
                            cfft_precision precision, int rotation_classes, int fill_taps,
                            const void* table, int src_is_host);

#ifdef __cplusplus
}
#endif

#endif /* CFFT_H */
