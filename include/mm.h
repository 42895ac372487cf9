/*
 * libmm -- GLS map-making on one GB300 (sm_103a).
 *
 * Solves (P^T N^-1 P) m = P^T N^-1 d by preconditioned conjugate gradients, after
 * Szydlarski, Grigori & Stompor, "Accelerating the cosmic microwave background
 * map-making procedure through preconditioning" (arXiv 1408.3048):
 *   P      pointing matrix, Eq. 1-2 (one pixel per sample; I/Q/U weights
 *          (1, cos 2phi, sin 2phi) for a polarisation-sensitive detector)
 *   N^-1   block-diagonal, one banded symmetric Toeplitz block per stationary
 *          interval, Eq. 4 and Sec. 4.1.4; rows from the noise PSD of Eq. 19 apodised
 *          by the window of Eq. 28 (App. D)
 *   A      = P^T N^-1 P (Eq. 5), applied matrix-free as in Eq. 8
 *   M_BD   block-Jacobi preconditioner, Eq. 10
 *   M_2lvl two-level preconditioner, Eq. 12, with the a posteriori coarse space of
 *          Sec. 3.3.2 (Ritz vectors of M_BD A) and the application order of App. C
 *
 * Conventions (every entry point):
 *   - A plan owns all of its device buffers; it never frees caller memory.
 *   - "device" pointers are CUDA device (or managed) memory of the current device;
 *     "host" pointers are ordinary host memory.  Where an argument says
 *     "host or device", the library inspects the pointer and copies as needed.
 *   - Maps are observed-pixel ordered (ascending sky index), pixel-major, with the
 *     ncomp Stokes components of one pixel adjacent: x[q*ncomp + c]  (n = npix_obs*ncomp).
 *   - Time-domain vectors are in sample order, length nt.
 *   - Work is issued on opts->stream; calls return after that work completes.
 *   - On error a call returns a non-zero mm_status and mm_last_error() describes it;
 *     output buffers are then unspecified.  The plan stays usable unless the status is
 *     MM_ERR_CUDA or MM_ERR_TIMEOUT.
 *   - Not thread-safe per plan: one call at a time on a given plan.
 */
#ifndef MM_H
#define MM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mm_plan_s* mm_plan_t;

typedef enum {
    MM_OK = 0,
    MM_ERR_ARG = 1,            /* invalid argument (sizes, offsets, pixel range, lambda) */
    MM_ERR_CUDA = 2,           /* a CUDA runtime call failed                              */
    MM_ERR_OOM = 3,            /* device allocation failed                                */
    MM_ERR_NOT_SPD = 4,        /* Toeplitz symbol <= 0, p^T A p <= 0 or E not SPD         */
    MM_ERR_NOT_CONVERGED = 5,  /* maxit reached; the best iterate is returned             */
    MM_ERR_NUMERIC = 6,        /* NaN/Inf met in a reduction                              */
    MM_ERR_TIMEOUT = 7,        /* a bounded device-side wait ran out                      */
    MM_ERR_STATE = 8           /* call needs state that is not built (e.g. coarse space)  */
} mm_status;

enum { MM_FP64 = 0, MM_FP32 = 1 };                 /* operator arithmetic               */
enum { MM_WINDOW_GAUSS = 0, MM_WINDOW_RECT = 1 };  /* apodisation window (Eq. 28 / none) */
enum { MM_PREC_BD = 0, MM_PREC_TWOLEVEL = 1, MM_PREC_ADEF2 = 2 };  /* preconditioner kind */
enum { MM_SOLVE_FP64 = 0, MM_SOLVE_MIXED = 1 };    /* solver arithmetic                 */

/* Noise PSD of one stationary piece, Eq. 19 with exponent alpha:
 * P(f) = sigma^2 t_samp (1 + (fknee/f)^alpha). */
typedef struct {
    double sigma;
    double fknee;
    double alpha;
} mm_psd;

typedef struct {
    int32_t ncomp;          /* 1 (temperature) or 3 (I, Q, U)                             */
    int32_t lambda;         /* Toeplitz half bandwidth: lags |k| <= lambda are kept       */
    int32_t window;         /* MM_WINDOW_GAUSS (default) or MM_WINDOW_RECT                */
    int32_t fft_log2_f64;   /* 0: automatic; else overlap-save block 2^v for FP64 (9..16) */
    int32_t fft_log2_f32;   /* 0: automatic; else overlap-save block 2^v for FP32 (9..17) */
    int32_t autotune;       /* 0: blocks by cost model; 1: time candidates, keep fastest  */
    double fsamp;           /* sampling frequency in Hz (> 0)                             */
    double rcond_min;       /* I/Q/U pixel acceptance (<= 0: 1e-6), see mm_plan           */
    void* stream;           /* cudaStream_t; NULL = legacy default stream                 */
    int32_t scatter_lanes;  /* 0: automatic (32, or timed when autotuning); else 32, 16 or 8
                               lanes per observed pixel in the scatter (mm_scatter_config)  */
} mm_opts;

typedef struct {
    int32_t iters;          /* A p products in PCG (all refinement steps)                 */
    int32_t outer;          /* refinement steps (1 for MM_SOLVE_FP64)                     */
    int32_t converged;      /* 1 when ||b - A m|| / ||b|| <= tol                         */
    int32_t fp64_products;  /* FP64 products A x spent on residuals (mixed)               */
    double rel_resid;       /* final true relative residual ||b - A m||_2 / ||b||_2       */
    double rel_resid_rec;   /* final recursive relative residual of the last PCG          */
    double ms_total;        /* device time of the call in milliseconds                   */
    double ms_rhs;          /* device time of b = P^T N^-1 d                             */
} mm_stats;

/*
 * mm_plan -- build the operators of one map-making problem.
 *
 * Paper: Sec. 2 (data model, Eq. 1-2, full-column-rank P), Eq. 4 and Sec. 4.1.4
 * (block-diagonal banded Toeplitz N^-1), Eq. 19 and App. D / Eq. 28 (rows from the PSD),
 * Eq. 10 (M_BD).
 *
 *   out          receives the plan (host pointer to a handle).
 *   pix          host or device int32[nt]: sky pixel of each sample, 0 <= pix < npix_sky.
 *   nt           number of samples, 1 <= nt < 2^31.
 *   npix_sky     number of sky pixels.
 *   weights      host or device double[nt][2] = (cos 2phi_t, sin 2phi_t) for ncomp = 3;
 *                must be NULL for ncomp = 1.
 *   interval_off host int64[K+1]: interval i is samples [off[i], off[i+1]);
 *                off[0] = 0, off[K] = nt, strictly increasing.
 *   K            number of stationary intervals (>= 1).
 *   interval_psd host int32[K]: PSD id of each interval, 0 <= id < npsd.
 *   psd          host mm_psd[npsd]: sigma > 0, fknee >= 0, alpha > 0.
 *   opts         host options; lambda must satisfy 0 <= lambda < shortest interval.
 *
 * Observed pixels (the columns of P): ncomp = 1 every pixel with >= 1 hit; ncomp = 3
 * every pixel with >= 3 hits whose unit-weight block sum_t w_t w_t^T has
 * lambda_min / lambda_max >= rcond_min.  Samples on other pixels have no entry in P.
 * Toeplitz row: r_k = (1/L) sum_{j<L} S_{min(j,L-j)}^-1 cos(2 pi j k / L) on the grid
 * L = 2^ceil(log2(longest interval)), S_j = sigma^2 (1 + (fknee/f_j)^alpha),
 * f_j = j fsamp / L, S_0^-1 = lim f->0 (0 if fknee > 0); t_k = w_k r_k with
 * w_k = exp(-2 (k/lambda)^2) (GAUSS) or 1 (RECT).  A row whose symbol
 * t_0 + 2 sum t_k cos(w k) is <= 0 anywhere on 2^ceil(log2(8 lambda)) frequencies is
 * rejected with MM_ERR_NOT_SPD.
 * Errors: MM_ERR_ARG (sizes, offsets, pixels, lambda, psd), MM_ERR_NOT_SPD,
 * MM_ERR_OOM, MM_ERR_CUDA.  On error *out is NULL.
 */
mm_status mm_plan(mm_plan_t* out, const int32_t* pix, int64_t nt, int32_t npix_sky,
                  const double* weights, const int64_t* interval_off, int32_t K,
                  const int32_t* interval_psd, const mm_psd* psd, int32_t npsd,
                  const mm_opts* opts);

/* Sizes of a plan.  Any output pointer may be NULL.  n = npix_obs * ncomp. */
mm_status mm_plan_info(mm_plan_t plan, int32_t* npix_obs, int64_t* n, int64_t* nkept,
                       int32_t* fft_block_f64, int32_t* fft_block_f32);

/*
 * Autotuning record (plans built with opts.autotune = 1; the paper has no counterpart).
 * ms_f64[v - 9] / ms_f32[v - 9]: average device milliseconds of one de-pointing Toeplitz
 * launch with the 2^v-real overlap-save block (v = 9..24), 0 for blocks not timed; at
 * most the three cheapest blocks of the cost model are timed per precision, the fastest
 * is kept.  Either pointer (host float[16]) may be NULL.
 */
mm_status mm_autotune_read(mm_plan_t plan, float* ms_f64, float* ms_f32);

/*
 * Pixel tile of the scatter P^T z: the number of lanes that share an observed pixel's
 * sorted samples (32, 16 or 8: one, two or four pixels per warp).  32 unless the plan
 * autotunes (opts.autotune), which times the FP32 scatter with each and keeps the
 * fastest.  lanes_per_pixel (host), ms (host float[3]: the timed launches for 32, 16 and
 * 8 lanes, or 0 when not timed); either may be NULL.  The paper has no counterpart.
 */
mm_status mm_scatter_config(mm_plan_t plan, int32_t* lanes_per_pixel, float* ms);

/*
 * Form of the batched operator (mm_apply_A_batch, mm_solve_batch), fixed once per plan by
 * its first batched call or by this call; the paper has no counterpart.
 *   kind  (host, in/out) in: -1 = choose, 0, 1 or 2 = use that form; out: the form in use.
 *         0: two right-hand sides per complex FFT of 2^log2_block points (real kernel
 *         spectrum: real and imaginary parts convolve independently);
 *         1: one real FFT per right-hand side with the FP32 block of mm_plan_info, the
 *         right-hand side as the fastest grid index;
 *         2: the band product as a dense contraction on the tensor cores (tcgen05 MMAs in
 *         FP16 on operands split as hi + 2^-11 lo after power-of-two scaling, FP32
 *         accumulators in tensor memory; 128-row tiles, window 128 + 2 lambda; the maps
 *         are de-pointed into a [R][nt] buffer first); log2_block reports 7 (the tile).
 *         Choosing times all three forms at R columns when the plan autotunes, else takes
 *         the cheaper FFT form by the cost model (the contraction costs 2 (2 lambda + 128)
 *         flops per sample and column against ~10 log2 B for the FFT).  Asking for a form
 *         other than the fixed one, or one that no block supports for this lambda, is
 *         MM_ERR_ARG.
 *   R     1..64, the column count for the timing (and the buffers it allocates).
 *   log2_block, ms (host float[3]: timed launches of forms 0, 1 and 2, or 0): may be NULL.
 */
mm_status mm_batch_config(mm_plan_t plan, int32_t R, int32_t* kind, int32_t* log2_block, float* ms);

/* obs2sky[q] (sky index of observed pixel q) and hits[q] (its sample count), both
 * host or device int32[npix_obs]; either may be NULL.  Bit-exact integer outputs. */
mm_status mm_plan_pixels(mm_plan_t plan, int32_t* obs2sky, int32_t* hits);

/* The Toeplitz row t_k, k = 0..lambda, of PSD id `psd_id` (host double[lambda+1]). */
mm_status mm_plan_row(mm_plan_t plan, int32_t psd_id, double* row);

/*
 * y = P x (de-pointing, Eq. 2; Sec. 2).  x device [n], y device [nt], in the arithmetic
 * `precision` (double for MM_FP64, float for MM_FP32).  Dropped samples give 0.
 */
mm_status mm_gather(mm_plan_t plan, int precision, const void* x, void* y);

/*
 * z = N^-1 y: the banded Toeplitz block of each stationary interval applied to that
 * interval only (Eq. 4, band of Sec. 4.1.4).  y, z device [nt] in `precision`.
 * Computed by overlap-save FFT in shared memory.
 */
mm_status mm_apply_ninv(mm_plan_t plan, int precision, const void* y, void* z);

/*
 * w = P^T z (pointing / scatter-add, Sec. 2).  z device [nt], w device [n] in
 * `precision`.  Deterministic segmented reduction over pixel-sorted samples.
 */
mm_status mm_scatter(mm_plan_t plan, int precision, const void* z, void* w);

/* y = A x = P^T [N^-1 [P x]] (Eq. 5, 8).  x, y device [n] in `precision`.  In FP32 on
 * an I/Q/U plan x is first copied, packed four floats per pixel, into a plan-owned buffer
 * that the de-pointing gather reads (one 16-byte load per sample); like the other scratch
 * buffers of a plan it is used in stream order on the plan's stream.  With unit-norm
 * weights the FP32 scatter forms each weight pair from a stored FP32 angle (within ~6e-7
 * of the pair); FP64 uses the pairs as given.
 * Errors of mm_gather, mm_apply_ninv, mm_scatter and mm_apply_A: MM_ERR_ARG for a null
 * vector, an unknown precision, or a precision with no overlap-save block for this
 * lambda (FP64 blocks reach lambda <= 32767, FP32 ones lambda <= 65535). */
mm_status mm_apply_A(mm_plan_t plan, int precision, const void* x, void* y);

/*
 * y = A x exactly as mm_apply_A, but without allocating device memory during the call.
 * The paper has no counterpart: this exists for callers that cannot allocate once they
 * run -- e.g. code whose GPU memory is already reserved by a pool it does not own (a
 * framework's caching allocator) or a latency-critical path where cudaMalloc could fail
 * or stall.  The time-domain intermediate of A x is kept in one 32 MiB array compiled
 * into the library (held on every device that loads it, until the process exits)
 * instead of in the plan's buffer; so nt * (8 for MM_FP64, 4 for MM_FP32) must not
 * exceed 32 MiB (nt <= 4194304 in FP64, 8388608 in FP32), else MM_ERR_ARG.
 * mm_plan looks up the array's device address (cudaGetSymbolAddress, with the plan's
 * device current), which also creates the array on that device; the call itself does
 * no set-up.  The call launches on the plan's stream and synchronises it before it
 * returns.  All calls share the array: every call rewrites what it reads, but calls
 * that overlap on the GPU (other streams, other host threads) race.  x, y device [n]
 * in `precision`.  Errors: those of mm_apply_A, and MM_ERR_ARG for a null plan.
 */
mm_status mm_apply_A_static(mm_plan_t plan, int precision, const void* x, void* y);

/* b = P^T N^-1 d (Eq. 7).  d device [nt] double, b device [n] double (FP64 arithmetic). */
mm_status mm_rhs(mm_plan_t plan, const double* d, double* b);

/*
 * z = M r with M = M_BD (Eq. 10; kind MM_PREC_BD), M_2lvl (Eq. 12; MM_PREC_TWOLEVEL,
 * applied as in App. C: v = E^-1 Z^T r, z = M_BD (r - (AZ) v) + Z v) or the A-DEF2 form
 * of App. B (Eq. B.1; MM_PREC_ADEF2: y = M_BD r, z = y + Z E^-1 (Z^T r - (AZ)^T y)).
 * r, z device [n] in `precision`.  The two-level kinds need a coarse space first
 * (MM_ERR_STATE).
 */
mm_status mm_precond(mm_plan_t plan, int kind, int precision, const void* r, void* z);

/*
 * Build the a posteriori coarse space Z_D of Sec. 3.3.2 (steps listed there; App. A):
 * one M_BD-preconditioned CG solve of A x' = b' (in `precision`, to rel. residual `tol`,
 * at most `maxit` steps), the Lanczos tridiagonal of that solve
 * (T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}, T_{j,j+1} = sqrt(beta_j)/alpha_j), its k
 * smallest Ritz pairs, Ritz vectors Z = sum_j (-1)^j z_j / sqrt(r_j^T z_j) s_j,
 * Euclidean orthonormalisation in FP64 (classical Gram-Schmidt projected twice, in
 * order; a column is dropped when its part orthogonal to the kept ones is below 1e-10
 * of the largest column norm -- an exact duplicate goes, a near-duplicate 1e-9 away
 * stays), then
 * AZ = A Z (FP64) and E = Z^T A Z, Cholesky-factored in FP64 (App. C, "Constructing"),
 * kept as E^-1 = L^-T L^-1 for the PCG kernels (when rounding leaves E numerically
 * indefinite, E^-1 comes from LU with partial pivoting, symmetrised).  A failed build
 * leaves the previous coarse space (or none) in place.
 *   k       requested coarse dimension, 1 <= k <= 64.
 *   bprime  device double[n] right-hand side of the first solve, or NULL for b' = the
 *           b of the last mm_solve (MM_ERR_STATE if there was none).
 * Errors: MM_ERR_NOT_SPD when E is singular, MM_ERR_NUMERIC when it holds NaN or Inf,
 * MM_ERR_ARG for k outside 1..64 or maxit < 1.
 */
mm_status mm_build_coarse(mm_plan_t plan, int k, int precision, const double* bprime,
                          double tol, int maxit);

/*
 * mm_build_coarse with the paper's selection rule (Sec. 5): the Ritz pairs kept are those
 * with |theta_i| < eps_tol (the paper uses 0.2), at most kmax of them, smallest first.
 * MM_ERR_STATE when no Ritz value lies below eps_tol (the previous coarse space, if any,
 * stays); MM_ERR_ARG for eps_tol <= 0.  Other arguments as mm_build_coarse.
 */
mm_status mm_build_coarse_eps(mm_plan_t plan, int kmax, double eps_tol, int precision, const double* bprime,
                              double tol, int maxit);

/*
 * The a posteriori coarse space from the paper's own Ritz source (App. A, Algorithm 1):
 * the basic Arnoldi process on B = M_BD A from w_1 = r_0/||r_0||, r_0 = M_BD b', in FP64
 * (classical Gram-Schmidt with one re-orthogonalisation pass), run until the GMRES
 * residual min ||beta e_1 - Hbar y|| <= tol beta, maxit steps or breakdown; the Ritz
 * pairs of H_m (Eq. A.4; Hessenberg QR and inverse iteration on the host) with
 * |Re lambda| < eps_tol (Sec. 5; the paper uses 0.2), at most kmax of them, smallest
 * real part first -- a complex pair contributes the real and imaginary parts of one
 * member's vector -- then Euclidean orthonormalisation with dropping and AZ, E, E^-1 as
 * for mm_build_coarse.  mm_coarse_info returns the selected real parts.  The basis
 * W_m lives in HBM (at most maxit + 1 columns of n doubles, grown on demand).
 *   bprime  device double[n] or NULL (the b of the last mm_solve).
 * Errors: MM_ERR_STATE when no Ritz value lies below eps_tol (previous space kept),
 * MM_ERR_NUMERIC if the Hessenberg QR fails, MM_ERR_ARG for bad arguments.
 */
mm_status mm_build_coarse_arnoldi(mm_plan_t plan, int kmax, double eps_tol, const double* bprime, double tol,
                                  int maxit);

/*
 * Install a given coarse basis Z (host or device double[k * n], column j at Z[j*n ..]):
 * its columns are orthonormalised in order with dependent ones dropped (the rule of
 * mm_build_coarse; a basis saved by mm_coarse_vectors is already orthonormal and comes
 * back unchanged up to rounding), then AZ = A Z, E = Z^T A Z, E^-1 as for
 * mm_build_coarse -- to reuse a basis saved from an earlier plan of the same pointing
 * without its construction solve.  mm_coarse_info reports the kept dimension.  The
 * columns must be finite (MM_ERR_NUMERIC otherwise, also when every column is zero);
 * the previous coarse space then stays.  1 <= k <= 64.
 * The paper has no counterpart beyond reusing a coarse space across solves.
 */
mm_status mm_coarse_import(mm_plan_t plan, const double* Z, int k);

/*
 * Build the a priori coarse space Z_S of Sec. 3.3.1 (Eq. 16-17) instead: column j of the
 * unmerged Z_S holds, for each observed pixel, the fraction of its samples inside
 * stationary interval j (temperature rows; Q/U rows 0), so each temperature row sums to
 * 1.  Its K columns are merged into r groups of consecutive intervals (interval i joins
 * group floor(i r / K); merged column = sum of its members, rows still sum to 1), as the
 * paper allows to reduce the coarse dimension.  The merged columns are replaced by an
 * orthonormal basis of their range (the orthonormalisation and dropping rule of
 * mm_build_coarse -- intervals that see the same hit fractions give equal columns,
 * which are dropped).  M_2lvl depends on Z only through its range, and the
 * orthonormal basis keeps E = Z^T A Z as well conditioned as A on that range (raw
 * hit-fraction columns of an evenly covered patch are nearly parallel).  Then AZ, E and
 * E^-1 as for mm_build_coarse.  No solve is needed.
 *   r       1 <= r <= min(64, K).
 * Errors: MM_ERR_ARG for r out of range, MM_ERR_NOT_SPD when E is not positive definite.
 */
mm_status mm_build_coarse_apriori(mm_plan_t plan, int r);

/* Kept coarse dimension and, for the a posteriori space, the k smallest Ritz values
 * (host double[k], may be NULL; nothing is written for the a priori space). */
mm_status mm_coarse_info(mm_plan_t plan, int32_t* k_kept, double* ritz_values);

/* The coarse basis Z (FP64), column j at Z[j*n .. j*n + n), host or device
 * double[k_kept * n], orthonormal (for the a priori space: a basis of the range of the
 * merged hit fractions).  MM_ERR_STATE before a coarse space was built. */
mm_status mm_coarse_vectors(mm_plan_t plan, double* Z);

/*
 * Solve A m = P^T N^-1 d by PCG from m_0 = 0 (Sec. 3.1), stopping when the relative
 * residual ||b - A m||_2 / ||b||_2 <= tol (the convergence measure of Sec. 5.1).
 *   d       host or device double[nt] time-ordered data.
 *   kind    MM_PREC_BD, MM_PREC_TWOLEVEL or MM_PREC_ADEF2 (the latter starts from
 *           x_0 = Z E^-1 Z^T b, which makes A-DEF2 equivalent to an SPD preconditioner in
 *           exact arithmetic, App. B; the others from x_0 = 0).
 *   solver  MM_SOLVE_FP64: all arithmetic FP64, stopping on the recursive residual.
 *           MM_SOLVE_MIXED: FP32 gather / Toeplitz / scatter and FP32 vectors with FP64
 *           dot products and step scalars inside PCG, FP64 E factor and solve, and an
 *           outer FP64 iterative-refinement loop m += A^-1 (b - A m) that stops on the
 *           true FP64 residual, computed from the data as P^T N^-1 (d - P m) (one FP64
 *           Toeplitz pass).  b itself is formed in FP32 (it seeds the first inner solve
 *           and scales the residual; ||b|| to FP32 accuracy) -- the one FP64 Toeplitz
 *           pass a converged first step needs is the residual.
 *   m       host or device double[n] output map.
 *   st      host stats (may be NULL).
 * Returns MM_ERR_NOT_CONVERGED (m = last iterate, st filled) when maxit is reached.
 */
mm_status mm_solve(mm_plan_t plan, const double* d, double tol, int maxit, int kind,
                   int solver, double* m, mm_stats* st);

/*
 * Per-stage device timers.  mm_profile(plan, 1) clears and enables them: every later
 * launch of the Toeplitz kernel (stage 0 FP64, 1 FP32; de-pointing fused or not), the
 * scatter kernel (2 FP64, 3 FP32), the PCG vector kernel (4 FP64, 5 FP32) and the
 * double-float Toeplitz kernel of the refinement residual (6) is bracketed by CUDA events
 * on the plan's stream (stage 7 is reserved).
 * mm_profile_read returns the summed milliseconds (host double[8]) and launch counts
 * (host int64[8]); either may be NULL.
 * The events add a few microseconds per launch; mm_profile(plan, 0) turns them off.
 */
mm_status mm_profile(mm_plan_t plan, int enable);
mm_status mm_profile_read(mm_plan_t plan, double* ms, int64_t* launches);

/*
 * Residual history of the last PCG solve on this plan (mm_solve, mm_solve_ex, the adjoint
 * solve of mm_grad, or the block-Jacobi solve inside an a posteriori mm_build_coarse*):
 * the relative recursive residual ||r_j||_2 / ||b||_2 after each product A p, the
 * convergence measure Sec. 5.1 plots.  Entry 0 is the start (1 for x_0 = 0, 0 when
 * b = 0; the A-DEF2 start of App. B is not counted: its entry 0 is also 1), entry j the
 * residual after the j-th product.  MM_SOLVE_MIXED concatenates its inner FP32 solves: their recursive
 * residuals, relative to the inner right-hand side r / ||r||, are scaled by the FP64
 * ||r|| / ||b|| of the refinement step they belong to, so each inner run starts at the
 * true residual and the entries estimate the true residual to FP32 accuracy.
 *   max        capacity of rel_resid (entries written: min(max, *count)).
 *   rel_resid  host double[max], may be NULL.
 *   count      host, may be NULL: number of entries, stats.iters + 1 (0 before any
 *              solve; fewer when a solve ran past 2^20 products, which are not kept).
 * Errors: MM_ERR_ARG for max < 0.  The batched solver keeps no history: after it the
 * entries are still those of the last single-right-hand-side solve.
 */
mm_status mm_solve_history(mm_plan_t plan, int32_t max, double* rel_resid, int32_t* count);

/*
 * Diagnostic of the bounded waits inside the persistent PCG kernels (the paper has no
 * counterpart).  Every grid-barrier wait of the cooperative PCG kernels is limited in
 * time (2 s in every solve) and a wait that runs out ends the kernel with
 * MM_ERR_TIMEOUT instead of hanging the GPU.  This call exercises that path without a
 * fault: it runs the FP64 block-Jacobi PCG start kernel on a zero right-hand side
 * through the solver's own driver, with the barrier counting `absent_blocks` blocks
 * that are never launched and each wait limited to `wait_s` seconds, and returns the
 * status the solver reports: MM_OK for absent_blocks = 0, MM_ERR_TIMEOUT (message in
 * mm_last_error) for absent_blocks > 0 after about wait_s.  The plan's barrier settings
 * go back to the defaults afterwards and the plan stays usable (every run starts from a
 * zeroed barrier counter).  The PCG vectors' contents are overwritten.
 *   absent_blocks  0 .. 1024;  wait_s  in (0, 10].
 * Errors: MM_ERR_ARG for arguments out of range.
 */
mm_status mm_pcg_barrier_check(mm_plan_t plan, int32_t absent_blocks, double wait_s);

/* Options of mm_solve_ex.  Zero-initialise and set what you need; 0 selects the default. */
typedef struct {
    double tol;             /* relative residual target (required, >= 0)                  */
    int32_t maxit;          /* total PCG iterations (required, >= 1)                      */
    int32_t kind;           /* MM_PREC_BD, MM_PREC_TWOLEVEL or MM_PREC_ADEF2               */
    int32_t solver;         /* MM_SOLVE_FP64 or MM_SOLVE_MIXED                             */
    int32_t max_outer;      /* refinement steps (MIXED), default 20                        */
    double inner_tol_min;   /* lower bound of the inner FP32 tolerance (MIXED), default 3e-7
                               (FP32 PCG tracks the true residual down to ~2e-7 relative)    */
    double first_inner_tol; /* inner tolerance of the first step (MIXED); default: the same
                               rule as later steps, max(inner_tol_min, 0.5 tol ||b||/||r||) */
    int32_t residual;       /* arithmetic of the refinement residuals (MIXED, and the batched
                               solver): MM_RESID_DF32 (default) or MM_RESID_FP64, see
                               mm_residual                                                  */
} mm_solve_opts;

/*
 * The residual of a map x from the data d, r = P^T N^-1 (d - P x) = b - A x (Eq. 5, 7),
 * in one pass: de-pointing and subtraction per sample in FP64, the band product N^-1 of
 * the residual data, then P^T in FP64.  `arith` selects the arithmetic of the band
 * product: MM_RESID_FP64 runs the overlap-save FFT in FP64; MM_RESID_DF32 runs the same
 * FFT in double-float arithmetic (unevaluated pairs of FP32 numbers, ~48-bit
 * significands, error-free two-sum and FMA two-product) on the FP32 pipe, which GB300
 * runs at 64 times its FP64 rate; its result agrees with the FP64 one to ~1e-13 of ||b||
 * and it is the default residual of the mixed-precision solver's iterative refinement.
 * The paper does not discuss arithmetic; this is this library's choice for Sec. 5.1's
 * stopping test at 1e-6 .. 1e-8.  d device double[nt], x, r device double[n].
 * Errors: MM_ERR_ARG for null vectors, an unknown `arith`, or no FP64 block for lambda.
 */
enum { MM_RESID_DF32 = 0, MM_RESID_FP64 = 1 };
mm_status mm_residual(mm_plan_t plan, int arith, const double* d, const double* x, double* r);

/* mm_solve with explicit options (same semantics and errors). */
mm_status mm_solve_ex(mm_plan_t plan, const double* d, const mm_solve_opts* opts, double* m, mm_stats* st);

/*
 * Many right-hand sides through one plan: R maps or data sets that share P, N^-1 and
 * M_BD (e.g. Monte-Carlo noise realisations).  The paper's setting for re-using a
 * precomputed preconditioner over many solves (Sec. 3.3.2); batching itself is not in it.
 *
 * mm_apply_A_batch: Y_r = A X_r (Eq. 8) in FP32 for r < R, 1 <= R <= 64; X, Y device
 * float[R][n].  Two right-hand sides share one complex FFT per overlap-save tile (the
 * Toeplitz spectrum is real), and each tile's pointing is read once for all of them.
 *
 * mm_solve_batch: solves A m_r = P^T N^-1 d_r for r < R (any R >= 1, processed 64 at a
 * time) with per-right-hand-side PCG scalars and stopping (Sec. 3.1 per column), block-
 * Jacobi preconditioner, MM_SOLVE_MIXED only: right-hand sides formed in one batched FP32
 * launch (they seed the first inner solve and scale the residual), FP64 refinement
 * residuals P^T N^-1 (d_r - P m_r) per column, batched FP32 inner PCG replayed from a
 * captured CUDA graph when the plan's stream is not the legacy default stream.  D host or
 * device double[R][nt], M host or device double[R][n], st host mm_stats[R] or NULL
 * (ms_total is the batch time divided by the columns of its group of 64).
 * MM_ERR_NUMERIC if a column's data holds NaN or Inf (that column: converged 0, rel_resid
 * NaN), else MM_ERR_NOT_CONVERGED if any column missed tol; all maps are still written.
 */
mm_status mm_apply_A_batch(mm_plan_t plan, int R, const float* X, float* Y);
mm_status mm_solve_batch(mm_plan_t plan, const double* D, int R, const mm_solve_opts* opts, double* M,
                         mm_stats* st);

/*
 * Gradients of a loss L(m) of the GLS map m = A^-1 P^T N^-1 d (Eq. 3, 5, 7), given
 * g = dL/dm at the solution m of the data d.  The paper does not differentiate Eq. 3;
 * with A symmetric one more PCG solve gives them:
 *   mu = A^-1 g                                     (adjoint solve, `opts` as mm_solve_ex)
 *   dL/dd = N^-1 P mu                               (dL_dd: host or device double[nt])
 *   dL/dtheta_pc = (P mu)^T (dN^-1/dtheta_pc) (d - P m)   (dL_dpsd: host double[npsd][3],
 *                                                    columns sigma, fknee, alpha)
 * dN^-1/dtheta is block Toeplitz with the derivative rows: the row transform of mm_plan
 * applied to d(1/S_j)/dtheta (analytic) times the window; the products u^T T v use the
 * same overlap-save kernel.  d, m, g: host or device, double.  Either output may be NULL.
 * The PSD gradient needs fknee > 0 for every PSD (MM_ERR_ARG otherwise).  All FP64
 * except the adjoint solve, which follows opts->solver.  Krylov vectors are not kept.
 */
mm_status mm_grad(mm_plan_t plan, const double* d, const double* m, const double* g, double* dL_dd,
                  double* dL_dpsd, const mm_solve_opts* opts, mm_stats* st);

/* Human-readable description of the last error on this plan (never NULL). */
const char* mm_last_error(mm_plan_t plan);

/* Release every device and host buffer of the plan.  NULL is accepted. */
void mm_destroy(mm_plan_t plan);

/* Library version string. */
const char* mm_version(void);

/* Number of CUDA kernels this process has launched through the library so far. */
int64_t mm_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* MM_H */
