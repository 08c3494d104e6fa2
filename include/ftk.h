/*
 * ftk.h -- C ABI of libftk, a GB300 (sm_103a) implementation of the FTK
 * pose-scoring path of "Factorization of the translation kernel for fast rigid
 * image alignment" (Rangan, Spivak, Anden, Barnett; arXiv 1905.12317).
 *
 * The library scores every image/template pair over all 2Q in-plane rotations
 * gamma_r = pi r / Q and a caller-given set of N shifts, through the rank-H SVD
 * factorization of the translation kernel (Section 4.5, eq. fbk3).
 *
 * Conventions (all calls):
 *  - Images are n x n float32, row-major, first index = x: pixel (i, j) sits at
 *    x_ij = (i dx - 1, j dx - 1), dx = 2/n (Section 2.1).
 *  - Fourier--Bessel coefficients are complex64 stored as interleaved float pairs
 *    (re, im), layout [B][M][2Q]: ring m (radial node k_m), angular frequency q
 *    at index q mod 2Q (Section 3.2, eq. aqkcalc).
 *  - Shifts are given in pixels; delta = s_px * dx. |s_px| must be <= 2W.
 *  - Scores are the real bandlimited inner product X(delta_s, gamma_r) of
 *    eq. (Xdg) as discretized in eq. (Xtrunc) (prefactor 2 pi and weights w_m
 *    included): the image is translated by delta, then rotated by gamma, then
 *    correlated with the template. X ~ (2 pi)^2 <R_gamma T_delta A, B>.
 *  - Coefficients passed to the align calls must come from real images: the
 *    kernels use the symmetry a(k; -q) = (-1)^q conj a(k; q) of real images to
 *    evaluate only the Bessel orders l >= 0 (orders -l contribute the complex
 *    conjugate of orders l).
 *  - d_* pointers are caller-owned device memory, h_* pointers caller-owned host
 *    memory. The library never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device calls are asynchronous on that stream; argument errors are returned
 *    before anything is launched. Errors raised on the device (a bounded wait
 *    that gave up) are latched in the plan and reported by ftk_stream_check.
 *  - All functions are thread-compatible, not thread-safe: do not use one plan
 *    from two host threads at once.
 */
#ifndef FTK_H_
#define FTK_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ftk_plan_s* ftk_plan_t;

typedef enum {
  FTK_OK = 0,
  FTK_ERR_ARG = 1,           /* invalid argument (null pointer, bad size)          */
  FTK_ERR_SHIFT_RANGE = 2,   /* a shift has |s_px| > 2W (outside Omega_D, Sec. 2)  */
  FTK_ERR_NOMEM = 3,         /* host or device allocation failed / workspace small */
  FTK_ERR_CUDA = 4,          /* a CUDA runtime call or kernel launch failed        */
  FTK_ERR_TIMEOUT = 5,       /* a device-side bounded wait gave up                 */
  FTK_ERR_PLAN_MISMATCH = 6, /* buffer sizes do not match the plan                 */
  FTK_ERR_UNSUPPORTED = 7,   /* configuration outside the implemented range       */
  FTK_ERR_SCRATCH_LIMIT = 8  /* problem too large for the fixed static scratch     */
} ftk_status;

/* Arithmetic of the pair engine (Steps 1-3). */
typedef enum {
  FTK_FP32 = 0,   /* FP32 SIMT kernels (FFMA only)                                  */
  FTK_BF16X3 = 1, /* tcgen05 BF16 tensor cores, 3-term split (hi*hi+hi*lo+lo*hi)    */
  FTK_BF16 = 2,   /* tcgen05 BF16 tensor cores, single term (for eps >= 1e-2 only)  */
  FTK_FP16 = 3    /* tcgen05 FP16 tensor cores, single term (11-bit significands;   */
                  /* operands must stay within the FP16 range, |x| < 65504)         */
} ftk_precision;

/*
 * ftk_plan_create -- image-independent planning (Section 4.5; excluded from the
 * timings, as in Section 6).
 *   n          image size (pixels), 8 <= n <= 256, even.
 *   K          band limit; K <= 0 selects the Nyquist value (pi/2) n (Remark r:nyq).
 *   W          maximum shift in wavelengths; shifts satisfy |s_px| <= 2W (Section 2).
 *   eps        SVD truncation: keep every Sigma_eta(l) > eps (eq. svdtrunc).
 *   M          radial Gauss--Jacobi(0,1) nodes on [0, K] (Section 3.1), 1..256.
 *   two_Q      angular nodes = rotations, 2Q = 2^a 3^b with 8 <= 2Q <= 768 (Sec. 3.2).
 *   shifts_px  host array [N][2] of shifts in pixels (x, y), copied.
 *   N          number of shifts, 1 <= N.
 *   out        receives the plan (owned by the library; free with ftk_plan_destroy).
 * Builds the radial rule (k_m, w_m), the per-order operator SVD of J_l(delta k)
 * (eq. Jsvd), keeps H_l terms per order, and uploads the radial factors
 * 2 pi w_m G_zeta(k_m) and the shift factors Y_zeta(delta_s) (eq. svdtrunc) to
 * the current CUDA device. Returns FTK_ERR_SHIFT_RANGE, FTK_ERR_ARG,
 * FTK_ERR_NOMEM or FTK_ERR_CUDA on failure (nothing is leaked), and
 * FTK_ERR_UNSUPPORTED if the largest kept Bessel order L reaches 2Q.
 */
ftk_status ftk_plan_create(int n, double K, double W, double eps, int M, int two_Q,
                           const double* shifts_px, int N, ftk_plan_t* out);

/*
 * ftk_plan_create_ctf -- a plan for CTF-filtered templates (Section 7.1): inner
 * products as a function of shift, rotation and defocus. The template is filtered
 * by the radially symmetric contrast transfer function
 *   C(k; tau_b) = -sin(pi tau_b (k / K)^2 + phase)
 * (defocus tau_b in half phase turns at k = K, no spherical aberration, `phase` the
 * amplitude-contrast phase), and F(delta, k) C(k; tau) is factorized per Bessel order
 * by one operator SVD over the rows (delta, tau_b), each defocus value weighted
 * 1 / n_defocus, and k. Steps 1-3 are those of ftk_plan_create with the N_shift x
 * n_defocus rows (defocus b, shift s) at row b N_shift + s in place of the shifts:
 * ftk_plan_info's N is that row count, ftk_align_scores writes [NI][NT][rows][R]
 * and ftk_align_best reports the row. defocus: host [n_defocus] (1..256 values,
 * |tau| <= 64); other arguments as ftk_plan_create. Truncation keeps Sigma > eps of
 * the joint kernel, so one defocus value's kernel error is up to sqrt(n_defocus) eps.
 * ftk_plan_defocus_count returns n_defocus (1 for a plan without CTF).
 */
ftk_status ftk_plan_create_ctf(int n, double K, double W, double eps, int M, int two_Q,
                               const double* shifts_px, int N, const double* defocus, int n_defocus,
                               double phase, ftk_plan_t* out);
int ftk_plan_defocus_count(ftk_plan_t plan);

/*
 * ftk_plan_create_weighted -- a plan whose modal SVDs use a spectral weight on k
 * (Section 4.5, the remark on alternative weight functions following Remark r:svd):
 * the L2 norm over the frequency disk becomes rho(k) k dk with
 *   rho(k) = exp(-decay (k/K)^2) decay / (1 - exp(-decay))
 * (a Gaussian power-spectral decay, normalized to unit mean over the disk; decay = 0
 * is ftk_plan_create). Per order l the SVD is that of J_l(delta k) sqrt(rho(k)); the
 * radial factors are Sigma V = Sigma Vtilde / sqrt(rho), so U Sigma V approximates
 * J_l(delta k) itself, optimally in the rho-weighted norm, and Steps 1-3 are
 * unchanged. For images whose power spectrum decays at least like rho (a Gaussian
 * blob of width sigma pixels has decay (pi sigma)^2), fewer terms (H) reach a given
 * accuracy of the inner products. decay: 0 <= decay <= 256 (FTK_ERR_ARG otherwise);
 * other arguments, ownership and errors as ftk_plan_create.
 * ftk_plan_spectral_decay returns the plan's decay (0 for a plan without a weight,
 * -1 for NULL).
 */
ftk_status ftk_plan_create_weighted(int n, double K, double W, double eps, int M, int two_Q,
                                    const double* shifts_px, int N, double decay, ftk_plan_t* out);
double ftk_plan_spectral_decay(ftk_plan_t plan);

/*
 * ftk_plan_save / ftk_plan_load -- the precomputation of Section 4.5 (quadrature
 * rule, kept terms with their Sigma, radial factors 2 pi w_m G_eta(k_m), shift
 * factors Y'(delta_s)), the shifts, CTF defocus values and phase, the spectral decay,
 * the rotation count and the tuning knobs, written to / read from a little-endian binary
 * file (magic "FTKPLAN1", 18 int32 header words, format version 2: K, W, eps, phase,
 * decay, then the arrays in that order; version 1 files, without the decay, are still
 * read as decay 0; the file is only meant for the machine family that wrote it). A loaded plan skips the modal SVDs:
 * its device tables are rebuilt from the stored factors on the current device, so
 * it gives the same results as the plan that was saved.
 *   ftk_plan_save: path host, NUL-terminated; the file is created or truncated.
 *     FTK_ERR_ARG on a NULL argument or an I/O failure.
 *   ftk_plan_load: *out receives a new plan owned by the caller (release with
 *     ftk_plan_destroy), NULL on failure. FTK_ERR_ARG if the file cannot be read,
 *     has the wrong magic or version, a size or knob out of the ranges that
 *     ftk_plan_create and ftk_plan_tune accept, or bytes left over;
 *     FTK_ERR_NOMEM / FTK_ERR_CUDA on device failure (nothing is leaked).
 */
ftk_status ftk_plan_save(ftk_plan_t plan, const char* path);
ftk_status ftk_plan_load(const char* path, ftk_plan_t* out);

/*
 * ftk_rank_profile -- host-only planning query (no device needed): the modal
 * ranks H_l = #{eta : Sigma_eta(l) > eps} of the operator SVD of J_l(delta k)
 * over the disk of radius D = 2 pi W / K (Section 4.5, eq. Jsvd; Lemma 1).
 *   max_l   orders 0..max_l are reported (>= 0).
 *   H_l     host output [max_l + 1] (may be NULL).
 *   sigma   host output [(max_l + 1) * n_sigma]: the n_sigma largest Sigma_eta(l)
 *           of each order, row l (may be NULL).
 *   H_total receives sum over all orders l in Z of H_l (both signs; may be NULL).
 * ftk_rank_profile_weighted: the same for the spectrally weighted SVD of
 * ftk_plan_create_weighted (0 <= decay <= 256, else FTK_ERR_ARG).
 */
ftk_status ftk_rank_profile_weighted(double W, double eps, double decay, int max_l, int* H_l, double* sigma,
                                     int n_sigma, int* H_total);
ftk_status ftk_rank_profile(double W, double eps, int max_l, int* H_l, double* sigma, int n_sigma,
                            int* H_total);

/* Destroys a plan and its device tables. NULL is accepted. */
void ftk_plan_destroy(ftk_plan_t plan);

/*
 * ftk_plan_info -- sizes of a plan. Any output pointer may be NULL.
 *   H        total rank sum_l H_l over all orders l (both signs; Section 4.5).
 *   H_half   number of terms with l >= 0 (what the kernels evaluate).
 *   L        largest order with H_l > 0.
 *   M, two_Q, N, n  as planned.
 */
ftk_status ftk_plan_info(ftk_plan_t plan, int* H, int* H_half, int* L, int* M, int* two_Q,
                         int* N, int* n);

/*
 * ftk_plan_set_rotations -- evaluate Step 2 on a finer rotation grid
 * gamma_r = 2 pi r / n_rot, r = 0..n_rot-1 (Section 3.2: the transform over q is
 * zero-padded from 2Q to n_rot points). n_rot must be a multiple of 2Q; n_rot = 2Q
 * restores the default grid. Other values need the tensor-core engine and
 * n_rot in {96, 192, 288, 384, 576, 768} (FTK_ERR_UNSUPPORTED otherwise); the FP32
 * engine then returns FTK_ERR_UNSUPPORTED. Afterwards ftk_align_scores writes
 * [NI][NT][N][n_rot] and ftk_align_best reports r in [0, n_rot). Synchronizes the
 * device (it replaces a device table). ftk_plan_rotations returns the current count.
 */
ftk_status ftk_plan_set_rotations(ftk_plan_t plan, int n_rot);
int ftk_plan_rotations(ftk_plan_t plan);

/*
 * ftk_plan_terms -- the retained terms with l >= 0, in kernel order (grouped by
 * l ascending, eta ascending). Host outputs of length H_half, any may be NULL:
 * l[zeta], sigma[zeta] = Sigma_eta(l) (Section 4.5, eq. Jsvd).
 */
ftk_status ftk_plan_terms(ftk_plan_t plan, int* l, double* sigma);

/*
 * ftk_plan_tune -- launch-shape knobs of the tensor-core kernels (results are
 * identical for every setting; only speed changes). `value` 0 restores the
 * default. Knobs:
 *   "step3_group_max"   upper bound on the shifts per Step-3 group (16..256, x16)
 *   "step3_a_stages"    minimum A K-slice pipeline stages of Step 3 (1..12); the
 *                       kernel uses as many as fit next to the resident B slice
 *   "step1_stages"      operand pipeline stages of Step 1 (1..8)
 *   "step1_ctas_per_sm" Step-1 work units per SM (1..8)
 *   "fft_lanes"         Step 2 + packing (all-scores path and plans the fused Steps 2-3
 *                       do not fit): 0 = the two-factor DFT 2Q = 12 N1 (2Q = 96, 192, 288,
 *                       384 with R = 2Q), else 16 lanes per transform; or the register FFT
 *                       with 8 (96, 192), 16 (96, 192, 288, 384) or 32 lanes per transform
 *   "transform"         0: polar transform on tensor cores where the plan has it
 *                       (n a multiple of 16, n <= 256), 1: the FP32 SIMT transform
 *   "step23"            best-pose searches (ftk_align_best and the calls built on it,
 *                       ftk_align_best_shortlist): 1 (default) runs Steps 2 and 3 as one
 *                       tensor-core kernel where the plan fits it (BF16x3 / BF16,
 *                       2Q = 96 or 192 with R = 2Q, 128-shift tiles x K and shared memory
 *                       within the SM's), 0 always the separate Step-2 and Step-3 kernels
 *   "cluster23"         with step23 = 1: 1 also fuses Steps 2 and 3 where 2Q = 128 R
 *                       (R = 2, 3, 4; 2Q = 384 at n = 128) over a cluster of CTAs, one per
 *                       Step-3 shift group (2..8 groups, K a multiple of 32), the DFT over q
 *                       of each pair computed once per cluster and shared between its CTAs'
 *                       shared memories; 0 (default) the separate kernels there
 *   "checks"            1: the fused Steps 2-3 check every global, shared-memory and tensor-
 *                       memory index against its buffer before the access; a violation
 *                       latches an index error (ftk_stream_check then reports FTK_ERR_ARG)
 *                       and the access is skipped. 0 (default): no checks
 * Changing a Step-3 knob synchronizes the device and rebuilds the plan's split
 * shift-factor tables. FTK_ERR_ARG for an unknown knob or a value out of range.
 * ftk_plan_tuning reports the effective Step-3 shape: shifts per group, number of
 * groups, A stages (outputs may be NULL).
 */
ftk_status ftk_plan_tune(ftk_plan_t plan, const char* knob, int value);
ftk_status ftk_plan_tuning(ftk_plan_t plan, int* step3_group, int* step3_groups, int* step3_a_stages);

/*
 * ftk_plan_radial_rule -- the radial nodes k_m and weights w_m (Section 3.1),
 * host outputs of length M. Either may be NULL.
 */
ftk_status ftk_plan_radial_rule(ftk_plan_t plan, double* k, double* w);

/*
 * ftk_transform -- pixel images to Fourier--Bessel coefficients.
 *   d_images  device [B][n][n] float32.
 *   B         number of images (>= 0; 0 is a no-op).
 *   d_coeffs  device [B][M][2Q] complex64 (interleaved float pairs), written.
 * Evaluates the trapezoid Fourier transform of eq. (Ahattrap) on the polar grid
 * (k_m, psi_p = pi p / Q) (Section 3.2) and the ring DFT of eq. (aqkcalc),
 * a(k_m; q) = (1/2Q) sum_p Ahat(k_m, psi_p) exp(-i q psi_p). For n a multiple of
 * 16 (n <= 256) the pixel sum runs on tensor cores with split-bf16 operands (three
 * products, FP32 accumulation; about 1e-6 of the peak coefficient); otherwise, or
 * with the "transform" knob at 1, in FP32 on CUDA cores. The tensor-core form
 * packs pixels into scratch owned by the plan: calls with the same plan must not
 * run concurrently on different streams.
 */
ftk_status ftk_transform(ftk_plan_t plan, const float* d_images, int B, float* d_coeffs,
                         void* stream);

/*
 * ftk_workspace_size -- device scratch for ftk_align_scores / ftk_align_best.
 *   min_bytes   smallest workspace that works (one pair block at a time).
 *   good_bytes  a size that lets the library use large chunks (>= min_bytes; on the
 *               tensor-core engine up to 16 GiB: larger chunks mean fewer, fuller launches).
 * Larger workspaces never change results, only the chunking of the pair space. On the
 * tensor-core engine a search picks, within the workspace it is given, the chunk shape
 * (images x templates) whose Step-1 work units fill whole rounds of the SMs, and keeps
 * the packed operands of all templates where they fit beside it; good_bytes is the
 * scratch of the shape it picks within 16 GiB.
 */
ftk_status ftk_workspace_size(ftk_plan_t plan, int precision, int NI, int NT,
                              size_t* min_bytes, size_t* good_bytes);

/*
 * ftk_align_scores -- all scores X(delta_s, gamma_r) for every pair
 * (Section 4.5, eq. fbk3 Steps 1-3).
 *   precision     an ftk_precision value.
 *   d_img_coeffs  device [NI][M][2Q] complex64 image coefficients (from ftk_transform).
 *   d_tpl_coeffs  device [NT][M][2Q] complex64 template coefficients.
 *   d_scores      device [NI][NT][N][R] float32, written (s-major, then r), R = the
 *                 plan's rotation count (2Q unless ftk_plan_set_rotations changed it).
 *   d_work        device scratch of work_bytes >= ftk_workspace_size(min_bytes),
 *                 256-byte aligned; contents are overwritten.
 */
ftk_status ftk_align_scores(ftk_plan_t plan, int precision, const float* d_img_coeffs, int NI,
                            const float* d_tpl_coeffs, int NT, float* d_scores, void* d_work,
                            size_t work_bytes, void* stream);

/*
 * ftk_align_best -- per image, the maximum score over (template, rotation,
 * shift) and where it is attained (Section 6, consistency check). The full
 * pairs x rotations x shifts tensor is never written to memory.
 *   d_tpl, d_rot, d_shift  device [NI] int32 outputs: template j, rotation r
 *                          (gamma = 2 pi r / R, R = the plan's rotation count, 2Q
 *                          by default), shift index s (into shifts_px).
 *   d_score                device [NI] float32 output: the maximum score.
 * Ties are broken by the lowest (template, rotation, shift) index. Any NT: where
 * NT * R * N reaches 2^32 the templates are searched in blocks of fewer than
 * 2^32 / (R N) (one per chunk), each block's maximum merged into the outputs after
 * it (same results and tie rule); R * N itself must stay below 2^32
 * (FTK_ERR_UNSUPPORTED otherwise). The call must be made with the plan's device
 * current (FTK_ERR_ARG otherwise), as must every call that launches work on a plan.
 */
ftk_status ftk_align_best(ftk_plan_t plan, int precision, const float* d_img_coeffs, int NI,
                          const float* d_tpl_coeffs, int NT, int* d_tpl, int* d_rot,
                          int* d_shift, float* d_score, void* d_work, size_t work_bytes,
                          void* stream);

/*
 * ftk_align_best_groups -- ftk_align_best over several groups in one call: each
 * group has its own plan (grid n, M, 2Q, shifts), image and template coefficients
 * and outputs, as in a batch of uneven image sizes. The groups run on the library's
 * own streams (created on the current device at the first call; make that call
 * outside stream capture), forked from and joined to `stream`, so that the GPU
 * overlaps them; the whole call can then be captured into a CUDA graph and
 * replayed as one launch. Results are those of ftk_align_best per group (same
 * kernels, same numbers).
 *   groups     host array [n_groups]; every plan on the current device; outputs as
 *              in ftk_align_best. Groups with NI = 0 are skipped.
 *   d_work     device, 256-byte aligned; split among the groups: every group gets
 *              its ftk_workspace_size good size if the total allows, otherwise its
 *              min size plus a share of the rest in proportion to (good - min).
 * ftk_groups_workspace_size returns the sums (over groups, with alignment) of the
 * per-group min and good sizes. Errors: FTK_ERR_ARG for a NULL array, n_groups < 1
 * or > FTK_MAX_GROUPS, or a group that ftk_align_best would reject;
 * FTK_ERR_NOMEM if work_bytes is below the min sum; otherwise the first failing
 * group's status (groups already launched keep running and are joined).
 */
#define FTK_MAX_GROUPS 64
typedef struct {
  ftk_plan_t plan;
  const float* d_img_coeffs; /* [NI][M][2Q] complex64 of this group's plan */
  int NI;
  const float* d_tpl_coeffs; /* [NT][M][2Q] complex64 */
  int NT;
  int* d_tpl;                /* outputs [NI], as ftk_align_best */
  int* d_rot;
  int* d_shift;
  float* d_score;
} ftk_group;
ftk_status ftk_groups_workspace_size(const ftk_group* groups, int n_groups, int precision, size_t* min_bytes,
                                     size_t* good_bytes);
ftk_status ftk_align_best_groups(const ftk_group* groups, int n_groups, int precision, void* d_work,
                                 size_t work_bytes, void* stream);

/*
 * ftk_search_workspace_size / ftk_search_host -- end-to-end call from host
 * buffers: copies h_images [NI][n][n] and h_templates [NT][n][n] (float32, host;
 * pinned memory recommended) to the device, transforms both (eq. Ahattrap,
 * aqkcalc), runs ftk_align_best, copies the [NI] results back to h_tpl, h_rot,
 * h_shift, h_score and synchronizes the stream. d_work (device, 256-byte aligned)
 * holds the pixels, the coefficients and the align workspace.
 */
ftk_status ftk_search_workspace_size(ftk_plan_t plan, int precision, int NI, int NT,
                                     size_t* min_bytes, size_t* good_bytes);
ftk_status ftk_search_host(ftk_plan_t plan, int precision, const float* h_images, int NI,
                           const float* h_templates, int NT, int* h_tpl, int* h_rot,
                           int* h_shift, float* h_score, void* d_work, size_t work_bytes,
                           void* stream);

/*
 * ftk_align_best_static -- ftk_align_best without a caller workspace and without
 * any device allocation. (The paper has no counterpart: this is a deployment
 * convenience of the library.)
 *
 * Who needs it: callers that cannot call cudaMalloc at this point. Typical cases
 * are programs whose device memory is owned by another allocator (a framework's
 * caching pool or a fixed-budget runtime that must account for every byte), and
 * pipelines that cannot afford an allocation at call time, because cudaMalloc
 * may block, may synchronize the device, or may fail late. Such a caller still
 * passes its own inputs and outputs; the scratch space of the pair engine comes
 * from one fixed array that the library reserves statically on every GPU that
 * loads it, FTK_STATIC_SCRATCH_BYTES in size, held until the process exits.
 *
 * Arguments and results are those of ftk_align_best (same kernels, same
 * numbers), minus d_work/work_bytes. Limits: the per-image keys (8 bytes per
 * image) plus the engine's minimum workspace for this plan and precision
 * (ftk_workspace_size's min_bytes) must fit in FTK_STATIC_SCRATCH_BYTES;
 * otherwise FTK_ERR_SCRATCH_LIMIT is returned before anything is launched.
 *
 * The first call on a device looks up the device address of the static array
 * (cudaGetSymbolAddress, with that device current); make that first call before
 * any stream capture. The call itself allocates nothing: no cudaMalloc, no
 * cudaFree, no allocating library routine.
 *
 * All calls in the process share the one array per device, and it keeps the
 * contents of the last call (the per-image maxima are re-initialized by each
 * call before use). Calls whose work overlaps on the GPU -- on different
 * streams, or from different host threads -- race on that array and must be
 * serialized by the caller.
 */
#define FTK_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)
ftk_status ftk_align_best_static(ftk_plan_t plan, int precision, const float* d_img_coeffs, int NI,
                                 const float* d_tpl_coeffs, int NT, int* d_tpl, int* d_rot,
                                 int* d_shift, float* d_score, void* stream);

/*
 * ftk_align_best_shortlist -- ftk_align_best restricted, per image, to a
 * shortlist of templates and optionally to a window of shifts. The paper has no
 * counterpart: it is the same Steps 1-3 of eq. fbk3 over fewer pairs and shifts,
 * used with the template-proposal network below.
 *   precision    FTK_FP32: FP32 SIMT engine for Steps 1-3. FTK_BF16X3 / FTK_BF16: the
 *                tensor-core engine of ftk_align_best (same precision semantics); Step 1
 *                multiplies each image with its own tile of shortlisted templates,
 *                gathered from one packing of all NT templates.
 *   d_shortlist  device [NI][K] int32 template indices (into d_tpl_coeffs, < NT).
 *   d_center_px  device [NI][2] float32 window centres in pixels, or NULL for
 *                every shift; a shift s is scored if max(|s_x - c_x|, |s_y - c_y|)
 *                <= window_px.
 * Outputs as ftk_align_best (template indices are global). An image with no shift
 * inside its window gets template = rotation = shift = -1 and score = -inf, and the
 * next ftk_stream_check returns FTK_ERR_ARG. Where NT * R * N reaches 2^32 the pose
 * keys count shortlist positions (K * R * N must stay below 2^32; equal scores then
 * keep the earlier list entry). A shortlist index outside [0, NT) is replaced by 0 and latched: the next
 * ftk_stream_check returns FTK_ERR_ARG. ftk_shortlist_workspace_size gives the
 * smallest d_work (one image per launch) and a size that runs up to 512 images per
 * launch within 16 GiB.
 */
ftk_status ftk_shortlist_workspace_size(ftk_plan_t plan, int precision, int NI, int NT, int K,
                                        size_t* min_bytes, size_t* good_bytes);
ftk_status ftk_align_best_shortlist(ftk_plan_t plan, int precision, const float* d_img_coeffs, int NI,
                                    const float* d_tpl_coeffs, int NT, const int* d_shortlist, int K,
                                    const float* d_center_px, float window_px, int* d_tpl, int* d_rot,
                                    int* d_shift, float* d_score, void* d_work, size_t work_bytes,
                                    void* stream);

/*
 * Template-proposal network building blocks (FP32 CUDA kernels; no paper
 * counterpart). Activations are NCHW contiguous, convolution weights
 * [Co][Ci][3][3], linear weights [O][I]. All pointers are device memory; every
 * call is asynchronous on `stream`; FTK_ERR_ARG for invalid sizes or pointers.
 *  ftk_nn_features     coefficients [B][M][2Q] complex64 -> x0 [B][1][M][Q] =
 *                      log(eps_f + |a(k_m; q)|), q < Q (rotation invariant, Section 3),
 *                      lin [B][4M] = (Re a(.,0), Im a(.,0), Re a(.,1), Im a(.,1)).
 *  ftk_nn_conv3x3      y = conv3x3(x, w) + b (zero padding 1), ReLU if relu != 0.
 *  ftk_nn_conv3x3_backward  from dz = dLoss/d(pre-activation): dx (if d_dx != NULL),
 *                      dw, db.
 *  ftk_nn_relu_backward  dy *= (y > 0), y the post-ReLU output, n elements.
 *  ftk_nn_pool2 / _backward  2x2 average pool on BC planes of H x W (H, W even).
 *  ftk_nn_gap / _backward    global average over HW per plane.
 *  ftk_nn_linear       y[B][O] = [x1 | x2][B][I] w^T + b (x1 has I1 columns, x2 the
 *                      remaining I - I1, may be NULL when I1 == I), ReLU if relu != 0.
 *  ftk_nn_linear_backward  dx1 (first I1 input columns, if d_dx1 != NULL), dw, db.
 *  ftk_nn_loss         per row b of out [B][NT + 2]: softmax cross entropy of the NT
 *                      logits with label[b] plus lam * squared error of the last two
 *                      outputs against target[b][2]; writes d(mean loss)/d out and
 *                      the row losses loss[B] (NaN for a label outside [0, NT)).
 *  ftk_nn_adam         Adam step t (>= 1) on n parameters.
 *  ftk_nn_topk         per row of out (row stride `stride`), the indices of the k
 *                      largest of the first NT values, descending (ties: lower index;
 *                      NaN ranks below -inf). NT <= 20480.
 *  ftk_nn_confidence   softmax of the first NT values of row b (row stride `stride`):
 *                      conf[b] = its mass on the K indices idx[b][0..K) (a shortlist), or
 *                      its largest value when idx is NULL.
 *  ftk_nn_eqhead       rotation-equivariant template head on the Fourier-Bessel
 *                      coefficients a [B][M][2Q] (complex64) with learned ring filters
 *                      W [NT][Mh][2Qh+1] (complex64, u = q + Qh) and biases beta [NT]:
 *                      X_ij(r) = Re sum_{m<Mh, |q|<=Qh} W_j(m,q) a_i(k_m;q) e^{-i q gamma_r},
 *                      gamma_r = 2 pi r / 2Q (the rotation grid of Section 3); writes
 *                      (or adds, if accumulate != 0) alpha max_r X_ij(r) + beta_j at
 *                      out[i * out_stride + j] and the first maximising r at rstar [B][NT].
 *                      A grid rotation of the image moves r* and keeps the logit.
 *                      Needs 1 <= Mh <= M, 2 Qh + 1 <= 2Q, out_stride >= NT.
 *  ftk_nn_eqhead_backward  from g = dout [B][out_stride] and rstar: dW (as d/dRe + i d/dIm)
 *                      and dbeta (overwritten).
 *  ftk_gather_rows     dst[r] = src[rows[r]] for n rows of row_elems floats; src has n_src
 *                      rows, and a row index outside [0, n_src) gives a row of NaN.
 *  ftk_scatter_rows    dst[rows[r]] = src[r] for n rows; dst has n_dst rows, and a row
 *                      index outside [0, n_dst) is skipped.
 *  ftk_select_below    rows[0..count) = the indices b < n with val[b] < thr, in no
 *                      particular order; *d_count (device int) receives count.
 *  ftk_nn_scale_filters  head filters with one spectral weight for all templates:
 *                      W [NT][S] = rho [S] * W0 [NT][S] (complex64 W0, W; real rho; S = Mh (2Qh+1)).
 *  ftk_nn_scale_filters_backward  drho [S] = sum_j Re(dW_j) Re(W0_j) + Im(dW_j) Im(W0_j) from
 *                      dW [NT][S] = dL/dRe W + i dL/dIm W (as ftk_nn_eqhead_backward writes it).
 *  ftk_nn_snap_to_shifts  out [B][2] = the shift of shifts [N][2] (pixels) nearest to
 *                      center [B][2] in the max norm (ties: lowest index): a shift window
 *                      (ftk_align_best_shortlist) around it is never empty.
 */
ftk_status ftk_nn_confidence(const float* d_out, int B, int stride, int NT, const int* d_idx, int K,
                             float* d_conf, void* stream);
ftk_status ftk_nn_features(const float* d_coeffs, int B, int M, int two_Q, float eps_f, float* d_x0,
                           float* d_lin, void* stream);
ftk_status ftk_nn_conv3x3(const float* d_x, const float* d_w, const float* d_b, float* d_y, int B, int Ci,
                          int Co, int H, int W, int relu, void* stream);
ftk_status ftk_nn_conv3x3_backward(const float* d_x, const float* d_w, const float* d_dz, float* d_dx,
                                   float* d_dw, float* d_db, int B, int Ci, int Co, int H, int W,
                                   void* stream);
ftk_status ftk_nn_relu_backward(const float* d_y, float* d_dy, long long n, void* stream);
ftk_status ftk_nn_pool2(const float* d_x, float* d_y, long long BC, int H, int W, void* stream);
ftk_status ftk_nn_pool2_backward(const float* d_dy, float* d_dx, long long BC, int H, int W, void* stream);
ftk_status ftk_nn_gap(const float* d_x, float* d_y, long long BC, int HW, void* stream);
ftk_status ftk_nn_gap_backward(const float* d_dy, float* d_dx, long long BC, int HW, void* stream);
ftk_status ftk_nn_linear(const float* d_x1, const float* d_x2, int I1, const float* d_w, const float* d_b,
                         float* d_y, int B, int I, int O, int relu, void* stream);
ftk_status ftk_nn_linear_backward(const float* d_x1, const float* d_x2, int I1, const float* d_w,
                                  const float* d_dy, float* d_dx1, float* d_dw, float* d_db, int B, int I,
                                  int O, void* stream);
ftk_status ftk_nn_loss(const float* d_out, const int* d_label, const float* d_target, int B, int NT,
                       float lam, float* d_dout, float* d_loss, void* stream);
ftk_status ftk_nn_adam(float* d_p, const float* d_g, float* d_m, float* d_v, long long n, float lr,
                       float b1, float b2, float eps, int t, void* stream);
ftk_status ftk_nn_topk(const float* d_out, int B, int stride, int NT, int k, int* d_idx, void* stream);
ftk_status ftk_nn_eqhead(const float* d_a, int B, int M, int two_Q, const float* d_W, const float* d_beta,
                         int NT, int Mh, int Qh, float alpha, float* d_out, int out_stride, int accumulate,
                         int* d_rstar, void* stream);
ftk_status ftk_nn_eqhead_backward(const float* d_a, int B, int M, int two_Q, const float* d_dout,
                                  int out_stride, const int* d_rstar, int NT, int Mh, int Qh, float alpha,
                                  float* d_dW, float* d_dbeta, void* stream);
ftk_status ftk_scatter_rows(const float* d_src, const int* d_rows, long long n, int row_elems, float* d_dst,
                            long long n_dst, void* stream);
ftk_status ftk_select_below(const float* d_val, long long n, float thr, int* d_rows, int* d_count,
                            void* stream);
ftk_status ftk_gather_rows(const float* d_src, long long n_src, const int* d_rows, long long n,
                           int row_elems, float* d_dst, void* stream);
ftk_status ftk_nn_snap_to_shifts(const float* d_center, int B, const float* d_shifts, int N, float* d_out,
                                 void* stream);
ftk_status ftk_nn_scale_filters(const float* d_W0, const float* d_rho, int NT, int S, float* d_W, void* stream);
ftk_status ftk_nn_scale_filters_backward(const float* d_W0, const float* d_dW, int NT, int S, float* d_drho,
                                         void* stream);

/*
 * ftk_stream_check -- synchronizes `stream` and reports errors: FTK_ERR_CUDA for
 * a CUDA error, FTK_ERR_TIMEOUT if a kernel latched a bounded-wait timeout since
 * the last check, FTK_ERR_ARG if a kernel latched an out-of-range device-side
 * index (a shortlist entry), else FTK_OK. The latch is cleared.
 */
ftk_status ftk_stream_check(ftk_plan_t plan, void* stream);

/*
 * ftk_selftest_timeout -- exercises the failure path of the bounded waits (no paper
 * counterpart): one thread waits, for at most limit_us microseconds (1..2e6), on a
 * device barrier that nothing completes; the wait gives up, latches the timeout in
 * the plan's error word and the kernel returns. The next ftk_stream_check on the
 * stream returns FTK_ERR_TIMEOUT (and clears the latch); the context stays usable.
 */
ftk_status ftk_selftest_timeout(ftk_plan_t plan, unsigned int limit_us, void* stream);

/* Static description of a status code. */
const char* ftk_status_string(ftk_status status);

/* Number of kernel launches issued through this plan since creation. */
long long ftk_plan_launch_count(ftk_plan_t plan);

/*
 * Launch profiler (measurement support, not part of the method). Between
 * ftk_profile_begin and ftk_profile_end every kernel launched through `plan` is
 * bracketed by CUDA events recorded on its launch stream. ftk_profile_end
 * synchronizes `stream`, accumulates the event durations and stops recording.
 * ftk_profile_kernel reads, for kernel id 0..FTK_NUM_KERNELS-1, its name, the
 * summed duration in milliseconds and the number of launches (outputs may be NULL;
 * FTK_ERR_ARG for an id out of range).
 */
#define FTK_NUM_KERNELS 15
ftk_status ftk_profile_begin(ftk_plan_t plan);
ftk_status ftk_profile_end(ftk_plan_t plan, void* stream);
ftk_status ftk_profile_kernel(ftk_plan_t plan, int id, const char** name, double* total_ms,
                              long long* launches);

#ifdef __cplusplus
}
#endif

#endif /* FTK_H_ */
