/*
 * zinv.h -- C ABI of libzinv.so: inverse and determinant of every pixel's 3x3
 * Hermitian positive-definite PolSAR covariance matrix on a GB300 (sm_103a).
 *
 * Method: D. F. G. Coelho, R. J. Cintra, A. C. Frery, V. S. Dimitrov, "Fast
 * Matrix Inversion and Determinant Computation for Polarimetric Synthetic
 * Aperture Radar", arXiv:1807.08084.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Packed Hermitian layout (§2.1: only the upper triangle is stored).  A pixel's
 *     Z = [[a, b, c], [conj b, d, e], [conj c, conj e, f]],  a, d, f real,
 * is stored as nine float planes in the paper's letter order
 *     plane 0:a 1:Re b 2:Im b 3:Re c 4:Im c 5:d 6:Re e 7:Im e 8:f
 * and element k of pixel p lives at ptr[k*ld + p] (ld >= n, in elements).  A
 * torch tensor of shape [9, H, W] (contiguous) is this layout with ld = H*W.
 * Outputs Z^-1 use the same layout; det is one float plane [n].
 *
 * Single-look data (§1: S = [S_HH, S_HV, S_VV]^T): three complex64 planes,
 * interleaved (re, im) floats; component i of pixel (y, x) at s[i*plane_ld + y*W + x]
 * (plane_ld and the index in complex elements).
 *
 * Memory: every pointer is owned by the caller.  Unless an entry point says
 * otherwise, pointers are device pointers (cudaMalloc, torch) or managed
 * memory; the library allocates no device memory in any call and keeps no
 * reference after the call returns.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Every call enqueues its work asynchronously on that stream and
 * returns without synchronizing; results are valid once the stream reaches
 * that point.  The device-pointer calls can be captured into a CUDA graph on
 * that stream (global capture mode included); replays give the eager results.
 * wishart_stat_fwd_noalloc must run once on a device before any capture (it
 * looks up its scratch address then).
 *
 * Errors: every int-returning call returns ZINV_OK (0) or a negative code.  An
 * argument error is detected on the host before anything is enqueued.  Nothing
 * in the library traps or asserts on the device; per-pixel problems (a matrix
 * that is not positive definite, non-finite input) are reported in the
 * optional status plane and counters and leave IEEE results in the outputs.
 * Calls that share output buffers and overlap on the GPU race; nothing else is
 * shared between calls, except the streams zinv_det_host keeps per device.
 */
#ifndef ZINV_H
#define ZINV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ZINV_ABI_VERSION 1

/* return codes */
#define ZINV_OK 0
#define ZINV_ERR_ARG (-1)    /* null/misaligned/inaccessible pointer, bad size or flag */
#define ZINV_ERR_LAUNCH (-2) /* a CUDA call or kernel launch failed */
#define ZINV_ERR_DEVICE (-3) /* current device is not an sm_103 GPU, or no device */

/* flags of zinv_det / multilook_zinv_det / zinv_det_host (bitwise or) */
#define ZINV_PLAIN 0u
#define ZINV_COMPENSATED 1u   /* FMA error-free products and sums in the cofactors and det */
#define ZINV_FP64_RECOMPUTE 2u /* recompute pixels with det <= tau*a*d*f in FP64 */
#define ZINV_HOST_STAGED 4u    /* zinv_det_host only: always stage through the workspace */

/* bits of the optional per-pixel status plane */
#define ZINV_PIX_NOT_PD 1u     /* det <= 0 or not finite: Z is not positive definite */
#define ZINV_PIX_RECOMPUTED 2u /* the pixel was recomputed in FP64 */

/* The ABI version this library implements (ZINV_ABI_VERSION). */
int zinv_abi_version(void);

/* Static string naming a return code. */
const char* zinv_status_string(int code);

/*
 * zinv_det -- Alg. 2 of the paper (§3.1): per pixel, the three real diagonal
 * and three complex upper cofactors (Eq. adjoint_elements), det as the real
 * part of the first-column cofactor expansion (Eq. det, Eq. detr), one
 * reciprocal t = 1/det, and Z^-1 = t * adj(Z) (Eq. inv_adjoint).
 *
 *   z      [9][ld] packed input (read only), n pixels.
 *   n      number of pixels, n >= 0 (n == 0 enqueues only the counter reset).
 *   ld     plane stride of z and zinv in floats, ld >= n.  With ld % 4 == 0 and
 *          16-byte aligned z, zinv, det (and 4-byte aligned status) the kernel
 *          moves four pixels per thread with 128-bit accesses; otherwise one.
 *   zinv   [9][ld] packed output: the upper triangle of Z^-1.  zinv == z (in
 *          place) is allowed; any other overlap with an input is not.
 *   det    [n] output: det Z.
 *   flags  ZINV_PLAIN, or ZINV_COMPENSATED and/or ZINV_FP64_RECOMPUTE.
 *   tau    threshold of ZINV_FP64_RECOMPUTE: a pixel is recomputed in FP64 when
 *          !(det > tau*a*d*f) (Hadamard: 0 < det <= a*d*f for positive definite
 *          Z), or when |det| is outside [2^-100, 2^100).  Must be finite and
 *          >= 0; ignored without the flag.
 *          Range: det scales with the cube of the entries.  Without the flag
 *          the FP32 routes need det and 1/det to be normal floats (entries
 *          roughly within 1e-12 .. 1e12); with it, pixels beyond that band are
 *          recomputed in FP64 and get the correctly rounded Z^-1 (det itself
 *          rounds to 0 or inf where it is outside the FP32 range).
 *   status [n] optional (NULL): per-pixel ZINV_PIX_* bits.
 *   counts [2] optional (NULL), device int64: overwritten with the number of
 *          pixels flagged ZINV_PIX_NOT_PD and ZINV_PIX_RECOMPUTED.
 */
int zinv_det(const float* z, int64_t n, int64_t ld, float* zinv, float* det, uint32_t flags,
             float tau, uint8_t* status, int64_t* counts, void* stream);

/*
 * chol_zinv_det -- the paper's baseline, Alg. 1 (§2.2): Z = L L^H with three
 * square roots and three reciprocals, T = L^-1, det = (l00 l11 l22)^2 and
 * Z^-1 = T^H T.  The paper's printed l21 is the conjugate of the correct one;
 * this kernel uses l21 = (conj(e) - l20 conj(l10)) / l11, which follows from
 * Z = L L^H.  Same layout, alignment rules and outputs as zinv_det; flags must
 * be ZINV_PLAIN (tau is ignored); status/counts report ZINV_PIX_NOT_PD.
 */
int chol_zinv_det(const float* z, int64_t n, int64_t ld, float* zinv, float* det,
                  uint32_t flags, float tau, uint8_t* status, int64_t* counts, void* stream);

/*
 * zinv_det_blockdiag -- multifrequency pixels (§5: with several bands the
 * matrices are block diagonal, each block Hermitian, and inverse and
 * determinant follow from Algorithm 2 applied to each diagonal block).  Pixel p
 * has nblocks (1..8) packed 3x3 blocks: block b's plane k at
 * z[(b*9 + k)*ld + p].  Outputs: zinv in the same layout (the diagonal blocks of
 * the inverse; the off-diagonal blocks are zero), det[p] = product of the
 * blocks' determinants.  flags, tau, status (OR over the blocks) and counts as
 * zinv_det; 128-bit path under the same alignment conditions.
 */
int zinv_det_blockdiag(const float* z, int nblocks, int64_t n, int64_t ld, float* zinv,
                       float* det, uint32_t flags, float tau, uint8_t* status, int64_t* counts,
                       void* stream);

/*
 * zinv_det_bwd -- backward of (Z^-1, det, log det) w.r.t. the nine packed reals
 * of Z, from the forward's saved outputs W = Z^-1 and det.  With G the
 * Hermitian matrix of the upstream packed gradient (G_ii = g_ii,
 * G_ij = (g_Re + i g_Im)/2 for i < j),
 *     M = -W G W + (g_det * det + g_logdet) * W,
 * and the output is [M00, 2Re M01, 2Im M01, 2Re M02, 2Im M02, M11, 2Re M12,
 * 2Im M12, M22] (dL = Re tr(M dZ); the factor 2 counts both off-diagonal
 * entries each packed real stands for).  The paper has no backward; this
 * differentiates Eq. inv_adjoint and Eq. det.
 *
 *   zinv    [9][ld] packed W (read only).
 *   det     [n] det Z (read only).
 *   g_zinv  [9][ld] upstream gradient of the packed W, or NULL (zero).
 *   g_det   [n] upstream gradient of det, or NULL (zero).
 *   g_logdet [n] upstream gradient of log det, or NULL (zero).
 *   g_z     [9][ld] output; may alias g_zinv exactly, nothing else.
 * 128-bit path when ld % 4 == 0 and every pointer is 16-byte aligned.
 */
int zinv_det_bwd(const float* zinv, const float* det, int64_t n, int64_t ld,
                 const float* g_zinv, const float* g_det, const float* g_logdet, float* g_z,
                 void* stream);

/*
 * multilook_zinv_det -- fused multilook and inverse: for every pixel p of an
 * H x W single-look image, the window covariance
 *     Z(p) = (1/N) sum_{k in win x win} S(p+k) S(p+k)^H      (boxcar, N = win^2)
 * (Eq. ZN, with S the column vector [S_HH, S_HV, S_VV]^T of §1), or
 *     Z(p) = sum_k w_k S(p+k) S(p+k)^H                         (weighted window),
 * with clamp-to-edge addressing at the image border, is formed on chip and
 * inverted by Algorithm 2 as in zinv_det.  Z is never written to memory.
 *
 *   s        complex64 single-look planes (read only): component i of pixel
 *            (y, x) at s[i*plane_ld + y*W + x] (interleaved re, im floats;
 *            8-byte aligned), plane_ld >= H*W in complex elements.
 *   win      window side: 3, 5 or 7 for the boxcar; any odd value up to 15
 *            with weights.
 *   weights  [win*win] device floats, row-major over (dy, dx) in [-r, r]^2,
 *            r = (win-1)/2, or NULL for the boxcar.
 *   zinv     [9][H*W] packed Z^-1 (plane stride H*W), det [H*W].
 *   flags, tau, status, counts  as zinv_det.
 */
int multilook_zinv_det(const float* s, int64_t H, int64_t W, int64_t plane_ld, int win,
                       const float* weights, float* zinv, float* det, uint32_t flags,
                       float tau, uint8_t* status, int64_t* counts, void* stream);

/*
 * nlm_wishart -- nonlocal-means filter of a packed covariance image with the
 * Wishart equal-looks distance, the workload the paper's introduction uses to
 * motivate fast inversion (§1: for every pixel a 23 x 23 search window of
 * determinant computations).  For pixels i, j:
 *     d(i, j) = ln det((Z_i + Z_j)/2) - (ln det Z_i + ln det Z_j)/2   (>= 0),
 *     w_ij    = exp(-looks * d(i, j) / h)   over the in-image j within `radius`,
 *     Z'_i    = sum_j w_ij Z_j / sum_j w_ij.
 * The per-pair determinant is computed by Algorithm 2's cofactor expansion
 * (method 0) or by Algorithm 1's Cholesky route (method 1), so the two can be
 * compared where arithmetic sets the time; method 2 is the compensated pair
 * determinant of nlm_stochastic (ZINV_NLM_COMPENSATED), for ill-conditioned
 * pixels.
 *
 *   z       [9][ld] packed input (read only), H x W pixels, positive definite.
 *   radius  search radius: 1, 2, 3, 5, 7, 11 (23 x 23 window) or 15.
 *   looks, h  positive and finite.
 *   z_out   [9][H*W] packed output (plane stride H*W); must not overlap z.
 */
int nlm_wishart(const float* z, int64_t H, int64_t W, int64_t ld, int radius, float looks,
                float h, int method, float* z_out, void* stream);

/*
 * nlm_stochastic -- the nonlocal-means filter of nlm_wishart with a choice of
 * stochastic distance between the pixels' complex Wishart laws of `looks`
 * looks (§1 lists the Kullback-Leibler, Hellinger, Renyi, Bhattacharyya,
 * triangular and harmonic divergences among the computations that need only
 * det Z and Z^-1).  Weights w_ij = exp(-d(i, j) / h), Z'_i as nlm_wishart, with
 * d (closed forms for equal looks, m = 3):
 *   ZINV_NLM_BHATTACHARYYA    d = L [ln det((Z_i + Z_j)/2) - (ln det Z_i + ln det Z_j)/2]
 *                             (equal to L [ln det((Z_i^-1 + Z_j^-1)/2) + (ln det Z_i
 *                             + ln det Z_j)/2]); the filter of nlm_wishart.
 *   ZINV_NLM_HELLINGER        d = 1 - exp(-d_Bhattacharyya)   (in [0, 1)).
 *   ZINV_NLM_KULLBACK_LEIBLER d = L [(tr(Z_i^-1 Z_j) + tr(Z_j^-1 Z_i))/2 - 3], the mean
 *                             of the two directed divergences; Z^-1 of every pixel
 *                             by Algorithm 2 (compensated cofactors and det).
 *   ZINV_NLM_RENYI            d = L/(1-b) [(ln det((1-b) Z_i + b Z_j) + ln det(b Z_i
 *                             + (1-b) Z_j))/2 - (ln det Z_i + ln det Z_j)/2], the mean
 *                             of the two directed divergences of order b = `order`
 *                             (b = 1/2 gives twice the Bhattacharyya distance; b -> 1
 *                             tends to Kullback-Leibler); two determinants per pair.
 *   order     the Renyi order b, in (0, 1); unused by the other distances.
 *   method    the per-pair determinants of Bhattacharyya, Hellinger and Renyi:
 *             ZINV_NLM_ADJUGATE (Algorithm 2) or ZINV_NLM_CHOLESKY (Algorithm 1);
 *             for Bhattacharyya and Hellinger also ZINV_NLM_COMPENSATED:
 *             Algorithm 2 on the exact pair sum (hi + lo per entry) with Dot2
 *             cofactors and det plus the first-order term of lo, which keeps
 *             the weights accurate for ill-conditioned pixels (cond ~1e6,
 *             where the FP32 rounding of the pair sum alone can move the plain
 *             det by its own size), at about 5x the plain filter's time
 *             (2.3x Algorithm 1's).
 *             Kullback-Leibler takes no per-pair determinant and accepts
 *             ZINV_NLM_ADJUGATE only.
 *   z, H, W, ld, radius, looks, h, z_out, stream  as nlm_wishart.
 * Returns ZINV_ERR_ARG for an unknown distance or method, a method the
 * distance does not take, or a Renyi order outside (0, 1), before any device
 * work.
 */
#define ZINV_NLM_ADJUGATE 0
#define ZINV_NLM_CHOLESKY 1
#define ZINV_NLM_COMPENSATED 2
#define ZINV_NLM_BHATTACHARYYA 0
#define ZINV_NLM_HELLINGER 1
#define ZINV_NLM_KULLBACK_LEIBLER 2
#define ZINV_NLM_RENYI 3
int nlm_stochastic(const float* z, int64_t H, int64_t W, int64_t ld, int radius, float looks,
                   float h, int distance, float order, int method, float* z_out, void* stream);

/*
 * Wishart change statistic between two dates with a learnable window (the
 * likelihood-ratio change test the paper lists among the consumers of det Z and
 * Z^-1, §1).  For every pixel p of two co-registered H x W single-look images
 * and t = 1, 2:
 *     Z_t(p) = sum_k w_k S_t(p+k) S_t(p+k)^H      (win x win window, clamp-to-edge)
 *     q(p)   = ln det Z1 + ln det Z2 - 2 ln det((Z1 + Z2)/2)   (<= 0; 0 iff Z1 = Z2)
 *     L      = sum_p q(p).
 * Determinants and inverses follow Algorithm 2 with compensated (Dot2)
 * arithmetic.  Deterministic: per-tile FP64 partial sums in the workspace,
 * added in a fixed order (no float atomics); repeated calls give the same bits.
 *
 *   s1, s2    complex64 single-look images, layout as multilook_zinv_det.
 *   win       3, 5 or 7.
 *   weights   [win*win] device floats, row-major over (dy, dx), r = (win-1)/2;
 *             positive weights keep Z positive definite (needs >= 3 distinct looks).
 *   ws, ws_bytes  caller-owned device workspace of at least
 *             wishart_workspace_bytes(H, W, win) bytes (8-byte aligned); its
 *             contents are scratch, overwritten by every call.
 *
 * wishart_stat_fwd: q_map [H*W] device floats or NULL; d_loss: one device double,
 *   overwritten with L.  A window whose Z is not positive definite gives NaN.
 * wishart_stat_bwd: recomputes every Z_t from s (nothing is kept from the
 *   forward) and writes grad_weights[k] = g * dL/dw_k (win*win device floats),
 *   g = *d_grad_loss (a device double; NULL means 1), where
 *     dL/dw_k = sum_p sum_t S_t(p+k)^H M_t(p) S_t(p+k),
 *     M_t = Z_t^-1 - 2 (Z1 + Z2)^-1.
 */
size_t wishart_workspace_bytes(int64_t H, int64_t W, int win);
int wishart_stat_fwd(const float* s1, const float* s2, int64_t H, int64_t W, int64_t plane_ld,
                     int win, const float* weights, float* q_map, double* d_loss, void* ws,
                     size_t ws_bytes, void* stream);
int wishart_stat_bwd(const float* s1, const float* s2, int64_t H, int64_t W, int64_t plane_ld,
                     int win, const float* weights, const double* d_grad_loss,
                     float* grad_weights, void* ws, size_t ws_bytes, void* stream);

/*
 * The change statistic with saved window covariances: the autograd trade of
 * memory for recomputation.  wishart_stat_fwd_save is wishart_stat_fwd that
 * also writes both dates' Z (the forward's window sums, from registers) to
 * z_saved; wishart_stat_bwd_saved takes them instead of recomputing the window
 * sums: a point-wise kernel forms M_t = Z_t^-1 - 2 (Z1 + Z2)^-1 of every pixel
 * (three compensated inverses), then a correlation kernel adds the weight
 * gradient.  Same
 * arithmetic and order as wishart_stat_bwd: the same bits.
 *
 *   z_saved   [18][H*W] device floats (72 bytes per pixel,
 *             wishart_saved_bytes(H, W)): date 1's nine packed planes, then
 *             date 2's, plane stride H*W, 4-byte aligned (16-byte aligned with
 *             W % 4 == 0 takes 128-bit stores).  Written by the forward, read
 *             by the backward (not modified), owned by the caller; valid for a
 *             backward with the same s1, s2, H, W, win and weights.
 *   ws, ws_bytes  wishart_stat_fwd_save: as wishart_stat_fwd.
 *             wishart_stat_bwd_saved: at least
 *             wishart_bwd_saved_workspace_bytes(H, W, win) bytes, 8-byte
 *             aligned (per-tile partials, then the packed M of every pixel;
 *             16-byte aligned with W % 4 == 0 takes 16-byte copies of M).
 *   other arguments as wishart_stat_fwd / wishart_stat_bwd (the backward
 *   takes no weights: they entered through Z).
 * Images of more than 2^56 pixels are refused (ZINV_ERR_ARG), as are the
 * argument errors of the recomputing calls; the size queries return 0 there.
 */
size_t wishart_saved_bytes(int64_t H, int64_t W);
size_t wishart_bwd_saved_workspace_bytes(int64_t H, int64_t W, int win);
int wishart_stat_fwd_save(const float* s1, const float* s2, int64_t H, int64_t W,
                          int64_t plane_ld, int win, const float* weights, float* q_map,
                          double* d_loss, float* z_saved, void* ws, size_t ws_bytes,
                          void* stream);
int wishart_stat_bwd_saved(const float* s1, const float* s2, int64_t H, int64_t W,
                           int64_t plane_ld, int win, const float* z_saved,
                           const double* d_grad_loss, float* grad_weights, void* ws,
                           size_t ws_bytes, void* stream);

/*
 * wishart_stat_fwd_noalloc -- wishart_stat_fwd for callers that cannot pass a
 * device workspace: code running inside a host application or framework that
 * owns every device allocation (so cudaMalloc is unavailable or would fragment
 * its pool), or a processing loop that must not allocate once it is running.
 * The paper has no counterpart; this is a property of the library, not of the
 * method.
 *
 * Same arguments and results as wishart_stat_fwd without ws and ws_bytes; the
 * caller still passes the inputs and outputs.  The per-tile partial sums go to
 * a fixed 1 MiB device array inside libzinv.so, held by every GPU that loads the
 * library until the process exits.  Maximum size: ceil(W/32) * ceil(H/16) <=
 * 131072 tiles (e.g. 8192 x 8192 pixels); larger images return ZINV_ERR_ARG.
 * The call allocates no device memory.  Its first call on a device looks up the
 * array's device address for that device; make that first call before any
 * stream capture.  Every call uses the same array: calls that overlap on the
 * GPU (other streams, other threads) race and give wrong results.  Nothing in
 * the array needs to start at zero: each call writes every slot it reads.
 */
int wishart_stat_fwd_noalloc(const float* s1, const float* s2, int64_t H, int64_t W,
                             int64_t plane_ld, int win, const float* weights, float* q_map,
                             double* d_loss, void* stream);

/*
 * zinv_det_host -- zinv_det over HOST buffers (the paper's §4.3: data larger than
 * device memory is fed through the GPU in pieces, processed and pulled back).
 * When all three host buffers are GPU-accessible (page-locked memory from
 * cudaHostAlloc or pinned torch tensors, or cudaHostRegister'ed memory) and
 * ZINV_HOST_STAGED is not set, the kernel reads and writes them directly over
 * the CPU-GPU link (one launch, no copies; d_ws may be NULL).  Otherwise the
 * image is staged in chunks through the workspace: copies in, kernel and
 * copies out of successive chunks overlap on three streams the library creates
 * once per device.
 *
 *   z_host, zinv_host, det_host  host buffers in the layout above (zinv_host
 *          [9][ld], det_host [n]); page-locked for the copies to be asynchronous.
 *   d_ws, ws_bytes  caller-owned device workspace for the staged way, at least
 *          zinv_det_host_workspace_bytes(chunk) bytes for some chunk >= 1;
 *          the chunk is the largest that fits (a multiple of 4 pixels when
 *          ws_bytes allows).
 *   flags, tau  as zinv_det, plus ZINV_HOST_STAGED.
 * The call is asynchronous with respect to the host and ordered after prior
 * work on `stream`; later work on `stream` waits for the last chunk to land.
 * The host buffers must stay valid until then.  Not re-entrant: two calls on
 * the same device must not overlap in time.  If a staged call fails after it
 * has queued copies, `stream` still waits for everything it queued (or the
 * call waits on the host before returning), so synchronizing `stream` after
 * an error is enough before the host buffers are freed or reused.
 */
size_t zinv_det_host_workspace_bytes(int64_t chunk);
int zinv_det_host(const float* z_host, int64_t n, int64_t ld, float* zinv_host,
                  float* det_host, uint32_t flags, float tau, void* d_ws, size_t ws_bytes,
                  void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ZINV_H */
