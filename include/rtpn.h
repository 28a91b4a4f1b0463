/*
 * rtpn.h -- C ABI of the GB300 staggered-grid P_N time step.
 *
 * The library advances the real 3D P_N moment system of Eq. (3) of Berghoff, Frank & Seibold,
 * "Massively Parallel Stencil Strategies for Radiation Transport Moment Model Simulations"
 * (arXiv 2004.02833):
 *
 *     du/dt + Mx du/dx + My du/dy + Mz du/dz + C u = q ,
 *
 * on a box of nx * ny * nz cells with the StaRMAP staggered-grid method of Section 2.1: the
 * (N+1)^2 moments live on 8 staggered sub-grids, x/y/z derivatives are two-point half-grid
 * differences, each class ("even"/"odd" grids) is advanced with the dual class frozen by the exact
 * scalar solution of Eq. (5), and one step is the Strang splitting of Eq. (6).
 *
 * Conventions used by every entry point:
 *   - A component index c at this interface is c = l*l + l + m (l = 0..N, m = -l..l).  The real
 *     basis has no Condon-Shortley phase: m > 0 is sqrt(2) N_l^m P_l^m(mu) cos(m phi), m < 0 the
 *     matching sin(|m| phi), m = 0 is N_l^0 P_l(mu), polar axis z.
 *   - Per-cell arrays are [z][y][x] with x fastest (nx*ny*nz values).  A full state is
 *     [c][z][y][x] ((N+1)^2 * nx*ny*nz values).  A component with sub-grid slot g = 1 along an axis
 *     sits at (i + 1/2) h on that axis, g = 2 at (i + 1) h (0-based cell i; h the cell size along
 *     that axis, see rtpn_set_spacing).
 *   - `where` says whether a caller pointer is host (RTPN_HOST) or device (RTPN_DEVICE) memory.
 *     Caller buffers are never retained.  Calls with host pointers synchronise before returning;
 *     calls with device pointers are ordered on the context stream and return without waiting.
 *   - Every call returns RTPN_OK (0) or a negative RTPN_E* code; rtpn_last_error() gives the
 *     context's last message.  A failed call leaves the state as it was unless stated otherwise.
 *   - The library owns all device memory it allocates; nothing here takes torch types.
 */
#ifndef RTPN_H
#define RTPN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define RTPN_OK            0
#define RTPN_EINVAL       -1   /* bad argument (N < 0, dims < 1, h <= 0, bad enum, NULL, ...)     */
#define RTPN_ECFL         -2   /* dt >= min(h)/3: outside the proven range of Section 2.1         */
#define RTPN_ENOMEM       -3   /* device allocation failed                                        */
#define RTPN_ECUDA        -4   /* a CUDA call failed (message in rtpn_last_error)                 */
#define RTPN_ETIMEOUT     -5   /* a bounded device wait ran out                                   */
#define RTPN_ENONFINITE   -6   /* NaN or Inf found by a diagnostic                                */
#define RTPN_EUNSUPPORTED -7   /* valid request the compiled library does not implement          */
#define RTPN_ESTATE       -8   /* call out of order (e.g. rtpn_step before rtpn_set_media)        */

/* ---- boundaries ---- */
#define RTPN_BC_PERIODIC 0     /* Section 2.1: indices wrap                                       */
#define RTPN_BC_VACUUM   1     /* every out-of-domain value of every component reads as 0        */

/* ---- storage precision of the state (arithmetic is FP32 for FP32/BF16, FP64 for FP64) ---- */
#define RTPN_FP64 0
#define RTPN_FP32 1
#define RTPN_BF16 2

/* ---- data types of caller arrays ---- */
#define RTPN_DTYPE_F64 0
#define RTPN_DTYPE_F32 1

/* ---- memory kinds of caller pointers ---- */
#define RTPN_HOST   0
#define RTPN_DEVICE 1

/* ---- step kernels ---- */
#define RTPN_KERNEL_AUTO    0  /* fastest available for (N, precision)                            */
#define RTPN_KERNEL_GENERIC 1  /* any N and precision: one thread per cell, partner-table gather   */
#define RTPN_KERNEL_WINDOW  2  /* FP32/BF16, compiled N: register-window scatter over m-columns  */
#define RTPN_KERNEL_STAGE   3  /* FP32/BF16, compiled N, nx*elem a multiple of 16 B: column loop
                                  with TMA-staged shared-memory tiles, persistent CTAs          */
#define RTPN_KERNEL_FUSED   4  /* FP32/BF16, compiled N (1, 3, 5, 7, 9): each (even full step, odd
                                  step) pair of rtpn_step in one z-streaming pass between two
                                  state buffers; single substeps use the window kernel          */

typedef struct rtpn_ctx rtpn_ctx;

typedef struct rtpn_info {
    int N;                 /* moment order                                   */
    int n_c;               /* (N+1)^2 components                             */
    int n_even, n_odd;     /* components on even / odd grids (even = even l) */
    int nx, ny, nz;
    int bc, precision, kernel;
    double h, dt;
    size_t state_bytes;    /* device bytes of the moment state               */
    size_t factor_bytes;   /* device bytes of the per-cell substep factors   */
    long long steps_done;  /* full steps taken since the last set_moments    */
    int tile[3];           /* CTA tile of the active kernel (0 = not tiled)  */
    int depth;             /* stage buffers of the staged kernel (1 = other) */
    double hy, hz;         /* cell sizes along y and z (h is the one along x) */
} rtpn_info;

/* Library version (major*10000 + minor*100 + patch). */
int rtpn_version(void);

/* Static text for a status code. */
const char* rtpn_strerror(int code);

/*
 * Component metadata (host only, no device needed).  For order N and interface index c, returns
 * l, m, the sub-grid slots (x, y, z; each 1 or 2) and the class (0 = even grid, 1 = odd grid).
 * Placement rule of Section 2.1: u_0 on G111 and every derivative along d switches slot d; the
 * slots equal the reflection parities of the real basis function (slot 1 = even parity).
 * Any output pointer may be NULL.  RTPN_EINVAL if N < 0 or c out of range.
 */
int rtpn_component_info(int N, int c, int* l, int* m, int slots[3], int* cls);

/*
 * Dense coupling matrix M_axis (axis 0 = x, 1 = y, 2 = z) of Eq. (3) in interface order, FP64,
 * row-major n_c * n_c, written to caller host memory `out`.  Entries are the closed forms of
 * int Omega_d Y_a Y_b dOmega from the Legendre ladder relations (the coefficients the kernels
 * use).  RTPN_EINVAL if N < 0 or N > 63, axis out of range or out == NULL.
 */
int rtpn_coupling_dense(int N, int axis, double* out);

/*
 * Create a context for order N on nx*ny*nz cells of size h, boundary bc, storage precision, time
 * step dt (dt <= 0 selects 0.3 h).  Allocates the state (zeroed) and the factor tables on the
 * current CUDA device and uses the legacy default stream until rtpn_set_stream.
 * Errors: RTPN_EINVAL (N < 0 or N > 63, dims < 1, h <= 0, bad bc/precision, out == NULL),
 * RTPN_ECFL (dt >= h/3, Section 2.1), RTPN_ENOMEM, RTPN_ECUDA.  *out is NULL on failure.
 */
int rtpn_create(rtpn_ctx** out, int N, int nx, int ny, int nz, double h, int bc,
                int precision, double dt);

/* Free every device allocation of the context (after synchronising its stream). NULL is a no-op. */
int rtpn_destroy(rtpn_ctx* ctx);

/* Anisotropic scattering (Section 2: Sigma_tl = Sigma_a + Sigma_s0 - Sigma_sl per moment order l):
 * Sigma_sl = f[l] * sigma_s with f[0] = 1 (sigma_s is Sigma_s0) and -1 <= f[l] <= 1, count = N + 1
 * (e.g. f[l] = g^l for a Henyey-Greenstein phase function); f = NULL or count = 0 restores isotropic
 * scattering.  Components of order l then decay by sigma_a + (1 - f[l]) sigma_s (mean over the
 * cells adjacent to their sub-grid point, as for isotropic media).  Runs on the generic kernel and,
 * for N <= 15 in FP32/BF16, on the window kernel (each target reads its own order's factor planes):
 * RTPN_EUNSUPPORTED if another kernel is selected explicitly, for a batch instance, and later for
 * rtpn_adjoint; RTPN_KERNEL_AUTO moves to the window kernel where it applies, else to the generic
 * one.  Allocates 32 (N + 1) more factor
 * planes (RTPN_ENOMEM leaves the context unchanged) and recomputes the factors of the media already
 * set; synchronises the context stream.  RTPN_EINVAL on a bad count or f. */
int rtpn_set_scattering(rtpn_ctx* ctx, const double* f, int count);

/* Cell sizes along x, y and z (rtpn_create sets all three to h): the differences of Section 2.1
 * divide by the cell size of their own axis, and dt must stay below min(hx, hy, hz)/3 (RTPN_ECFL
 * otherwise; the spacing is then unchanged).  Non-cubic cells run on the staged and generic kernels
 * (and the adjoint): RTPN_EUNSUPPORTED if the window or fused kernel is selected explicitly, and
 * for a batch instance (its spacing is fixed at rtpn_batch_create); RTPN_KERNEL_AUTO moves to the
 * staged or generic kernel.  Rebuilds the
 * coupling tables (synchronises the context stream); the media factors do not depend on h. */
int rtpn_set_spacing(rtpn_ctx* ctx, double hx, double hy, double hz);

/* Order all later work of the context on `stream` (a cudaStream_t; NULL = legacy default). */
int rtpn_set_stream(rtpn_ctx* ctx, void* stream);

/* Select the step kernel (RTPN_KERNEL_*) and its CTA tile (tile_x * tile_y * tile_z threads, one
 * cell each; all 0 = default).  RTPN_KERNEL_WINDOW: the tile must hold a multiple of 32 threads, at
 * most 256 (RTPN_EINVAL); default 32 x 4 x 2.  RTPN_KERNEL_STAGE: the tile must be one compiled for
 * N (RTPN_EUNSUPPORTED otherwise).  RTPN_KERNEL_FUSED: the CTA tile is fixed at 32 x 8 cells, so
 * tile_x and tile_y must be 0 (or 32 and 8); tile_z is the number of z planes a CTA streams through
 * (0 = one wave of resident CTAs).  Selecting it allocates a second state buffer (RTPN_ENOMEM if
 * that fails); RTPN_EUNSUPPORTED for a batch instance.
 * RTPN_KERNEL_AUTO picks STAGE (for N >= 15), then WINDOW, then GENERIC; with non-cubic cells STAGE
 * (any compiled N), else GENERIC; with anisotropic scattering GENERIC.
 * RTPN_EUNSUPPORTED if the kernel is not compiled for (N, precision, nx) or does not take the
 * context's cells or scattering; the previous selection then stays. */
int rtpn_set_kernel(rtpn_ctx* ctx, int kernel, int tile_x, int tile_y, int tile_z);

/* As rtpn_set_kernel, and for RTPN_KERNEL_STAGE the pipeline depth: the number of shared-memory
 * stage buffers, of which all but one hold copies in flight (2..8; 0 = any compiled).  The staged
 * kernel runs two threads per cell of the tile (one per target type) plus one producer warp.
 * RTPN_EINVAL for a depth outside 0..8, RTPN_EUNSUPPORTED if no staged variant is compiled for
 * (N, tile, depth). */
int rtpn_set_kernel_ex(rtpn_ctx* ctx, int kernel, int tile_x, int tile_y, int tile_z, int depth);

/*
 * Media: per-cell sigma_a >= 0, sigma_s >= 0 and source q (added to the u_0 equation), each
 * [z][y][x] of type dtype at `where`.  On the device, in FP64, each sub-grid point takes the mean
 * of sigma over its 2^k adjacent cells (periodic: wrapped; vacuum: in-domain cells only), then
 * c = sigma_a (u_0) or sigma_a + sigma_s (all others) and the factors of Eq. (5),
 * alpha = exp(-c tau) and beta = tau E(-c tau), for tau = dt and dt/2, rounded to the storage
 * precision.  May be called again between steps: media and source then vary in time piecewise
 * constantly at step resolution (the time dependence of the coefficients in Eq. 1), stream-ordered
 * after the steps already enqueued.  RTPN_EINVAL on NULL or bad enums; negative sigma is not
 * checked.
 */
int rtpn_set_media(rtpn_ctx* ctx, const void* sigma_a, const void* sigma_s, const void* q,
                   int dtype, int where);

/* Full state [c][z][y][x] in interface order, converted to the storage precision. */
int rtpn_set_moments(rtpn_ctx* ctx, const void* u, int dtype, int where);
/* Copy the full state out ([c][z][y][x], interface order) into a caller-owned buffer. */
int rtpn_get_moments(rtpn_ctx* ctx, void* u, int dtype, int where);
/* One component (interface index c), [z][y][x]. */
int rtpn_set_component(rtpn_ctx* ctx, int c, const void* field, int dtype, int where);
int rtpn_get_component(rtpn_ctx* ctx, int c, void* field, int dtype, int where);
/* Set every moment to 0. */
int rtpn_zero_moments(rtpn_ctx* ctx);

/*
 * Advance k >= 0 full steps of Eq. (6).  The k steps run as one odd half step, k-1 pairs of
 * (even full step, odd full step) -- two adjacent odd half steps merged, exact because the even
 * class is frozen between them (Eq. 5) -- then an even full step and an odd half step.
 * Asynchronous on the context stream; the launch sequence is replayed from a cached CUDA graph.
 * With RTPN_KERNEL_FUSED each (even full step, odd step) pair, the last one with the odd half step,
 * is one pass from one state buffer into the other (the context keeps track of which holds the
 * state; get/set/sum see the current one).  When the context stream is being captured by the
 * caller, rtpn_step runs the two-pass schedule in place instead, so the captured pointers stay
 * valid on replay.
 * RTPN_ESTATE if media were never set.
 */
int rtpn_step(rtpn_ctx* ctx, int k);

/*
 * One substep S^cls_tau of Eq. (5) alone: every component of class cls (0 even, 1 odd) is advanced
 * with the dual class frozen, tau = dt (half = 0) or dt/2 (half = 1).  rtpn_step(k) is the
 * schedule of these passes given above; this entry lets a caller run or time a single pass.
 * Half steps exist for the odd class only (RTPN_EINVAL for cls = 0 with half = 1).
 * Asynchronous; RTPN_ESTATE without media.
 */
int rtpn_substep(rtpn_ctx* ctx, int cls, int half);

/*
 * Halo exchange between the blocks of a decomposed domain (Section 3: each block of the
 * block-structured grid keeps one halo layer per face, refreshed from its neighbours between the
 * sweeps).  Copies z-planes [src_z, src_z + nz) of every component of class cls (0 even, 1 odd,
 * -1 both) from src's state into planes [dst_z, dst_z + nz) of dst's, device to device in one
 * strided copy.  The contexts must share N, precision, nx and ny (and the device); the planes must
 * lie inside both grids and not overlap within one context.  Ordered on dst's stream after the work
 * queued on src's stream, and src's later work waits for it (when the streams differ).
 * Asynchronous; RTPN_EINVAL on a mismatch or out-of-range planes.
 */
int rtpn_copy_planes(rtpn_ctx* dst, int dst_z, rtpn_ctx* src, int src_z, int nz, int cls);

/* Sum of u_0 over all cells, accumulated in FP64 in a fixed order (deterministic).
 * Writes the host double *out; synchronises. */
int rtpn_sum_u0(rtpn_ctx* ctx, double* out);

/* Number of non-finite values in the state (host *out); synchronises.  Returns RTPN_ENONFINITE
 * when the count is nonzero (the count is still written). */
int rtpn_count_nonfinite(rtpn_ctx* ctx, long long* out);

/*
 * FP64 sum of n values of a device array x (dtype RTPN_DTYPE_F64 or RTPN_DTYPE_F32), written to the
 * device double *out, ordered on `stream` (a cudaStream_t; NULL = legacy default stream).  The
 * paper has no counterpart; this entry point is for callers that cannot allocate device memory at
 * the point where they need a sum -- code running while a framework's caching pool owns the
 * device memory (a private cudaMalloc can fail there or fragment the pool), or a time-critical
 * loop where cudaMalloc / cudaFree would synchronise the whole device.  It allocates nothing: its
 * scratch is a file-scope device array of 2^16 FP64 partial sums (512 KB) that every GPU which
 * loads this library holds until the process exits, so n is limited to 2^30 values (RTPN_EINVAL
 * beyond, with the reason in rtpn_last_error(NULL)).  The sum is taken in a fixed order and is
 * reproducible.  The first call on a device looks up the scratch's device address (again after a
 * device reset gives the device a new context), so make that first call before any stream capture.  Every call shares the one scratch array and each call
 * overwrites the partials it reads (nothing has to start at zero); calls that overlap on the GPU
 * (on streams with no ordering between them) race and give wrong sums.  Asynchronous; RTPN_EINVAL
 * on NULL pointers, n < 0 or a bad dtype; RTPN_ECUDA if a launch fails.
 */
int rtpn_sum_static(const void* x, int dtype, long long n, double* out, void* stream);

/*
 * Discrete adjoint (gradients of a detector functional).  Starting from the context's current state
 * u(0) and media, runs k steps of Eq. (6) and returns
 *     J = sum over cells of w * u_0(after k steps)          (host double *J)
 * and dJ/dsigma_a, dJ/dsigma_s, dJ/dq per cell ([z][y][x], FP64, host or device per out_where).
 * Each substep u_A' = alpha u_A + beta r_A (Eq. 5) is pulled back exactly: lam_A <- alpha lam_A,
 * lam_B <- lam_B - K^T (beta lam_A) with the transposed staggered stencil, and the media collect
 * lam (dalpha/dc u + dbeta/dc r) at the staggered points, spread to the cells through the
 * transpose of the point mean, plus beta_0 lam_0 for q.  States are checkpointed every ckpt_every
 * steps and each segment is recomputed forward before its backward sweep.
 * Schedules: with the staged kernel active (FP32) every segment runs the merged form of its steps
 * (odd half pass, even and odd full passes, closing odd half pass: the literal step up to rounding)
 * with each pass written out of place, device memory ~ (k/ckpt_every + ckpt_every + 4) states;
 * otherwise the steps are taken literally (odd half, even full, odd half substeps: the schedule
 * the oracle's discrete adjoint transposes), device memory ~ (k/ckpt_every + 3 ckpt_every + 4)
 * states.  w is [z][y][x] of dtype at `where`.  Afterwards the context holds u(k).  FP64 and FP32
 * storage (RTPN_EUNSUPPORTED for BF16); RTPN_ESTATE without media; RTPN_ENOMEM if the states do
 * not fit; RTPN_ETIMEOUT if a staged kernel's bounded wait ran out.  Synchronises.
 */
int rtpn_adjoint(rtpn_ctx* ctx, const void* w, int dtype, int where, int k, int ckpt_every,
                 double* g_sa, double* g_ss, double* g_q, int out_where, double* J);

/*
 * Frees the work buffers rtpn_adjoint keeps between calls.  With the staged kernel active (FP32)
 * the checkpoints, segment states, multipliers and tensor maps of a call stay allocated on the
 * context's device (about (k/ckpt_every + ckpt_every + 4) states), so that the next call with the
 * same or a smaller k/ckpt_every layout neither allocates nor rebuilds its tensor maps (the
 * backward of a training loop); rtpn_destroy frees them too.  Not from the paper: workspace
 * management of this library.  Waits for the context's stream first.  RTPN_ECUDA if the free
 * fails; a context without kept buffers returns RTPN_OK.
 */
int rtpn_adjoint_release(rtpn_ctx* ctx);

/*
 * The detector functional that rtpn_adjoint differentiates, on the current state:
 *     J = sum over cells of w * u_0
 * accumulated in FP64 in a fixed order (1024 block partials, then one block; deterministic).  The
 * paper defines no detector; this is the functional of the adjoint form.  w is [z][y][x] of dtype
 * (RTPN_DTYPE_F64 / _F32) at `where`; J is one double at J_where (RTPN_HOST: synchronises;
 * RTPN_DEVICE: ordered on the context's stream, nothing waits).  RTPN_EINVAL on NULL pointers or
 * a bad dtype/where.
 */
int rtpn_detector(rtpn_ctx* ctx, const void* w, int dtype, int where, double* J, int J_where);

/* ======================================================================== batched form
 * Many independent instances of uneven order N and grid size advanced together.  Each pass of the
 * merged Strang schedule (see rtpn_step) is ONE persistent kernel launch over the tiles of every
 * instance (CTAs draw tiles from a work counter, largest orders first); k-step sequences are
 * replayed from cached CUDA graphs.  Storage FP32 or BF16; orders 1, 3, 5, 7, 9, 15.
 */
typedef struct rtpn_batch rtpn_batch;

/* Create `count` instances: per-instance arrays N, nx, ny, nz, h, bc and dt (dt may be NULL:
 * 0.3 h each).  Every instance gets its own context (see rtpn_batch_instance).
 * RTPN_EUNSUPPORTED for an order outside {1,3,5,7,9,15} or precision RTPN_FP64; otherwise the
 * errors of rtpn_create.  *out is NULL on failure. */
int rtpn_batch_create(rtpn_batch** out, int count, const int* N, const int* nx, const int* ny,
                      const int* nz, const double* h, const int* bc, const double* dt,
                      int precision);
int rtpn_batch_destroy(rtpn_batch* b);
/* Number of instances (RTPN_EINVAL for NULL). */
int rtpn_batch_count(const rtpn_batch* b);
/* The context of instance i, owned by the batch (do not destroy it): use it for set_media,
 * set/get_moments, sum_u0 and the other per-instance calls.  NULL if i is out of range. */
rtpn_ctx* rtpn_batch_instance(rtpn_batch* b, int i);
/* Order the batch's work (and every instance's) on `stream` (NULL = the batch's own stream). */
int rtpn_batch_set_stream(rtpn_batch* b, void* stream);
/* CTA tile of the grouped kernel (threads a multiple of 32, at most 256); default 32 x 4 x 2. */
int rtpn_batch_set_tile(rtpn_batch* b, int tile_x, int tile_y, int tile_z);
int rtpn_batch_get_tile(const rtpn_batch* b, int* tile_x, int* tile_y, int* tile_z);
/* Advance every instance k steps with one grouped launch per pass.  RTPN_ESTATE if some instance
 * has no media. */
int rtpn_batch_step(rtpn_batch* b, int k);
/* The same k steps as a loop of per-instance launches of the single-instance kernel (the
 * comparison baseline for the grouped launch). */
int rtpn_batch_step_looped(rtpn_batch* b, int k);
int rtpn_batch_synchronize(rtpn_batch* b);
const char* rtpn_batch_last_error(const rtpn_batch* b);

/* ======================================================================== autotuner
 * Pick the configuration of the active kernel by timing candidates on the object's own data: CTA
 * tiles of the register-window kernel (a multiple of 32 threads, at most 256), or the compiled
 * (tile, stage depth) variants of the staged kernel.  The state is copied aside first and restored,
 * so the moments are unchanged (needs device memory for one copy of the state: RTPN_ENOMEM if absent).
 * The best tile is applied, written to tile[3] and its time to *ms (one even + odd pass pair for a
 * context, one rtpn_batch_step(b, 1) for a batch); either output may be NULL.  Results are cached
 * for the process per (orders, precision, boundary, grid, device) and, when the environment
 * variable RTPN_TUNE_CACHE names a file, kept there across processes.  Synchronises.
 * RTPN_ESTATE without media; RTPN_EUNSUPPORTED if neither the window nor the staged kernel is
 * active (a batch always runs the window kernel).
 */
int rtpn_autotune(rtpn_ctx* ctx, int reps, int tile[3], double* ms);
int rtpn_batch_autotune(rtpn_batch* b, int reps, int tile[3], double* ms);

/* Wait for all work on the context stream.  Returns RTPN_ETIMEOUT (and clears the flag) if a
 * bounded wait inside a staged kernel ran out since the last check; the context stays usable, but
 * the state of the pass that timed out is undefined (reload it). */
int rtpn_synchronize(rtpn_ctx* ctx);

/* Test hook for the timeout path: one staged pass of class cls in which one stage's copies are
 * deliberately never issued, with `wait_limit` mbarrier polls (each sleeps up to 2 us), so every
 * CTA's bounded wait must run
 * out, set the status word and leave.  The next rtpn_synchronize returns RTPN_ETIMEOUT.  Leaves the
 * state undefined.  RTPN_EUNSUPPORTED unless the staged kernel is active. */
int rtpn_test_wait_timeout(rtpn_ctx* ctx, int cls, long long wait_limit);

/* Context facts (host struct). */
int rtpn_get_info(const rtpn_ctx* ctx, rtpn_info* out);

/* Last error message of the context ("" if none). */
const char* rtpn_last_error(const rtpn_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* RTPN_H */
