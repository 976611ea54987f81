/*
 * spg.h - C ABI of the GB300 reweighted smoothing-proximal-gradient solver.
 *
 * The solver minimises, for each volume and each re-weighting round r,
 *
 *   F_r(x) = 1/2 sum_v w_v (x_v - b_v)^2                     data term (Sec. 2.2, Eq. 28;
 *                                                            the 1/2 of Eq. 31)
 *          + lambda_l1 sum_v om1_v |x_v|                     weighted l1 (Eq. 11)
 *          + lambda_tv sum_v omtv_v h_mu((Dx)_v)             weighted smoothed TV (Eq. 11, 14)
 *
 * over a real-space density x on an nx*ny*nz grid (Sec. 2.1, the vectorised
 * volume of Eq. 8). D is the backward difference of Eq. 12 (zero on the first
 * plane of each axis), h_mu is Nesterov's smoothing of the Euclidean norm
 * (Eq. 14), whose gradient z/max(mu,|z|) is Eq. 16, and D^T is Eq. 17. The
 * weights are re-set between rounds from the current iterate (Eq. 11, scaled
 * by eps as Sec. 2.5 prescribes):
 *
 *   om1_v = eps / (|x_v| + eps),   omtv_v = eps_tv / (|(Dx)_v| + eps_tv).
 *
 * Each iteration is one fused pass over the volume (Eq. 20 and Eq. 21 with
 * FISTA extrapolation; beta = 0 gives the paper's plain update):
 *
 *   y       = x_k + beta_k (x_k - x_{k-1})
 *   x_{k+1} = soft(y - tau grad f(y), tau lambda_l1 om1),
 *   grad f  = w (y - b) + lambda_tv D^T(omtv grad h_mu(D y)),
 *
 * with tau = 1/L, L = max w + 12 lambda_tv max(omtv) / mu (|D|^2 <= 12).
 *
 * Conventions (every entry point):
 *  - Volumes are dense float32 (or bfloat16 where stated) arrays in C order
 *    [nz][ny][nx], x fastest, no padding. Pointers may be device pointers or
 *    host pointers (pinned or pageable): copies use unified addressing. The
 *    library never frees a caller pointer and keeps none beyond the call,
 *    except where an entry point states otherwise (spg_grid_add reads device
 *    inputs in place, in stream order).
 *  - Work is enqueued on the CUDA stream given at creation (NULL: the
 *    context creates and owns a stream). Entry points that return host
 *    values synchronise that stream; the others are asynchronous.
 *  - Every call returns an spg_status; spg_last_error() gives a message. No
 *    C++ exception crosses this interface. There is no CPU fallback: without
 *    a usable CUDA device, spg_create fails with SPG_ECUDA.
 *  - One context is used by one host thread at a time.
 */
#ifndef SPG_H
#define SPG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spg_ctx spg_ctx;

typedef enum {
    SPG_OK = 0,
    SPG_EINVAL = -1,      /* bad argument (NULL, size, dtype, volume index, w <= 0 ...) */
    SPG_ENOMEM = -2,      /* device allocation failed */
    SPG_ECUDA = -3,       /* CUDA runtime / driver error */
    SPG_ENOTREADY = -4,   /* call order violated (e.g. iterate before set_data/reweight) */
    SPG_ENONFINITE = -5,  /* a non-finite objective value or input was detected */
    SPG_ETIMEOUT = -6,    /* a bounded device-side wait gave up (context stays usable) */
    SPG_ECHECK = -7       /* an index check of the checked build (-DSPG_CHECK) failed */
} spg_status;

typedef enum { SPG_F32 = 0, SPG_BF16 = 1 } spg_dtype;

/* SPG_FISTA: Beck-Teboulle extrapolation, restarted every round.
 * SPG_ISTA: beta = 0, the paper's Eq. 20-21 update as printed. */
typedef enum { SPG_FISTA = 0, SPG_ISTA = 1 } spg_momentum;

/* How the extrapolation pair is kept between iterations (float32 either way).
 * SPG_STORE_DELTA: x_k and the increment d_k = x_k - x_{k-1} as computed before
 *   x_k was rounded; 32 bytes of HBM traffic per voxel-iteration. The momentum
 *   term then carries no rounding of x, which keeps long float32 solves within
 *   about 1e-6 (relative L2) of exact arithmetic.
 * SPG_STORE_PREV: x_k and x_{k-1}; 28 bytes per voxel-iteration; the rounding
 *   of each stored iterate re-enters the momentum term (about 1e-5 after
 *   3 x 300 iterations on a 256^3 volume). */
typedef enum { SPG_STORE_DELTA = 0, SPG_STORE_PREV = 1 } spg_iterate_storage;

/* Per-volume problem description. eps/eps_tv set the weight scale of Eq. 11
 * (Sec. 2.5 multiplies the weights by eps so that a zero voxel gets weight 1). */
typedef struct {
    int nx, ny, nz;
    float lambda_l1;   /* alpha of Eq. 8-11 */
    float lambda_tv;   /* beta of Eq. 8-11 */
    float mu;          /* Nesterov smoothing parameter of Eq. 14 */
    float eps;         /* epsilon of Eq. 9/11 for the l1 weights */
    float eps_tv;      /* epsilon' of the TV weights (Sec. 2.5; the paper uses eps' <= eps) */
} spg_volume_params;

/* Context-wide options. Zero-initialised options are valid defaults. */
typedef struct {
    spg_dtype data_dtype;     /* storage of b and w on the device: SPG_F32 or SPG_BF16
                                 (arithmetic stays float32 either way) */
    spg_momentum momentum;    /* SPG_FISTA (default) or SPG_ISTA */
    int hist_every;           /* record F(x_k) every this many iterations; 0 = 1 */
    int hist_capacity;        /* entries kept in the history ring; 0 = 4096 */
    int max_iters_per_round;  /* length of the extrapolation table; 0 = 100000 */
    int tile;                 /* 0 = built-in choice, else an spg_tile_* code */
    int zchunk;               /* 0 = built-in choice, else planes per work item */
    int ctas_per_sm;          /* 0 = occupancy limit, else a cap */
    spg_iterate_storage iterate_storage;  /* SPG_STORE_DELTA (default) or SPG_STORE_PREV */
    int restart;              /* 0: fixed FISTA schedule (default); 1: gradient restart of the
                                 extrapolation (per volume, whenever <y_k - x_{k+1}, x_{k+1} - x_k> > 0,
                                 O'Donoghue and Candes 2015); decided on the device every iteration */
    int readings;             /* 0: the adopted readings of the paper; otherwise an OR of
                                 SPG_READ_* flags (below) */
} spg_options;

/* Alternative readings of the paper, for spg_options.readings. The adopted
 * reading (0) takes Eq. 12's backward differences, which vanish where the
 * neighbour lies outside the volume (the paper names no boundary), and puts
 * the TV weight inside the divergence, D^T(omtv grad h_mu(D x)), the gradient
 * of the weighted TV term of Eq. 11. The flags select instead:
 *   SPG_READ_FORWARD   forward differences x_{v+e_a} - x_v (and their adjoint);
 *   SPG_READ_PERIODIC  differences that wrap around the volume;
 *   SPG_READ_POST_DIV  the weight after the divergence, omtv D^T(grad h_mu(D x)),
 *                      as Eq. 20 prints it (not the gradient of any objective
 *                      unless omtv is constant).
 * They apply to the re-weighting (|D x|), the objective (TV term) and the
 * iteration.
 *
 * SPG_READ_FORWARD alone runs the fused kernels, on volumes held with every
 * axis reversed: with R that reversal, forward differences are -R D_b R, and
 * the Huber term, the weights, the data and l1 terms commute with R, so the
 * forward-difference solve of (b, w) is R applied to the backward-difference
 * solve of (R b, R w). Every volume is reversed as it enters the context
 * (spg_set_data, spg_set_x, spg_set_anchor, spg_set_state, the gradient given
 * to spg_backward) and as it leaves (spg_get_x, spg_get_state, spg_unrolled's
 * x_K, spg_backward's gradients), so callers see their own orientation;
 * reading a volume out reverses the context's copy twice on its stream. Every
 * entry point of the real-space data term is available, at the adopted
 * path's speed; the Fourier-domain data term is not.
 *
 * Any other non-zero combination iterates with one plain kernel per step
 * instead of the fused one (it re-evaluates the differences at every
 * neighbour from global memory: about a ninth of the fused step's speed, a
 * path for comparing readings, not for production) and needs float32 data
 * with the real-space data term; restart, the certificate, the adjoint and
 * autotuning are not available for it. */
enum { SPG_READ_FORWARD = 1, SPG_READ_PERIODIC = 2, SPG_READ_POST_DIV = 4 };

/* Tile codes for spg_options.tile: x extent = 32 * vx, y extent = ty.
 * SPG_TILE_128x7_S4 is the 128x7 tile with a 4-deep copy pipeline, the
 * built-in choice for volumes that fill 128-wide tiles; SPG_TILE_128x7 is the
 * same tile with 3 stages. */
enum { SPG_TILE_AUTO = 0, SPG_TILE_128x8 = 1, SPG_TILE_128x4 = 2, SPG_TILE_64x8 = 3,
       SPG_TILE_64x4 = 4, SPG_TILE_128x7 = 6, SPG_TILE_128x15 = 7, SPG_TILE_64x7 = 8,
       SPG_TILE_128x7_S4 = 9 };

/* Create a solver for one volume (spg_create) or for nvol independent
 * volumes of possibly different sizes advanced together, one fused launch per
 * iteration for all of them (spg_create_batch; the paper refines classes and
 * the two gold-standard half-maps independently, Sec. 2 and Sec. 2.3).
 * params: one (or nvol) descriptions, copied. opt: NULL for defaults.
 * stream: a cudaStream_t or NULL. On success *out owns all device memory it
 * allocated (8 volumes of 4 bytes per voxel with SPG_STORE_DELTA, 7 with
 * SPG_STORE_PREV; b and w take 2 bytes with SPG_BF16). Errors: SPG_EINVAL for a
 * non-positive size or parameter, SPG_ENOMEM, SPG_ECUDA. */
spg_status spg_create(const spg_volume_params *params, const spg_options *opt, void *stream,
                      spg_ctx **out);
spg_status spg_create_batch(int nvol, const spg_volume_params *params, const spg_options *opt,
                            void *stream, spg_ctx **out);

/* Set the data volume b (the kernel-regression numerator over N(n), Eq. 28)
 * and the weight volume w (N(n), Eq. 28) of volume `vol`. src_dtype is the
 * dtype of the caller's arrays (SPG_F32 or SPG_BF16); they are converted with
 * round-to-nearest-even when the context stores the other dtype. w must be
 * finite and > 0, b finite: checked on the device, SPG_EINVAL / SPG_ENONFINITE
 * otherwise. Synchronises (it reduces max w in double precision). */
spg_status spg_set_data(spg_ctx *ctx, int vol, const void *b, const void *w, spg_dtype src_dtype);

/* Fourier-domain data term (Sec. 2.5, Eq. 31): replace the data term of a
 * single-volume context by 1/2 |y - D A x|^2, A the unitary 3-D DFT
 * (A x = FFT(x) / sqrt(nx ny nz)) and D = diag sqrt(N). y_half (complex64,
 * interleaved re/im) and N_half (float32, N >= 0) hold the real-to-complex
 * half spectrum [nz][ny][nx/2+1] of a Hermitian y and a centro-symmetric N;
 * host or device pointers, copied. Each iteration then transforms the
 * extrapolated point y_k (written by the previous fused step), forms the
 * residual spectrum N A y_k - D y and transforms back to get the data
 * gradient A^H (N A y_k - D y) for the fused step; for power-of-two nz from 8
 * to 4096 the transforms are per-plane ones and the library's own transform
 * along z, which forms the residual inside its pass: with power-of-two nx
 * from 128 to 1024 an own pass along the rows (the spectrum held kx-major in
 * between) and cuFFT along y over contiguous lines, otherwise cuFFT's
 * per-plane 2-D transforms (also chosen by SPG_ROW_PASS=0 in the
 * environment when the data are set); for other nz, 3-D cuFFT transforms
 * around a separate spectrum pass (volumes of fewer than 2^31 voxels; larger
 * ones need a power-of-two nz, else SPG_EINVAL). cuFFT is loaded at run time. L = max N + 12 lambda_tv max(omtv) / mu. Needs SPG_F32 data storage and
 * SPG_STORE_DELTA; certificate and adjoint are not available in this
 * mode. The objective history records the l1 and TV terms only (its data
 * column is 0); spg_objective returns all terms. spg_set_data switches back
 * to the real-space data term. Synchronises. */
spg_status spg_set_data_fourier(spg_ctx *ctx, int vol, const void *y_half, const float *N_half);

/* Kernel-regression back-projection (Sec. 2.2, Eq. 24-28): a streaming
 * accumulator that grids batches of projection images into the (y, N) of
 * the Fourier-domain data term, for spg_set_data_fourier.
 *
 * Image i's coefficient X at 2-D frequency index (kx, ky) (fftfreq order,
 * |k| <= n/2 - 2) lands at p = R_i (kx, ky, 0) (Eq. 24) and adds
 * P K CTF X to num(n) and P K CTF^2 to N(n) for the grid points n near p:
 * kernel 0 is the Gaussian K = exp(-|p - n|^2 / h) on the 27 points
 * round(p) + {-1,0,1}^3 (the paper uses h = 2); kernel 1 the trilinear
 * weights on the 8 cell corners. Each image is one image-pose pair with
 * posterior probability P = P(phi | X_i, V_0) (Eq. 26-28): an image with
 * several candidate poses is added once per pose.
 *
 * Images are real and CTFs centro-symmetric, so only the half ky >= 0 of
 * each spectrum (kx >= 0 on ky = 0) is read; the other half enters as its
 * conjugate. Sums are FP64 (atomics: the last bits can vary between runs).
 *
 * spg_grid_create: n even >= 4 (n^3 <= 2^31), kernel 0 or 1, h > 0; the
 *   accumulator (32 B per half-spectrum point) is owned by the object; all
 *   work is queued on `stream` (a cudaStream_t, NULL = default stream).
 * spg_grid_add: m image-pose pairs, asynchronous on the stream:
 *   rot:  m row-major 3x3 rotations (float32); columns 0, 1 map the image axes
 *   X:    m x n x n image spectra (complex64 interleaved, [ky][kx]), whose
 *         real-space origin is the image centre
 *   ctf:  m x n x n contrast transfer values (float32)
 *   pw:   m posterior weights (float32, meant to be >= 0; not checked), or
 *         NULL for weight 1 each
 *   Device arrays are read in place (they must stay valid until the work
 *   queued on the stream is done); host arrays are copied to a staging
 *   buffer first.
 * spg_grid_finish: writes the half spectra [n][n][n/2+1] (host or device):
 *   y_half (complex64) and N_half (float32), N' = V N and
 *   y = (-1)^(kx+ky+kz) num / sqrt(N) (0 where N = 0), V = n^3: the data
 *   term 1/2 |y - sqrt(N') A x|^2 of a volume whose origin is voxel 0.
 *   Keeps the sums (more images may be added); synchronises the stream.
 * spg_grid_reset: zeroes the sums. spg_grid_count: image-pose pairs added.
 * Messages of failed calls in spg_grid_last_error(g) (g = NULL: of a failed
 * spg_grid_create). */
typedef struct spg_grid spg_grid;
spg_status spg_grid_create(int n, int kernel, float h, void *stream, spg_grid **out);
spg_status spg_grid_add(spg_grid *g, int m, const float *rot, const void *X, const float *ctf, const float *pw);
spg_status spg_grid_finish(spg_grid *g, void *y_half, float *N_half);
spg_status spg_grid_reset(spg_grid *g);
long long spg_grid_count(const spg_grid *g);
const char *spg_grid_last_error(const spg_grid *g);
void spg_grid_destroy(spg_grid *g);

/* One-shot back-projection: create, add the m images, finish, destroy.
 * Message in spg_backproject_last_error(). */
spg_status spg_backproject(int n, int m, const float *rot, const void *X, const float *ctf, const float *pw,
                           int kernel, float h, void *y_half, float *N_half, void *stream);
const char *spg_backproject_last_error(void);

/* Proximal anchor of the implicit-gradient term (Sec. 2.1 Eq. 22, Eq. 31):
 * adds gamma |x - x_anchor|^2 to the data term of volume `vol`. Because
 *   1/2 w (x - b)^2 + gamma (x - a)^2 = 1/2 w' (x - b')^2 + const,
 *   w' = w + 2 gamma,  b' = (w b + 2 gamma a) / w',
 * the term folds exactly into (b, w): the call replaces the stored b and w of
 * the volume by b' and w' (computed in float32 on the device, rounded to the
 * storage dtype). x_anchor is a float32 volume (host or device), typically
 * the previous maximisation step's solution; gamma >= 0. Objective values
 * reported afterwards omit the constant. With the Fourier-domain data term
 * (after spg_set_data_fourier) the term enters the spectrum pass instead:
 * its gradient 2 gamma (y - a) = A^H(2 gamma A y - 2 gamma A a), so the step
 * uses N + 2 gamma and sqrt(N) y / sqrt(V) + 2 gamma (A a) / sqrt(V); the
 * objective then includes gamma |x - a|^2 itself. Either way L grows by
 * 2 gamma. Call after the data and before spg_reweight. Synchronises. */
spg_status spg_set_anchor(spg_ctx *ctx, int vol, float gamma, const float *x_anchor);

/* Parameter scales of Sec. 2.5 for volume `vol`, from the stored b and w:
 * out = {RMS(w b), mean(w), max(w), min(w)}. In the real-space reading of
 * the data term, w b is the kernel-regression numerator (the inverse
 * transform of D y in Eq. 31, up to normalisation), so the paper's rules
 * read lambda_l1 = c1 RMS(w b) eps, lambda_tv = c2 RMS(w b) eps_tv and
 * gamma = c3 mean(w). With the Fourier-domain data term (spg_set_data_fourier)
 * the same rules read off the spectrum: out = {RMS(A^H D y), mean(N'),
 * max(N'), min(N')} over the full spectrum (RMS by Parseval, A unitary).
 * Synchronises. */
spg_status spg_param_scales(spg_ctx *ctx, int vol, double out[4]);

/* Set / read the current iterate of volume `vol` (float32, nx*ny*nz).
 * The initial iterate is 0. spg_set_x also restarts the momentum
 * (x_{k-1} = x, i.e. d_k = 0). spg_get_x is asynchronous unless `x` is pageable host memory. */
spg_status spg_set_x(spg_ctx *ctx, int vol, const float *x);
spg_status spg_get_x(spg_ctx *ctx, int vol, float *x);

/* Start a round: re-set om1 and omtv from the current iterate of every
 * volume (Eq. 11), reduce max omtv (and nnz, sums) in double precision, set
 * tau = 1/L per volume and restart the extrapolation (t = 1, x_{-1} = x).
 * Asynchronous; per-volume statistics are read with spg_round_stats. */
spg_status spg_reweight(spg_ctx *ctx);

/* Run k iterations (one fused launch each, replayed from a captured CUDA
 * graph when k is large). Asynchronous. Errors: SPG_ENOTREADY before the
 * first spg_reweight, SPG_EINVAL if the round would exceed
 * max_iters_per_round. */
spg_status spg_iterate(spg_ctx *ctx, int k);

/* F at the current iterate of volume `vol`: out = {data, l1, tv, total}
 * (host doubles). Synchronises. */
spg_status spg_objective(spg_ctx *ctx, int vol, double out[4]);

/* Objective history of volume `vol`: entries (k, data, l1, tv, total), 5
 * doubles each, one per recorded iteration (F(x_k) is recorded by the launch
 * that consumes x_k; k counts iterations since creation). Copies at most
 * max_entries of the newest entries in increasing k to `host`, sets *n.
 * Synchronises. */
spg_status spg_history(spg_ctx *ctx, int vol, double *host, int max_entries, int *n);

/* Statistics of the last spg_reweight for volume `vol`:
 * out = {max omtv, nnz(x), sum om1, sum omtv, L, tau}. Synchronises. */
spg_status spg_round_stats(spg_ctx *ctx, int vol, double out[6]);

/* z-slab decomposition of one volume over several contexts (one per GPU in a
 * multi-GPU run; no counterpart in the paper, whose solver runs on one GPU).
 * A volume of nz planes is cut into slabs of consecutive planes; each
 * context holds its slab plus a one-plane halo: the plane just below it
 * (halo_lo = 1, absent for the first slab) and the plane just above it
 * (halo_hi = 1, absent for the last slab). A halo plane is read by the fused
 * step (its x_k and pair enter the differences of Eq. 12 and the divergence
 * of Eq. 17 at the slab's edge) but never written, and is left out of the
 * objective sums and of the re-weighting statistics, so each context's
 * history and statistics cover its own planes only. After every iteration
 * the halo planes are refreshed with the neighbours' new values
 * (spg_get_planes / spg_set_planes: the exchange a multi-GPU run makes with
 * send/receive), and after every spg_reweight all slabs take one step size
 * from the maxima over all slabs (spg_step_bound, then spg_set_step_bound).
 * With these exchanges the slabs together compute bitwise the iterates of
 * one context holding the whole volume; the objective is the sum of the
 * slabs' histories.
 *
 * spg_set_halo marks the first (lo = 1) and/or last (hi = 1) plane of volume
 * `vol` as halo planes (0 or 1 each; nz - lo - hi >= 1) and re-plans the
 * fused step; call it before spg_autotune. Needs the adopted readings, no
 * gradient restart and the real-space data term. Synchronises. */
spg_status spg_set_halo(spg_ctx *ctx, int vol, int lo, int hi);

/* out = {max w, max omtv} of volume `vol` in the current round (after
 * spg_reweight; halo planes excluded from max omtv). Synchronises. */
spg_status spg_step_bound(spg_ctx *ctx, int vol, double out[2]);

/* Sets volume `vol`'s step of the current round to tau = 1/L with
 * L = max_w + 12 lambda_tv max_omtv / mu, the expression spg_reweight uses,
 * from maxima supplied by the caller (the maxima over all slabs); call after
 * spg_reweight and before the round's first iteration. spg_round_stats then
 * reports that L and tau. Errors: SPG_EINVAL, SPG_ENOTREADY. Synchronises. */
spg_status spg_set_step_bound(spg_ctx *ctx, int vol, double max_w, double max_omtv);

/* Replace volume `vol`'s weights lambda_l1 and lambda_tv of the l1 and TV
 * terms (Sec. 2.1, Eq. 11), e.g. between solves that learn them. The step
 * tau = 1/L depends on lambda_tv, so the context then needs spg_reweight
 * before it iterates or differentiates again (SPG_ENOTREADY until then).
 * Values as in spg_create: finite and >= 0, else SPG_EINVAL with nothing
 * changed. Synchronises. */
spg_status spg_set_lambdas(spg_ctx *ctx, int vol, float lambda_l1, float lambda_tv);

/* Copy planes [z0, z0 + n) of volume `vol`'s current iterate x_k (into x) and
 * of its pair (into pair: the increment d_k with SPG_STORE_DELTA, x_{k-1}
 * with SPG_STORE_PREV) out of the context, or into it. x and pair (either may
 * be NULL) are contiguous float32 [n][ny][nx] arrays, host or device; the
 * caller keeps ownership. Needs the adopted readings. Synchronises. */
spg_status spg_get_planes(spg_ctx *ctx, int vol, int z0, int n, float *x, float *pair);
spg_status spg_set_planes(spg_ctx *ctx, int vol, int z0, int n, const float *x, const float *pair);

/* Strong-convexity certificate of the last iteration of volume `vol`:
 * out = |r|^2 with r = grad f(x_{k+1}) - grad f(y_k) + (y_k - x_{k+1})/tau, an
 * element of the subdifferential of F at x_{k+1}; F(x_{k+1}) - F* <=
 * |r|^2 / (2 min w). Needs at least one iteration in the round. Synchronises. */
spg_status spg_certificate(spg_ctx *ctx, int vol, double *out);

/* Iteration counters: total iterations since creation and within the round. */
spg_status spg_counters(spg_ctx *ctx, long long *k_total, int *k_round);

/* Checkpoint / resume. A state blob holds, for every volume, x_k, then d_k
 * (SPG_STORE_DELTA) or x_{k-1} (SPG_STORE_PREV), om1, omtv, tau, and the
 * counters; spg_set_state on a context created with the same parameters
 * continues bit-identically. The data (b and w, or the Fourier-domain
 * spectra and anchor) are not in the blob: a new context needs them set
 * first. With blob == NULL, spg_get_state only sets *size. Synchronise. */
spg_status spg_get_state(spg_ctx *ctx, void *blob, size_t *size);
spg_status spg_set_state(spg_ctx *ctx, const void *blob, size_t size);

/* Adjoint of K unrolled iterations of one round with the current weights
 * and tau held fixed, starting from the current iterate as x_0 (with
 * x_{-1} = x_0), single volume contexts only. gx: dLoss/dx_K (float32
 * volume). Writes gb = dLoss/db, gw = dLoss/dw (float32 volumes) and
 * g_scalars = {dLoss/dlambda_l1, dLoss/dlambda_tv}. Recomputes the forward
 * iterates from checkpoints of (x_k, x_{k-1}) taken every `ckpt_every`
 * iterations (0 = 10). The context's own iterate is left unchanged.
 * Working memory (2 ceil(K / ckpt_every) checkpoint volumes, ckpt_every + 2
 * segment volumes and 6 more) comes from a workspace the context owns: it
 * is allocated on first use, grown when a call needs more and kept until
 * spg_destroy, so repeated calls allocate nothing. Synchronises. */
spg_status spg_backward(spg_ctx *ctx, int K, const float *gx, float *gb, float *gw,
                        double g_scalars[2], int ckpt_every);

/* Run the forward part of spg_backward: K iterations from the current
 * iterate with fixed weights and tau, writing x_K to `xK` (float32 volume);
 * the context's iterate is left unchanged. Its three iterate buffers come
 * from the same context-owned workspace as spg_backward's. Synchronises. */
spg_status spg_unrolled(spg_ctx *ctx, int K, float *xK);

/* Self-test of the bounded device-side wait used by the fused step: launches
 * one CTA that waits on a barrier nothing ever completes, with a limit of
 * `timeout_ns`. Returns SPG_ETIMEOUT when the wait gave up as designed (the
 * context stays usable), SPG_OK if it did not time out. Synchronises. */
spg_status spg_probe_timeout(spg_ctx *ctx, long long timeout_ns);

/* Autotuner: times every compiled tile shape of the fused step, each with a
 * few z-splits of the work, for `trial_iters` iterations on this context's
 * own data, keeps the fastest plan and restores the iterate, counters and
 * history afterwards (results are unaffected). With the environment variable
 * SPG_AUTOTUNE_CACHE naming a file, choices are cached there per (volume
 * sizes, data dtype, iterate storage, GPU) and reused without timing.
 * Needs spg_set_data for every volume and a spg_reweight first. info as
 * spg_plan_info. Synchronises; allocates scratch for the saved state. */
spg_status spg_autotune(spg_ctx *ctx, int trial_iters, int info[6]);

/* Kernel launches issued by this context so far (for launch accounting). */
long long spg_launch_count(const spg_ctx *ctx);

/* Number of volumes, and the tile and work split chosen for the fused step:
 * info = {vx*32, ty, zchunk, work items, grid size, ctas per SM}. */
spg_status spg_plan_info(const spg_ctx *ctx, int info[6]);

/* Allocation-free objective (no counterpart in the paper; it exists for
 * callers that cannot allocate device memory themselves: code whose device
 * memory is owned entirely by another allocator, such as a framework's caching
 * pool or a fixed arena sized at start-up, and latency-critical paths that
 * must not trigger the device-wide synchronisation cudaMalloc can cause).
 *
 * Computes out = {data, l1, tv, total} of F at x, from caller-provided device
 * arrays x, b, w, om1, omtv (float32, contiguous [nz][ny][nx], no padding)
 * and the volume's lambda_l1, lambda_tv and mu; out is a device pointer to 4
 * doubles; stream is a cudaStream_t or NULL. Asynchronous. It covers the
 * default form only: the adopted readings (backward differences, the Neumann
 * edge, the TV weight inside the divergence), float32 b and w, and the
 * real-space data term of Eq. 28; for such a context it agrees with
 * spg_objective to a relative 1e-6 (same float32 per-voxel terms and
 * compensated sums, summed in another order).
 * It calls no cudaMalloc, cudaFree or allocating routine: its scratch (one
 * partial sum per z-plane and a counter) is a static device array of
 * SPG_NOALLOC_MAX_PLANES planes (about 128 KiB) inside this library, which
 * every GPU that loads the library holds until the process exits.
 * nz > SPG_NOALLOC_MAX_PLANES is rejected with SPG_EINVAL.
 * The first call in each CUDA context (a device's primary context, or a
 * context the caller created with the driver API and made current) looks up
 * the array's device address in that context; make that first call before
 * any stream capture.
 * Every call shares the array, which keeps the previous call's contents (the
 * counter is cleared at the start of each call): calls that overlap on the
 * GPU, from other streams or threads, race and must be serialised by the
 * caller. Errors: SPG_EINVAL, SPG_ECUDA; message in spg_noalloc_last_error()
 * ("no error" after a successful call on the calling thread). */
#define SPG_NOALLOC_MAX_PLANES 4096
spg_status spg_objective_noalloc(int nx, int ny, int nz, float lambda_l1, float lambda_tv, float mu,
                                 const float *x, const float *b, const float *w, const float *om1,
                                 const float *omtv, double *out, void *stream);
const char *spg_noalloc_last_error(void);

/* Gold-standard Fourier shell correlation (Sec. 2.3, Eq. 30) of two real
 * n x n x n maps a and b (float32, host or device, C order):
 *   fsc[k] = sum_{|k'|=k} Re F(k') G*(k') / sqrt(sum |F|^2 sum |G|^2),
 * shells k = 0 .. n/2, the shell of frequency index (h, k, l) being the
 * nearest integer to sqrt(h^2 + k^2 + l^2). counts (optional) receives the
 * number of coefficients per shell. fsc and counts are host arrays of at least
 * n/2 + 1 entries (max_shells). Uses cuFFT and allocates its own temporaries;
 * synchronises `stream`. Errors: SPG_EINVAL, SPG_ENOMEM, SPG_ECUDA with a
 * message in spg_fsc_last_error(). */
spg_status spg_fsc(int n, const float *a, const float *b, int max_shells, double *fsc, double *counts,
                   void *stream);
const char *spg_fsc_last_error(void);

/* Message for the last failing call on ctx (or a global message if ctx is
 * NULL); never NULL. */
const char *spg_last_error(const spg_ctx *ctx);

/* Free everything the context allocated. NULL is a no-op. */
void spg_destroy(spg_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SPG_H */
