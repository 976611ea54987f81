// Internal layout shared by the host side (spg_api.cu) and the kernels
// (spg_step.cu, spg_aux.cu) of the GB300 reweighted SPG solver.
//
// Device layout of a context with V volumes:
//  - every volume-shaped array is one flat allocation holding all V volumes
//    back to back; volume j starts at element VolDesc::off (a multiple of 64
//    elements, so every volume starts on a 256-byte boundary);
//  - inside a volume, rows of nx elements are padded to `pitch` elements
//    (a multiple of 8: 32-byte rows for float32, 16-byte for bfloat16), the
//    layout the TMA tensor maps and the 16-byte vector stores need;
//  - iterates: with increment storage (default) x lives in X[0..1] and the
//    increment d_k = x_k - x_{k-1} in X[2..3] (ping-pong, DevState::cur names
//    x_k = X[cur], d_k = X[2+cur]); with previous-iterate storage X[0..2]
//    rotate as x_{k-1}, x_k, x_{k+1} and DevState::cur names x_k.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "spg.h"

namespace spg {

struct VolDesc {
    int nx, ny, nz, pitch;
    long long off;           // element offset of the volume in every flat array
    float lambda_l1, lambda_tv, mu, eps, eps_tv;
    float tau;               // 1/L of the current round (written by the re-weighting kernel)
    int item_begin, item_end;    // work items of the fused step that belong to this volume
    int plane_begin;             // index of the volume's first z-plane among all planes
    int kmom;                    // index of the next step's extrapolation weight in the beta table
    float beta_last;             // extrapolation weight used by the last step
    int readings;                // SPG_READ_* flags (0: the adopted readings, the fused path)
    int halo_lo, halo_hi;        // first / last z-plane is a neighbour's plane (read, never written or summed)
};

// One work item of the fused step: an x-y tile [x0, x0+TX) x [y0, y0+TY) of
// volume `vol`, marching over the z-planes [z0, z1).
struct WorkItem {
    int vol, x0, y0, z0, z1, pad0, pad1, pad2;
};

// Tensor maps of one volume (device memory, 64-byte aligned).
struct TmapSet {
    CUtensorMap x[4];   // iterate buffers, box (TX+8) x (TY+2) x 1, origin (x0-4, y0-1, z)
    CUtensorMap omtv;   // TV weights,      box (TX+4) x (TY+1) x 1, origin (x0, y0, z)
    CUtensorMap b, w;   // data and weight, box TX x TY x 1,         origin (x0, y0, z-1)
    CUtensorMap om1;    // l1 weights,      box TX x TY x 1
};

// Device-resident solver state; the last CTA of each fused step advances it,
// so the same launch (or captured graph node) serves every iteration.
struct DevState {
    int cur;                 // buffer holding x_k
    int k_round;             // iterations done in the current round
    long long k_total;       // iterations since creation
    unsigned int ticket;     // arrival counter of the fused step
    unsigned int ticket_aux; // arrival counter of the auxiliary reductions
    int err;                 // first device-detected error (spg_status), 0 if none
    int hist_count;          // history entries written so far
    unsigned int err_info;   // where the error was raised
    int pad;
};

struct StepParams {
    const VolDesc *vols;
    const WorkItem *items;
    const int *sched;        // CTA g runs items sched[G+1+p] for p in [sched[g], sched[g+1]), G = gridDim.x
    const TmapSet *tmaps;
    float *xbuf[4];
    const float *beta;       // extrapolation table beta_k (float32)
    int beta_len;            // its length
    DevState *st;
    double *partials;        // [nitems][4] objective sums (data, l1, tv) and restart dot of the last step
    double *hist;            // ring [hist_cap][nvol][5]
    int nitems, nvol, hist_cap, hist_every;
    int restart;             // gradient restart of the extrapolation, per volume
    int fourier;             // data gradient = b (A^H (N A y - D y) of the Fourier-domain term), no w tile
    float *ybuf;             // Fourier-domain term: the step also writes y_{k+1} = x_{k+1} + beta_{k+1} d_{k+1} here
    long long timeout_ns;    // bound on any single barrier wait
};

// Variant of the fused step: tile = (32*vx) x ty voxels, `stages` pipeline stages.
struct StepVariant {
    int vx, ty, stages;
    bool bf16;
    bool xd;   // x_k and the increment d_k are stored (instead of x_k and x_{k-1})
};

// Host-callable launchers (spg_step.cu).
size_t step_smem_bytes(const StepVariant &v);
cudaError_t step_configure(const StepVariant &v, int *ctas_per_sm);
cudaError_t step_launch(const StepVariant &v, int grid, const StepParams &p, cudaStream_t s);
bool step_variant_supported(const StepVariant &v);

// Auxiliary kernels (spg_aux.cu). Every one runs AUX_SEG CTAs per z-plane of
// every volume (row segments) and reduces per-segment partials in a fixed order.
constexpr int AUX_SEG = 8;
struct AuxParams {
    const VolDesc *vols;
    const int *plane_vol;    // volume of each global plane
    int nplanes, nvol;
    DevState *st;
    double *plane_part;      // [nplanes * AUX_SEG][4]
    double *vol_out;         // [nvol][8]
    int readings;            // SPG_READ_* flags of the context (0: the row-vector kernels)
};

cudaError_t launch_validate(const AuxParams &a, int vol, int nz, const void *b, const void *w, bool bf16,
                            double *maxw_out, cudaStream_t s);
cudaError_t launch_convert_to_bf16(const float *src, uint16_t *dst, long long n, cudaStream_t s);
cudaError_t launch_convert_to_f32(const uint16_t *src, float *dst, long long n, cudaStream_t s);
cudaError_t launch_reverse_axes(void *v, size_t es, int nx, int ny, int nz, int pitch, cudaStream_t s);
cudaError_t launch_reweight(const AuxParams &a, const float *const *xbuf, float *om1, float *omtv,
                            const double *maxw, double *rstats, VolDesc *vols_rw, cudaStream_t s);
cudaError_t launch_objective(const AuxParams &a, const float *const *xbuf, const void *b, const void *w,
                             bool bf16, const float *om1, const float *omtv, cudaStream_t s);
// Strong-convexity certificate of the last step, xbuf = {x_{k+1}, x_k,
// x_{k-1} or null, d_k or null}: two row-vector passes (Q = P(x+) - P(y) stored in
// 3 fields of `stride` elements each, then the residual sum).
cudaError_t launch_certificate4(const AuxParams &a, const float *const *xbuf, const void *w, bool bf16,
                                const float *omtv, float *Q, long long stride, cudaStream_t s);

// Adjoint of one step (spg_aux.cu): given gnext = dL/dx_{k+1} and the step's
// inputs, accumulates into gcur (dL/dx_k), gprev (dL/dx_{k-1}), gb, gw and the
// per-plane scalar partials {dL/dlambda_l1, dL/dlambda_tv}.
struct AdjParams {
    const VolDesc *vols;     // single volume
    int nplanes;
    const float *xk, *xkm1;  // step inputs
    float beta;
    const void *b, *w;
    bool bf16;
    const float *om1, *omtv;
    const float *gnext;
    float *m;                // scratch volume: masked cotangent of z
    float *gcur, *gprev, *gb, *gw;
    double *plane_part;      // [nblocks][4]: the mask pass's scalar partials, one per CTA
    int nblocks;             // CTAs of each pass: adjoint_blocks(nx, ny, nz)
    int prev_fresh;          // gprev has no earlier contribution: write it instead of adding
};
// The adjoint of one step in two passes marching over z: the mask (p, the
// mask m, the scalar partials, gb, gw), then the update of the cotangents
// (H_mu D m and ybar). Each is one kernel of adjoint_blocks(...) CTAs.
int adjoint_blocks(int nx, int ny, int nz);
cudaError_t launch_adjoint_mask(const AdjParams &a, cudaStream_t s);
cudaError_t launch_adjoint_apply(const AdjParams &a, cudaStream_t s);
cudaError_t launch_timeout_probe(DevState *st, long long timeout_ns, cudaStream_t s);
// One iteration under alternative readings (VolDesc.readings != 0): the fused
// step's arithmetic in a plain kernel over row segments of every plane, with
// the same device-state protocol (history, extrapolation index, buffers).
struct GenericParams {
    VolDesc *vols;
    const int *plane_vol;
    int nplanes, nvol;
    DevState *st;
    double *plane_part;       // [nplanes * AUX_SEG][4]
    float *xbuf[4];           // iterate buffers (see StepParams)
    int xd;                   // increment storage
    const float *b, *w, *om1, *omtv;
    const float *beta;
    double *hist;
    int hist_cap, hist_every;
};
cudaError_t launch_generic_step(const GenericParams &g, cudaStream_t s);
// Fourier-domain data term (spg_fourier.cu), single float32 volume with increment storage.
// y = x_k + beta d_k over the whole pitched volume (cur and beta read on the device).
cudaError_t launch_form_y(const DevState *st, const VolDesc *vols, const float *beta, float *const *xbuf,
                          float *y, long long n, cudaStream_t s);
// out = {RMS(A^H D y)^2, sum N, max N, min N} over the full spectrum (partials: 1024 x 4 doubles).
cudaError_t launch_spec_scales(const float2 *C, const float *N, int nz, int ny, int nx, double *partials,
                               double *out, cudaStream_t s);
// Nst = N + two_gamma, Cst = C + two_gamma inv_v FA (the implicit-gradient term in the spectrum pass).
cudaError_t launch_spec_anchor(const float *N, const float2 *C, const float2 *FA, long long n, float two_gamma,
                               float inv_v, float *Nst, float2 *Cst, cudaStream_t s);
// *out = sum of (x - a)^2 over the volume's voxels (pitched, n elements; partials: 1024 doubles).
cudaError_t launch_sq_diff(const float *x, const float *a, int nx, int pitch, long long n, double *partials,
                           double *out, cudaStream_t s);
// F <- N F scale - C over n half-spectrum coefficients.
cudaError_t launch_spec_scale(float2 *F, const float *N, const float2 *C, long long n, float scale, cudaStream_t s);
// F = Y * sqrt(N) * scale.
cudaError_t launch_spec_prep(float2 *F, const float2 *Y, const float *N, long long n, float scale,
                             cudaStream_t s);
// max of n non-negative floats into *out (device float, initialised here).
cudaError_t launch_spec_max(const float *N, long long n, float *out, cudaStream_t s);
// out = 1/2 sum_full |Y - sqrt(N) F scale|^2 over the half spectrum (nz, ny, nxh; nx for the weights);
// partials: at least 1024 doubles.
cudaError_t launch_spec_data_value(const float2 *F, const float2 *Y, const float *N, int nz, int ny, int nx,
                                   float scale, double *partials, double *out, cudaStream_t s);

// Transform along z of a half spectrum viewed as [n][M] (spg_zfft.cu),
// power-of-two n from 8 to 4096.
constexpr int kZMaxN = 4096;
struct ZPlan {
    int n;        // transform length (nz)
    int log2n;    // log2 of n
    long long M;  // columns (ny (nx/2 + 1))
};
// Plan and twiddle table w^m = e^(-2 pi i m / nz), m < nz; false if nz is not
// a power of two in range (the caller then uses 3-D library transforms).
bool zfft_plan(int nz, long long M, ZPlan *p, std::vector<float2> *table);
// Tensor maps of the TMA-fed fused z pass: the spectrum F and the C data as
// [n][2M] float rows, N as [n][M], boxes of 16 columns by min(n, 256) rows.
struct ZMaps {
    CUtensorMap f, n, c;
};
// The TMA-fed form applies: n from 128 to 512 and M a multiple of 4 (row strides of 16-byte multiples).
bool zfft_tma_ok(const ZPlan &p);
// The fused z pass (as launch_zfft_residual) fed by TMA; a copy that never
// arrives within 2 s sets *err = SPG_ETIMEOUT.
cudaError_t launch_zfft_residual_tma(float2 *F, float scale, const ZPlan &p, const float2 *tw, const ZMaps &maps,
                                     int *err, cudaStream_t s);
// F <- A_z F (unnormalised forward transform along z of every column).
cudaError_t launch_zfft(float2 *F, const ZPlan &p, const float2 *tw, cudaStream_t s);

// Row pass of the Fourier-domain term for power-of-two nx = 128 .. 1024
// (spg_xpass.cu): real rows [nz][ny][pitch] <-> half spectrum held kx-major,
// [nz][nx/2+1][ny], unnormalised; and the transposes that put arrays of the
// standard half layout [nz][ny][nx/2+1] into that order.
bool xpass_supported(int nx, int nz);
void xpass_twiddles(int nx, std::vector<float2> *table);
cudaError_t launch_xpass_r2c(int nx, const float *Y, int pitch, int ny, int nz, float2 *F, const float2 *tw,
                             cudaStream_t s);
// The forward row pass of y_k = x_k + beta_k d_k formed from the increment-
// storage buffers (xbuf[0..1]: x, xbuf[2..3]: d; the current pair and beta_k
// read on the device, as the step that follows reads them).
cudaError_t launch_xpass_r2c_extrap(int nx, const DevState *st, const VolDesc *vols, const float *beta,
                                    float *const *xbuf, int pitch, int ny, int nz, float2 *F, const float2 *tw,
                                    cudaStream_t s);
cudaError_t launch_xpass_c2r(int nx, const float2 *F, int ny, int nz, float *Y, int pitch, const float2 *tw,
                             cudaStream_t s);
cudaError_t launch_kx_major(const float *in, float *out, int ny, int nxh, int nz, cudaStream_t s);
cudaError_t launch_kx_major(const float2 *in, float2 *out, int ny, int nxh, int nz, cudaStream_t s);
// F <- A_z^-1 ((A_z F) N scale - Cd), A_z^-1 the unnormalised inverse.
cudaError_t launch_zfft_residual(float2 *F, const float *N, const float2 *Cd, float scale, const ZPlan &p,
                                 const float2 *tw, cudaStream_t s);

// Fold gamma |x - a|^2 into (b, w) of volume `vol` (a: float32 volume in the pitched layout).
cudaError_t launch_anchor(const AuxParams &a, int vol, int nz, void *b, void *w, bool bf16, const float *anchor,
                          float gamma, double *maxw_out, cudaStream_t s);
// RMS(w b), mean w, max w, min w of volume `vol` into vol_out[vol][0..3].
cudaError_t launch_scales(const AuxParams &a, int vol, int nz, const void *b, const void *w, bool bf16,
                          cudaStream_t s);

}  // namespace spg
