// Kernel-regression back-projection (Sec. 2.2, Eq. 24-28) on the GPU.
//
// Image i's coefficient X at 2-D frequency index (kx, ky) lands at the 3-D
// position p = R_i (kx, ky, 0) (Eq. 24). Every grid point n of the kernel's
// support around p receives
//     num(n) += P K CTF X,    N(n) += P K CTF^2        (Eq. 26-28)
// with P the posterior weight of the image-pose pair (1 for known poses) and
// K = exp(-|p - n|^2 / h) on the 27 points round(p) + {-1,0,1}^3 (the
// Gaussian kernel of Sec. 2.2) or the trilinear weights on the 8 corners of
// p's cell (the interpolation kernel the paper attributes to Relion).
//
// Images are real, so X(-k) = conj X(k), and CTFs are centro-symmetric: the
// coefficient -k lands at -p with the conjugate contribution. Only the half
// ky > 0 (and kx >= 0 on ky = 0) is read, and each contribution is added at n
// or, mirrored, at -n, whichever lies in the stored half spectrum
// [n][n][n/2+1] (both on the planes kx = 0 and kx = n/2). This halves both
// the atomics and the accumulator against a full-spectrum scatter and gives
// the same sums. A CTA takes an 8 x 8 tile of one image's coefficients,
// sums their FP32 deposits in a shared-memory box and adds each touched
// point once, with FP64 atomics, into an interleaved accumulator
// (Re num, Im num, N, unused: one 32-byte sector per grid point). A finishing
// pass writes the Eq. 31 data term: N' = V N and
// y = (-1)^(kx+ky+kz) num / sqrt(N), the sign moving the
// transform's origin from the box centre (image convention) to voxel 0 (the
// solver's convention; n even).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <string>

#include "spg.h"
#include "spg_trace.h"

namespace {

thread_local std::string g_grid_err = "no error";

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 152 * 16;

__device__ __forceinline__ int wrap(int i, int n) { return ((i % n) + n) % n; }

// Add (re, im, w) at full-spectrum point (x, y, z) (any integers), and, unless
// the sample is its own mate (k = 0), the mate's (re, -im, w) at (-x, -y, -z):
// each where it falls in the stored half.
__device__ __forceinline__ void deposit(double *acc, int n, int x, int y, int z, double re, double im, double w,
                                        bool self_mate)
{
    const int nh = n / 2 + 1;
    const int xw = wrap(x, n);
    if (xw < nh) {
        double *a = acc + 4 * (((long long)wrap(z, n) * n + wrap(y, n)) * nh + xw);
        atomicAdd(a + 0, re);
        atomicAdd(a + 1, im);
        atomicAdd(a + 2, w);
    }
    if (self_mate) return;
    const int mx = wrap(-x, n);
    if (mx < nh) {
        double *a = acc + 4 * (((long long)wrap(-z, n) * n + wrap(-y, n)) * nh + mx);
        atomicAdd(a + 0, re);
        atomicAdd(a + 1, -im);
        atomicAdd(a + 2, w);
    }
}

// One image coefficient's contribution: the first grid point of its support
// on each axis and the per-axis kernel factors (the kernel factorises over
// the axes: a product of 1-D Gaussians, or of 1-D hat functions); the
// factors and the deposits are FP32 (the FP64 pipe is narrow), positions and
// the nearest-point / floor decisions FP64 so they match a double-precision
// reference.
struct Sample {
    int bx, by, bz;
    float wx[3], wy[3], wz[3];
    float vre, vim, vcc;
};

__device__ __forceinline__ void make_sample(int n, const float *__restrict__ rot, const float2 *__restrict__ X,
                                            const float *__restrict__ ctf, const float *__restrict__ pw, int kernel,
                                            float h, int img, int kx, int ky, Sample &S)
{
    const float *R = rot + (long long)img * 9;  // row-major 3x3; columns 0 and 1 span the image plane
    const double px = __dadd_rn(__dmul_rn(R[0], kx), __dmul_rn(R[1], ky));
    const double py = __dadd_rn(__dmul_rn(R[3], kx), __dmul_rn(R[4], ky));
    const double pz = __dadd_rn(__dmul_rn(R[6], kx), __dmul_rn(R[7], ky));
    const long long src = (long long)img * n * n + (long long)ky * n + wrap(kx, n);
    const float2 x = X[src];
    const float c = ctf[src];
    const float pc = pw ? pw[img] * c : c;
    S.vre = pc * x.x;
    S.vim = pc * x.y;
    S.vcc = pc * c;
    if (kernel == 0) {
        S.bx = __double2int_rn(px);
        S.by = __double2int_rn(py);
        S.bz = __double2int_rn(pz);
        const float fx = (float)(px - S.bx), fy = (float)(py - S.by), fz = (float)(pz - S.bz);
        const float ih = 1.0f / h;
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const float ex = fx - (d - 1), ey = fy - (d - 1), ez = fz - (d - 1);
            S.wx[d] = expf(-ex * ex * ih);
            S.wy[d] = expf(-ey * ey * ih);
            S.wz[d] = expf(-ez * ez * ih);
        }
        S.bx -= 1;
        S.by -= 1;
        S.bz -= 1;
    } else {
        const double flx = floor(px), fly = floor(py), flz = floor(pz);
        S.bx = (int)flx;
        S.by = (int)fly;
        S.bz = (int)flz;
        const float fx = (float)(px - flx), fy = (float)(py - fly), fz = (float)(pz - flz);
        S.wx[0] = 1.f - fx;
        S.wx[1] = fx;
        S.wy[0] = 1.f - fy;
        S.wy[1] = fy;
        S.wz[0] = 1.f - fz;
        S.wz[1] = fz;
        S.wx[2] = S.wy[2] = S.wz[2] = 0.f;
    }
}

// All deposits of one sample straight into the FP64 accumulator.
__device__ __forceinline__ void deposit_sample(double *acc, int n, int span, const Sample &S, bool self_mate)
{
    for (int dz = 0; dz < span; dz++)
        for (int dy = 0; dy < span; dy++) {
            const float kyz = S.wy[dy] * S.wz[dz];
            for (int dx = 0; dx < span; dx++) {
                const float K = S.wx[dx] * kyz;
                deposit(acc, n, S.bx + dx, S.by + dy, S.bz + dz, (double)(K * S.vre), (double)(K * S.vim),
                        (double)(K * S.vcc), self_mate);
            }
        }
}

// One CTA grids an 8 x 8 tile of one image's half spectrum (kx in tile
// columns, ky >= 0): the tile's deposits are first summed in FP32 in a
// shared-memory box covering the support of all its samples, then each
// touched box point goes to the FP64 accumulator once (with its mirror
// point, as deposit() does). Neighbouring coefficients share most of their
// support points, so this issues several times fewer global atomics than
// depositing every sample directly. A tile whose box does not fit, and the
// coefficient k = 0 (its own mate), deposit directly.
constexpr int kTile = 8;
constexpr int kBoxCap = 1536;  // box points (3 floats each: 18 KB)

__global__ void __launch_bounds__(kTile * kTile) scatter_tile_kernel(int n, int m, const float *__restrict__ rot,
                                                                     const float2 *__restrict__ X,
                                                                     const float *__restrict__ ctf,
                                                                     const float *__restrict__ pw, int kernel,
                                                                     float h, double *acc)
{
    extern __shared__ float box[];  // [kBoxCap][3]
    __shared__ int red[kTile * kTile / 32][6];
    __shared__ int geo[7];  // lo x, y, z; dims x, y, z; use box
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int span = kernel == 0 ? 3 : 2;
    const int ntx = (n + kTile - 1) / kTile, nty = (n / 2 + kTile - 1) / kTile;
    const long long ntiles = (long long)m * nty * ntx;
    const float rmax2 = (n * 0.5f - 2.0f) * (n * 0.5f - 2.0f);
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int img = (int)(t / ((long long)nty * ntx));
        const int rem = (int)(t % ((long long)nty * ntx));
        const int kx = -n / 2 + (rem % ntx) * kTile + tid % kTile;
        const int ky = (rem / ntx) * kTile + tid / kTile;
        const bool ok = kx < n / 2 && ky < n / 2 && (ky > 0 || kx >= 0) && (float)(kx * kx + ky * ky) <= rmax2;
        const bool self_mate = kx == 0 && ky == 0;
        Sample S;
        if (ok) make_sample(n, rot, X, ctf, pw, kernel, h, img, kx, ky, S);
        // bounding box of the tile's supports (the self-mate sample goes direct)
        const bool inbox = ok && !self_mate;
        int v[6] = {inbox ? S.bx : INT_MAX, inbox ? S.by : INT_MAX, inbox ? S.bz : INT_MAX,
                    inbox ? S.bx : INT_MIN, inbox ? S.by : INT_MIN, inbox ? S.bz : INT_MIN};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < 6; c++) {
                const int u = __shfl_down_sync(0xffffffffu, v[c], o);
                v[c] = c < 3 ? min(v[c], u) : max(v[c], u);
            }
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < 6; c++) red[warp][c] = v[c];
        __syncthreads();
        if (tid == 0) {
            int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
            for (int w = 0; w < kTile * kTile / 32; w++)
                for (int c = 0; c < 3; c++) {
                    lo[c] = min(lo[c], red[w][c]);
                    hi[c] = max(hi[c], red[w][3 + c]);
                }
            long long vol = 0;
            if (lo[0] != INT_MAX) {
                vol = 1;
                for (int c = 0; c < 3; c++) {
                    geo[c] = lo[c];
                    geo[3 + c] = hi[c] - lo[c] + span;
                    vol *= geo[3 + c];
                }
            }
            geo[6] = (vol > 0 && vol <= kBoxCap) ? (int)vol : 0;
        }
        __syncthreads();
        const int vol = geo[6];
        if (vol > 0) {
            for (int q = tid; q < 3 * vol; q += blockDim.x) box[q] = 0.f;
            __syncthreads();
            if (inbox) {
                const int dx0 = S.bx - geo[0], dy0 = S.by - geo[1], dz0 = S.bz - geo[2];
                for (int dz = 0; dz < span; dz++)
                    for (int dy = 0; dy < span; dy++) {
                        const float kyz = S.wy[dy] * S.wz[dz];
                        float *row = box + 3 * (((dz0 + dz) * geo[4] + (dy0 + dy)) * geo[3] + dx0);
                        for (int dx = 0; dx < span; dx++) {
                            const float K = S.wx[dx] * kyz;
                            atomicAdd(row + 3 * dx + 0, K * S.vre);
                            atomicAdd(row + 3 * dx + 1, K * S.vim);
                            atomicAdd(row + 3 * dx + 2, K * S.vcc);
                        }
                    }
            }
            __syncthreads();
            for (int q = tid; q < vol; q += blockDim.x) {
                const float re = box[3 * q], im = box[3 * q + 1], w = box[3 * q + 2];
                if (re == 0.f && im == 0.f && w == 0.f) continue;
                const int gx = geo[0] + q % geo[3], gy = geo[1] + (q / geo[3]) % geo[4], gz = geo[2] + q / (geo[3] * geo[4]);
                deposit(acc, n, gx, gy, gz, (double)re, (double)im, (double)w, false);
            }
        } else if (inbox) {
            deposit_sample(acc, n, span, S, false);
        }
        if (ok && self_mate) deposit_sample(acc, n, span, S, true);
        __syncthreads();  // the box and geo are reused by the next tile
    }
}

__global__ void finish_kernel(int n, const double *__restrict__ acc, float2 *y_half, float *N_half)
{
    const int nh = n / 2 + 1;
    const long long total = (long long)n * n * nh;
    const double V = (double)n * n * n;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int kx = (int)(q % nh);
        const int ky = (int)((q / nh) % n);
        const int kz = (int)(q / ((long long)nh * n));
        const double *a = acc + 4 * q;
        const double w = a[2];
        const double sgn = ((kx + ky + kz) & 1) ? -1.0 : 1.0;
        float2 y = make_float2(0.f, 0.f);
        if (w > 0) {
            const double s = sgn / sqrt(w);
            y = make_float2((float)(a[0] * s), (float)(a[1] * s));
        }
        y_half[q] = y;
        N_half[q] = (float)(V * w);
    }
}

int blocks_for(long long work)
{
    const long long b = (work + kThreads - 1) / kThreads;
    return (int)(b < kMaxBlocks ? (b > 0 ? b : 1) : kMaxBlocks);
}

bool on_device(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

struct spg_grid {
    int n = 0, kernel = 0;
    float h = 2.f;
    cudaStream_t stream = nullptr;
    double *acc = nullptr;  // [n][n][n/2+1][4]
    void *stage = nullptr;  // device copies of host inputs / outputs
    size_t stage_bytes = 0;
    long long images = 0;
    std::string err = "no error";
    size_t half() const { return (size_t)n * n * (n / 2 + 1); }
};

namespace {

spg_status gfail(spg_grid *g, spg_status s, const std::string &m)
{
    (g ? g->err : g_grid_err) = m;
    return s;
}

spg_status cuda_fail(spg_grid *g, cudaError_t e, const char *what)
{
    cudaGetLastError();
    return gfail(g, e == cudaErrorMemoryAllocation ? SPG_ENOMEM : SPG_ECUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

// Make sure the staging buffer holds `bytes`; waits for the stream before
// replacing a buffer that queued work may still read.
cudaError_t ensure_stage(spg_grid *g, size_t bytes)
{
    if (bytes <= g->stage_bytes) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return e;
    if (g->stage) cudaFree(g->stage);
    g->stage = nullptr;
    g->stage_bytes = 0;
    e = cudaMalloc(&g->stage, bytes);
    if (e == cudaSuccess) g->stage_bytes = bytes;
    return e;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" spg_status spg_grid_create(int n, int kernel, float h, void *stream, spg_grid **out)
{
    SPG_TRACE();
    if (!out) return gfail(nullptr, SPG_EINVAL, "spg_grid_create: null output");
    *out = nullptr;
    if (n < 4 || n % 2 || (kernel != 0 && kernel != 1) || !(h > 0.f))
        return gfail(nullptr, SPG_EINVAL, "spg_grid_create: bad arguments (even n >= 4, kernel 0 or 1, h > 0)");
    if ((long long)n * n * n > (1LL << 31)) return gfail(nullptr, SPG_EINVAL, "spg_grid_create: volume too large");
    spg_grid *g = new spg_grid;
    g->n = n;
    g->kernel = kernel;
    g->h = h;
    g->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMalloc(&g->acc, g->half() * 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(g->acc, 0, g->half() * 4 * sizeof(double), g->stream);
    if (e != cudaSuccess) {
        spg_status s = cuda_fail(nullptr, e, "spg_grid_create");
        if (g->acc) cudaFree(g->acc);
        delete g;
        return s;
    }
    *out = g;
    return SPG_OK;
}

extern "C" spg_status spg_grid_add(spg_grid *g, int m, const float *rot, const void *X, const float *ctf,
                                   const float *pw)
{
    SPG_TRACE();
    if (!g) return gfail(nullptr, SPG_EINVAL, "spg_grid_add: null accumulator");
    if (m < 1 || !rot || !X || !ctf) return gfail(g, SPG_EINVAL, "spg_grid_add: m >= 1 and non-null arrays");
    const int n = g->n;
    const size_t img = (size_t)m * n * n;
    struct In {
        const void *src;
        size_t bytes;
        const void *dev;
        bool host;
    } in[4] = {{rot, (size_t)m * 9 * sizeof(float), nullptr, false},
               {X, img * sizeof(float2), nullptr, false},
               {ctf, img * sizeof(float), nullptr, false},
               {pw, pw ? (size_t)m * sizeof(float) : 0, nullptr, false}};
    size_t need = 0;
    for (auto &a : in) {
        a.host = a.src && !on_device(a.src);
        if (a.host) need += align256(a.bytes);
    }
    cudaError_t e = ensure_stage(g, need);
    if (e != cudaSuccess) return cuda_fail(g, e, "spg_grid_add: staging buffer");
    size_t off = 0;
    for (auto &a : in) {
        if (!a.host) {
            a.dev = a.src;
            continue;
        }
        void *dst = static_cast<char *>(g->stage) + off;
        e = cudaMemcpyAsync(dst, a.src, a.bytes, cudaMemcpyHostToDevice, g->stream);
        if (e != cudaSuccess) return cuda_fail(g, e, "spg_grid_add: copy");
        a.dev = dst;
        off += align256(a.bytes);
    }
    // the tile kernel's shared box exceeds the default 48 KB (set per call: per device)
    e = cudaFuncSetAttribute(scatter_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kBoxCap * 3 * (int)sizeof(float));
    if (e != cudaSuccess) return cuda_fail(g, e, "spg_grid_add: configure");
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles = (long long)m * ((n / 2 + kTile - 1) / kTile) * ((n + kTile - 1) / kTile);
    const int grid = (int)std::min<long long>(tiles, (long long)std::max(nsm, 1) * 12 * 4);
    scatter_tile_kernel<<<grid, kTile * kTile, kBoxCap * 3 * sizeof(float), g->stream>>>(
        n, m, static_cast<const float *>(in[0].dev), static_cast<const float2 *>(in[1].dev),
        static_cast<const float *>(in[2].dev), static_cast<const float *>(in[3].dev), g->kernel, g->h, g->acc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(g, e, "spg_grid_add: launch");
    g->images += m;
    return SPG_OK;
}

extern "C" spg_status spg_grid_finish(spg_grid *g, void *y_half, float *N_half)
{
    SPG_TRACE();
    if (!g) return gfail(nullptr, SPG_EINVAL, "spg_grid_finish: null accumulator");
    if (!y_half || !N_half) return gfail(g, SPG_EINVAL, "spg_grid_finish: null output");
    const size_t half = g->half();
    const bool dy = on_device(y_half), dn = on_device(N_half);
    const size_t ybytes = dy ? 0 : align256(half * sizeof(float2));
    const size_t need = ybytes + (dn ? 0 : align256(half * sizeof(float)));
    cudaError_t e = ensure_stage(g, need);
    if (e != cudaSuccess) return cuda_fail(g, e, "spg_grid_finish: staging buffer");
    float2 *yo = dy ? static_cast<float2 *>(y_half) : static_cast<float2 *>(g->stage);
    float *no = dn ? N_half : reinterpret_cast<float *>(static_cast<char *>(g->stage) + ybytes);
    finish_kernel<<<blocks_for((long long)half), kThreads, 0, g->stream>>>(g->n, g->acc, yo, no);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(g, e, "spg_grid_finish: launch");
    if (!dy) {
        e = cudaMemcpyAsync(y_half, yo, half * sizeof(float2), cudaMemcpyDeviceToHost, g->stream);
        if (e != cudaSuccess) return cuda_fail(g, e, "spg_grid_finish: copy");
    }
    if (!dn) {
        e = cudaMemcpyAsync(N_half, no, half * sizeof(float), cudaMemcpyDeviceToHost, g->stream);
        if (e != cudaSuccess) return cuda_fail(g, e, "spg_grid_finish: copy");
    }
    e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_fail(g, e, "spg_grid_finish: synchronise");
    return SPG_OK;
}

extern "C" spg_status spg_grid_reset(spg_grid *g)
{
    SPG_TRACE();
    if (!g) return gfail(nullptr, SPG_EINVAL, "spg_grid_reset: null accumulator");
    cudaError_t e = cudaMemsetAsync(g->acc, 0, g->half() * 4 * sizeof(double), g->stream);
    if (e != cudaSuccess) return cuda_fail(g, e, "spg_grid_reset");
    g->images = 0;
    return SPG_OK;
}

extern "C" long long spg_grid_count(const spg_grid *g) { return g ? g->images : 0; }

extern "C" const char *spg_grid_last_error(const spg_grid *g) { return g ? g->err.c_str() : g_grid_err.c_str(); }

extern "C" void spg_grid_destroy(spg_grid *g)
{
    SPG_TRACE();
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    if (g->acc) cudaFree(g->acc);
    if (g->stage) cudaFree(g->stage);
    delete g;
}

extern "C" const char *spg_backproject_last_error(void) { return g_grid_err.c_str(); }

extern "C" spg_status spg_backproject(int n, int m, const float *rot, const void *X, const float *ctf,
                                      const float *pw, int kernel, float h, void *y_half, float *N_half, void *stream)
{
    SPG_TRACE();
    spg_grid *g = nullptr;
    spg_status s = spg_grid_create(n, kernel, h, stream, &g);
    if (s != SPG_OK) return s;  // message already in g_grid_err
    s = spg_grid_add(g, m, rot, X, ctf, pw);
    if (s == SPG_OK) s = spg_grid_finish(g, y_half, N_half);
    if (s != SPG_OK) g_grid_err = g->err;
    spg_grid_destroy(g);
    return s;
}
