// C ABI of the GB300 reweighted SPG solver (include/spg.h): contexts, device
// layout, TMA tensor maps, the work plan of the fused step, CUDA-graph replay
// of iterations, checkpoints and the adjoint driver.
#include <cudaTypedefs.h>

#include <algorithm>
#include <functional>
#include <numeric>
#include <queue>
#include <climits>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "spg.h"
#include "spg_trace.h"
#include "spg_cufft.h"
#include "spg_internal.h"

using namespace spg;

namespace {

thread_local std::string g_last_error = "no error";

constexpr long long kTimeoutNs = 2000000000LL;  // 2 s bound on any device-side wait
constexpr int kGraphLen = 10;                   // iterations per captured graph
constexpr uint64_t kStateMagic = 0x5350475354415445ull;  // "SPGSTATE"

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

long long round_up(long long a, long long b) { return (a + b - 1) / b * b; }

}  // namespace

struct spg_ctx {
    int nvol = 0;
    std::vector<spg_volume_params> vp;
    spg_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    // Forward differences alone run the adopted kernels on a layout with every
    // axis reversed: with R the reversal, D_f x = -R D_b R x, and h_mu, the
    // weights, the data term and the l1 term commute with R, so the solve of
    // (b, w) under forward differences is R applied to the backward-difference
    // solve of (R b, R w). Volumes are reversed on the way in and out.
    bool reversed = false;
    int kread = 0;  // readings the kernels implement (0: the fused path)

    std::vector<VolDesc> vols_h;
    std::vector<int> plane_vol_h;
    long long total = 0;  // elements per flat volume array
    int nplanes = 0;

    VolDesc *vols_d = nullptr;
    WorkItem *items_d = nullptr;
    int *sched_d = nullptr;   // per-CTA item ranges (grid + 1) then the item order
    TmapSet *tmaps_d = nullptr;
    int *plane_vol_d = nullptr;
    float *X[4] = {nullptr, nullptr, nullptr, nullptr};
    void *B = nullptr, *W = nullptr;
    float *OM1 = nullptr, *OMTV = nullptr;
    float *beta_d = nullptr;
    DevState *st_d = nullptr;
    double *partials_d = nullptr;
    double *hist_d = nullptr;
    double *plane_part_d = nullptr;
    double *vol_out_d = nullptr;
    double *maxw_d = nullptr;
    double *rstats_d = nullptr;

    StepVariant var{4, 8, 3, false, true};
    int zchunk = 0, grid = 0, ctas_per_sm = 0, nitems = 0;
    std::vector<WorkItem> items_h;

    long long k_total = 0;  // host mirror of the device counters
    int k_round = 0;
    int cur0 = 0;           // x_k lives in X[(cur0 + k_total) % nbuf()]
    bool reweighted = false;
    std::vector<char> data_set;
    int hist_every = 1, hist_cap = 4096, max_iters = 100000;

    // Fourier-domain data term (single volume)
    bool fourier = false;
    float *Ybuf = nullptr;   // extrapolated point y_k (pitched)
    bool y_fresh = false;    // Ybuf holds the next step's y (written by the previous fused step)
    float2 *Fh = nullptr;    // spectrum scratch
    float2 *Yh = nullptr;    // data spectrum y
    float *Nh = nullptr;     // weights N
    float2 *Ch = nullptr;    // data spectrum sqrt(N) y / sqrt(V) subtracted in the spectrum pass
    float gamma_f = 0.f;     // implicit-gradient weight with the Fourier-domain term
    float *Anc = nullptr;    // its anchor (pitched volume)
    float *Nst = nullptr;    // N + 2 gamma and C + 2 gamma A a / V: what the step uses when gamma_f > 0
    float2 *Cst = nullptr;
    float *certQ = nullptr;  // 3-vector field of the certificate passes (allocated on first use)
    float *Nmax = nullptr;
    double *fpart = nullptr; // reduction partials of the Fourier data value
    // zown: per-plane 2-D transforms (batch nz) and the own transform along z
    // (power-of-two nz); otherwise 3-D transforms and a separate spectrum pass
    cufftHandle pr2c = 0, pc2r = 0;
    bool plans = false;
    bool zown = false;
    ZPlan zplan{};
    float2 *ztw = nullptr;           // twiddle table of the transform along z
    ZMaps zmaps[2]{};                // TMA maps of the z pass: with (N, C), with (N + 2 gamma, C + ...)
    bool zmaps_ok[2] = {false, false};
    // xown: each iteration's in-plane transforms are the own row pass
    // (power-of-two nx 128 .. 1024) and the library's transform along y over
    // the contiguous lines of the kx-major spectrum [nz][nx/2+1][ny]; the z
    // pass then reads N and C (and their anchor variants) in that order
    bool xown = false;
    float2 *xtw = nullptr;           // twiddle table of the row pass
    cufftHandle pyc = 0;             // complex transform along y, nz (nx/2+1) contiguous lines
    float *Nx = nullptr;             // N, C, N + 2 gamma, C + ... held kx-major
    float2 *Cx = nullptr;
    float *Nstx = nullptr;
    float2 *Cstx = nullptr;
    ZMaps zmapsx[2]{};
    bool zmapsx_ok[2] = {false, false};
    long long nhalf = 0;

    cudaGraphExec_t gexec = nullptr;
    // workspace of spg_unrolled and spg_backward: one device buffer, grown
    // when a call needs more and kept until spg_destroy
    void *ws = nullptr;
    size_t ws_bytes = 0;
    long long launches = 0;
    std::string err = "no error";

    bool bf16() const { return opt.data_dtype == SPG_BF16; }
    bool xd() const { return opt.iterate_storage == SPG_STORE_DELTA; }
    int nbuf() const { return xd() ? 2 : 3; }  // rotation length of the iterate buffers
    int nalloc() const { return xd() ? 4 : 3; }
    size_t data_es() const { return bf16() ? 2 : 4; }
    int cur() const { return (int)(((cur0 + k_total) % nbuf() + nbuf()) % nbuf()); }
    // second buffer of the extrapolation pair for the current iterate: d_k or x_{k-1}
    int aux_of(int c) const { return xd() ? 2 + c : (c + 2) % 3; }
};

namespace {

spg_status fail(spg_ctx *c, spg_status s, const std::string &msg)
{
    if (c)
        c->err = msg;
    else
        g_last_error = msg;
    return s;
}

spg_status cuda_fail(spg_ctx *c, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();  // clear a non-sticky error
    return fail(c, e == cudaErrorMemoryAllocation ? SPG_ENOMEM : SPG_ECUDA, m);
}

#define CK(call, what)                                              \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what);     \
    } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t bytes)
{
    return cudaMalloc(reinterpret_cast<void **>(p), bytes ? bytes : 16);
}

void free_all(spg_ctx *c)
{
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->plans) {
        spg::cufft_api().destroy(c->pr2c);
        spg::cufft_api().destroy(c->pc2r);
    }
    if (c->xown) spg::cufft_api().destroy(c->pyc);
    void *fs[] = {c->Ybuf, c->Fh, c->Yh, c->Nh, c->Ch, c->Nmax, c->fpart, c->Anc, c->Nst, c->Cst, c->certQ, c->ztw, c->xtw, c->Nx,
                  c->Cx, c->Nstx, c->Cstx};
    for (void *p : fs)
        if (p) cudaFree(p);
    void *ps[] = {c->vols_d, c->items_d, c->sched_d, c->tmaps_d, c->plane_vol_d, c->X[0], c->X[1], c->X[2], c->X[3], c->B, c->W,
                  c->OM1, c->OMTV, c->beta_d, c->st_d, c->partials_d, c->hist_d, c->plane_part_d,
                  c->vol_out_d, c->maxw_d, c->rstats_d};
    for (void *p : ps)
        if (p) cudaFree(p);
    if (c->ws) cudaFree(c->ws);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

StepVariant variant_from_tile(int tile, bool bf16, bool xd)
{
    switch (tile) {
    case SPG_TILE_128x4: return {4, 4, 4, bf16, xd};
    case SPG_TILE_64x8: return {2, 8, 4, bf16, xd};
    case SPG_TILE_64x4: return {2, 4, 4, bf16, xd};
    case SPG_TILE_128x7: return {4, 7, 3, bf16, xd};
    case SPG_TILE_128x7_S4: return {4, 7, 4, bf16, xd};
    case SPG_TILE_128x15: return {4, 15, 2, bf16, xd};
    case SPG_TILE_64x7: return {2, 7, 4, bf16, xd};
    case SPG_TILE_128x8:
    default: return {4, 8, 3, bf16, xd};
    }
}

int tile_code(const StepVariant &v)
{
    if (v.vx == 4 && v.ty == 8) return SPG_TILE_128x8;
    if (v.vx == 4 && v.ty == 4) return SPG_TILE_128x4;
    if (v.vx == 2 && v.ty == 8) return SPG_TILE_64x8;
    if (v.vx == 2 && v.ty == 4) return SPG_TILE_64x4;
    if (v.vx == 4 && v.ty == 7) return v.stages == 4 ? SPG_TILE_128x7_S4 : SPG_TILE_128x7;
    if (v.vx == 4 && v.ty == 15) return SPG_TILE_128x15;
    if (v.vx == 2 && v.ty == 7) return SPG_TILE_64x7;
    return 0;
}

// Built-in tile choice: the widest tile that the volumes fill well.
StepVariant default_variant(const spg_ctx *c)
{
    long long vox = 0, waste128 = 0, waste64 = 0;
    for (const auto &v : c->vols_h) {
        const long long n = (long long)v.nx * v.ny * v.nz;
        vox += n;
        waste128 += (round_up(v.nx, 128) - v.nx) * (long long)v.ny * v.nz;
        waste64 += (round_up(v.nx, 64) - v.nx) * (long long)v.ny * v.nz;
    }
    const bool wide = waste128 <= vox / 8;
    // 4 copy stages in flight: two CTAs per SM still fit (2 x 111 KB of shared
    // memory), and at 512^3 the deeper pipeline moves 8 % more bytes per second
    if (wide) return {4, 7, 4, c->bf16(), c->xd()};
    if (waste64 <= vox / 8) return {2, 7, 4, c->bf16(), c->xd()};
    return {2, 4, 4, c->bf16(), c->xd()};
}

cudaError_t encode_map(CUtensorMap *m, CUtensorMapDataType dt, void *base, const VolDesc &v, size_t es, int bx,
                       int by)
{
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    cuuint64_t dims[3] = {(cuuint64_t)v.nx, (cuuint64_t)v.ny, (cuuint64_t)v.nz};
    cuuint64_t strides[2] = {(cuuint64_t)v.pitch * es, (cuuint64_t)v.pitch * v.ny * es};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    char *addr = static_cast<char *>(base) + (size_t)v.off * es;
    CUresult r = fn(m, dt, 3, addr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tensor maps of the TMA-fed z pass over the half spectrum viewed as [n][M]:
// F and C as rows of 2M floats, N as rows of M floats; boxes of 16 columns by
// min(n, 256) rows.
bool encode_zmaps(const ZPlan &p, float2 *F, const float *N, const float2 *C, ZMaps *m)
{
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint32_t rows = (cuuint32_t)(p.n < 256 ? p.n : 256);
    cuuint32_t estr[2] = {1, 1};
    auto one = [&](CUtensorMap *map, const void *base, long long inner, size_t row_bytes, cuuint32_t box_inner) {
        cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)p.n};
        cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
        cuuint32_t box[2] = {box_inner, rows};
        return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    std::memset(m, 0, sizeof(*m));
    return one(&m->f, F, 2 * p.M, (size_t)p.M * sizeof(float2), 32) &&
           one(&m->n, N, p.M, (size_t)p.M * sizeof(float), 16) &&
           one(&m->c, C, 2 * p.M, (size_t)p.M * sizeof(float2), 32);
}

// Tensor maps of one volume for variant v: the iterate boxes of the given
// buffers (null entries are left zero), then omtv, b, w and om1.
cudaError_t encode_set(const spg_ctx *ctx, const VolDesc &d, const StepVariant &v, float *const xq[4], TmapSet *m)
{
    const int TX = 32 * v.vx, TY = v.ty;
    const CUtensorMapDataType dt_data = v.bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    std::memset(m, 0, sizeof(*m));
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < 4 && e == cudaSuccess; q++)
        if (xq[q]) e = encode_map(&m->x[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, xq[q], d, 4, TX + 8, TY + 2);
    if (e == cudaSuccess) e = encode_map(&m->omtv, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, ctx->OMTV, d, 4, TX + 4, TY + 1);
    if (e == cudaSuccess) e = encode_map(&m->b, dt_data, ctx->B, d, ctx->data_es(), TX, TY);
    if (e == cudaSuccess) e = encode_map(&m->w, dt_data, ctx->W, d, ctx->data_es(), TX, TY);
    if (e == cudaSuccess) e = encode_map(&m->om1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, ctx->OM1, d, 4, TX, TY);
    return e;
}

// Work of an item in plane steps: its planes plus the two-plane prologue of
// the copy pipeline.
long long item_cost(int z0, int z1) { return (long long)(z1 - z0) + 2; }

// Longest-processing-time-first assignment of items to G CTAs: each item,
// longest first, goes to the least-loaded CTA (lowest index on ties). Returns
// the makespan in plane steps; with order/first given, fills the items of
// CTA g as order[first[g] .. first[g+1]), longest first.
long long lpt_schedule(const std::vector<long long> &cost, int G, std::vector<int> *order, std::vector<int> *first)
{
    const int n = (int)cost.size();
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    using Slot = std::pair<long long, int>;
    std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
    for (int g = 0; g < G; g++) heap.push({0, g});
    std::vector<int> owner(order ? n : 0);
    long long makespan = 0;
    for (int i : idx) {
        Slot sl = heap.top();
        heap.pop();
        sl.first += cost[i];
        makespan = std::max(makespan, sl.first);
        if (order) owner[i] = sl.second;
        heap.push(sl);
    }
    if (order) {
        first->assign(G + 1, 0);
        for (int i = 0; i < n; i++) (*first)[owner[i] + 1]++;
        for (int g = 0; g < G; g++) (*first)[g + 1] += (*first)[g];
        order->assign(n, 0);
        std::vector<int> pos(first->begin(), first->end() - 1);
        for (int i : idx) (*order)[pos[owner[i]]++] = i;
    }
    return makespan;
}

// Work plan: tensor maps for the variant's boxes, work items, grid size.
spg_status build_plan(spg_ctx *ctx, const StepVariant &v, int zchunk_opt)
{
    if (!step_variant_supported(v)) return fail(ctx, SPG_EINVAL, "unsupported tile variant");
    int occ = 0;
    CK(step_configure(v, &occ), "configure fused step");
    if (occ < 1) return fail(ctx, SPG_ECUDA, "fused step does not fit on an SM");
    if (ctx->opt.ctas_per_sm > 0) occ = std::min(occ, ctx->opt.ctas_per_sm);
    const int TX = 32 * v.vx, TY = v.ty;
    const long long slots = (long long)ctx->num_sms * occ;

    long long columns = 0, plane_tiles = 0;
    for (const auto &d : ctx->vols_h) {
        const long long cols = (long long)((d.nx + TX - 1) / TX) * ((d.ny + TY - 1) / TY);
        columns += cols;
        plane_tiles += cols * (d.nz - d.halo_lo - d.halo_hi);
    }
    // Planes per work item: the z-chunk whose items, scheduled longest first
    // over the resident CTAs, give the shortest makespan (one wave of equal
    // items when every column fits; finer chunks balance uneven batches).
    auto costs_for = [&](int chunk) {
        std::vector<long long> c;
        for (const auto &d : ctx->vols_h) {
            const long long cols = (long long)((d.nx + TX - 1) / TX) * ((d.ny + TY - 1) / TY);
            const int nzi = d.nz - d.halo_lo - d.halo_hi;  // planes written (halo planes are only read)
            const int nch = (nzi + chunk - 1) / chunk;
            for (int q = 0; q < nch; q++) {
                const int z0 = (int)((long long)nzi * q / nch), z1 = (int)((long long)nzi * (q + 1) / nch);
                if (z1 > z0) c.insert(c.end(), cols, item_cost(z0, z1));
            }
        }
        return c;
    };
    int maxnz = 0;
    for (const auto &d : ctx->vols_h) maxnz = std::max(maxnz, d.nz);
    int chunk;
    if (zchunk_opt > 0) {
        chunk = zchunk_opt;
    } else {
        std::vector<int> cand = {8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024};
        for (int k = 1; k <= 16; k++) cand.push_back((maxnz + k - 1) / k);
        if (columns <= slots) cand.push_back((int)((maxnz + std::max<long long>(1, slots / columns) - 1) /
                                                   std::max<long long>(1, slots / columns)));
        long long best = -1;
        chunk = maxnz;
        for (int c : cand) {
            if (c < 1 || c > maxnz) continue;
            if (plane_tiles / c > 400000) continue;  // keep the plan small
            const auto cost = costs_for(c);
            const int G = (int)std::min<long long>((long long)cost.size(), slots);
            const long long ms = lpt_schedule(cost, G, nullptr, nullptr);
            if (best < 0 || ms < best || (ms == best && c > chunk)) {
                best = ms;
                chunk = c;
            }
        }
    }
    chunk = std::max(1, chunk);

    std::vector<WorkItem> items;
    for (int j = 0; j < ctx->nvol; j++) {
        VolDesc &d = ctx->vols_h[j];
        d.item_begin = (int)items.size();
        const int nzi = d.nz - d.halo_lo - d.halo_hi;
        const int nch = (nzi + chunk - 1) / chunk;
        for (int c = 0; c < nch; c++) {
            const int z0 = d.halo_lo + (int)((long long)nzi * c / nch);
            const int z1 = d.halo_lo + (int)((long long)nzi * (c + 1) / nch);
            if (z1 <= z0) continue;
            for (int ty = 0; ty < (d.ny + TY - 1) / TY; ty++)
                for (int tx = 0; tx < (d.nx + TX - 1) / TX; tx++)
                    items.push_back(WorkItem{j, tx * TX, ty * TY, z0, z1, 0, 0, 0});
        }
        d.item_end = (int)items.size();
    }

    // tensor maps
    std::vector<TmapSet> maps(ctx->nvol);
    for (int j = 0; j < ctx->nvol; j++) {
        float *xq[4] = {nullptr, nullptr, nullptr, nullptr};
        for (int q = 0; q < ctx->nalloc(); q++) xq[q] = ctx->X[q];
        CK(encode_set(ctx, ctx->vols_h[j], v, xq, &maps[j]), "tensor maps");
    }

    // schedule: CTA g runs items order[first[g] .. first[g+1])
    const int G = (int)std::min<long long>((long long)items.size(), slots);
    std::vector<long long> cost(items.size());
    for (size_t i = 0; i < items.size(); i++) cost[i] = item_cost(items[i].z0, items[i].z1);
    std::vector<int> order, first;
    lpt_schedule(cost, G, &order, &first);
    std::vector<int> sched(first);
    sched.insert(sched.end(), order.begin(), order.end());

    if (ctx->items_d) cudaFree(ctx->items_d);
    if (ctx->partials_d) cudaFree(ctx->partials_d);
    if (ctx->sched_d) cudaFree(ctx->sched_d);
    ctx->items_d = nullptr;
    ctx->partials_d = nullptr;
    ctx->sched_d = nullptr;
    CK(dalloc(&ctx->sched_d, sched.size() * sizeof(int)), "alloc schedule");
    CK(cudaMemcpyAsync(ctx->sched_d, sched.data(), sched.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream),
       "upload schedule");
    CK(dalloc(&ctx->items_d, items.size() * sizeof(WorkItem)), "alloc items");
    CK(dalloc(&ctx->partials_d, items.size() * 4 * sizeof(double)), "alloc partials");
    CK(cudaMemcpyAsync(ctx->items_d, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice,
                       ctx->stream),
       "upload items");
    CK(cudaMemcpyAsync(ctx->tmaps_d, maps.data(), maps.size() * sizeof(TmapSet), cudaMemcpyHostToDevice, ctx->stream),
       "upload tensor maps");
    // item ranges changed: refresh descriptors (tau and the extrapolation index are device-owned)
    std::vector<VolDesc> dev(ctx->nvol);
    CK(cudaMemcpyAsync(dev.data(), ctx->vols_d, ctx->nvol * sizeof(VolDesc), cudaMemcpyDeviceToHost, ctx->stream),
       "read descriptors");
    CK(cudaStreamSynchronize(ctx->stream), "sync");
    for (int j = 0; j < ctx->nvol; j++) {
        ctx->vols_h[j].tau = dev[j].tau;
        ctx->vols_h[j].kmom = dev[j].kmom;
        ctx->vols_h[j].beta_last = dev[j].beta_last;
    }
    CK(cudaMemcpyAsync(ctx->vols_d, ctx->vols_h.data(), ctx->nvol * sizeof(VolDesc), cudaMemcpyHostToDevice,
                       ctx->stream),
       "upload descriptors");
    CK(cudaStreamSynchronize(ctx->stream), "sync");

    ctx->var = v;
    ctx->zchunk = chunk;
    ctx->items_h = items;
    ctx->nitems = (int)items.size();
    ctx->ctas_per_sm = occ;
    ctx->grid = G;
    if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    return SPG_OK;
}

StepParams step_params(const spg_ctx *c)
{
    StepParams p;
    p.vols = c->vols_d;
    p.items = c->items_d;
    p.sched = c->sched_d;
    p.tmaps = c->tmaps_d;
    for (int q = 0; q < 4; q++) p.xbuf[q] = c->X[q];
    p.beta = c->beta_d;
    p.beta_len = c->max_iters;
    p.st = c->st_d;
    p.partials = c->partials_d;
    p.hist = c->hist_d;
    p.nitems = c->nitems;
    p.nvol = c->nvol;
    p.hist_cap = c->hist_cap;
    p.hist_every = c->hist_every;
    p.restart = c->opt.restart ? 1 : 0;
    p.fourier = c->fourier ? 1 : 0;
    // the library's transforms read y_{k+1} from a buffer the step writes; the
    // own row pass forms it from x_{k+1} and d_{k+1} as it reads them
    p.ybuf = (c->fourier && !c->xown) ? c->Ybuf : nullptr;
    p.timeout_ns = kTimeoutNs;
    return p;
}

AuxParams aux_params(const spg_ctx *c)
{
    AuxParams a;
    a.vols = c->vols_d;
    a.plane_vol = c->plane_vol_d;
    a.nplanes = c->nplanes;
    a.nvol = c->nvol;
    a.st = c->st_d;
    a.plane_part = c->plane_part_d;
    a.vol_out = c->vol_out_d;
    a.readings = c->kread;
    return a;
}

// Read the device error word (synchronises); returns and clears it.
spg_status device_status(spg_ctx *ctx)
{
    DevState st;
    CK(cudaMemcpyAsync(&st, ctx->st_d, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream), "read state");
    CK(cudaStreamSynchronize(ctx->stream), "synchronise");
    if (st.err != 0) {
        int zero = 0;
        cudaMemcpyAsync(&ctx->st_d->err, &zero, sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        if (st.err == SPG_ETIMEOUT) return fail(ctx, SPG_ETIMEOUT, "a device-side wait timed out");
        if (st.err == SPG_ENONFINITE) return fail(ctx, SPG_ENONFINITE, "non-finite objective value");
        if (st.err == SPG_ECHECK) {
            unsigned zero_u = 0;
            cudaMemcpyAsync(&ctx->st_d->err_info, &zero_u, sizeof(unsigned), cudaMemcpyHostToDevice, ctx->stream);
            cudaStreamSynchronize(ctx->stream);
            return fail(ctx, SPG_ECHECK, "index check " + std::to_string(st.err_info) + " failed (checked build)");
        }
        return fail(ctx, (spg_status)st.err, "device error");
    }
    return SPG_OK;
}

bool params_ok(const spg_volume_params &p)
{
    auto pos = [](float v) { return std::isfinite(v) && v > 0.f; };
    auto nonneg = [](float v) { return std::isfinite(v) && v >= 0.f; };
    return p.nx > 0 && p.ny > 0 && p.nz > 0 && nonneg(p.lambda_l1) && nonneg(p.lambda_tv) && pos(p.mu) &&
           pos(p.eps) && pos(p.eps_tv) && (long long)p.nx * p.ny < (1LL << 31);
}

// Unpitched volumes move as one linear copy (row-by-row 2-D copies to or from
// host memory run several times slower than a linear one).
spg_status copy_volume_in(spg_ctx *ctx, void *dst_base, size_t es, const VolDesc &d, const void *src)
{
    char *dst = static_cast<char *>(dst_base) + (size_t)d.off * es;
    if (d.pitch == d.nx)
        CK(cudaMemcpyAsync(dst, src, (size_t)d.nx * d.ny * d.nz * es, cudaMemcpyDefault, ctx->stream),
           "copy volume in");
    else
        CK(cudaMemcpy2DAsync(dst, (size_t)d.pitch * es, src, (size_t)d.nx * es, (size_t)d.nx * es,
                             (size_t)d.ny * d.nz, cudaMemcpyDefault, ctx->stream),
           "copy volume in");
    if (ctx->reversed) CK(launch_reverse_axes(dst, es, d.nx, d.ny, d.nz, d.pitch, ctx->stream), "reverse axes");
    return SPG_OK;
}

// With reversed axes the context's volume is reversed in place, copied and
// reversed back (stream-ordered; the destination may be host memory).
spg_status copy_volume_out(spg_ctx *ctx, void *dst, const void *src_base, size_t es, const VolDesc &d)
{
    const char *src = static_cast<const char *>(src_base) + (size_t)d.off * es;
    char *src_rw = const_cast<char *>(src);
    if (ctx->reversed) CK(launch_reverse_axes(src_rw, es, d.nx, d.ny, d.nz, d.pitch, ctx->stream), "reverse axes");
    if (d.pitch == d.nx)
        CK(cudaMemcpyAsync(dst, src, (size_t)d.nx * d.ny * d.nz * es, cudaMemcpyDefault, ctx->stream),
           "copy volume out");
    else
        CK(cudaMemcpy2DAsync(dst, (size_t)d.nx * es, src, (size_t)d.pitch * es, (size_t)d.nx * es,
                             (size_t)d.ny * d.nz, cudaMemcpyDefault, ctx->stream),
           "copy volume out");
    if (ctx->reversed) CK(launch_reverse_axes(src_rw, es, d.nx, d.ny, d.nz, d.pitch, ctx->stream), "reverse axes");
    return SPG_OK;
}

// One iteration: the fused step, preceded for the Fourier-domain data term by
// y_k, its spectrum, the residual spectrum N A y_k - D y and the inverse
// transform into b (= the data gradient).
cudaError_t issue_iteration(spg_ctx *ctx, const StepParams &p)
{
    if (ctx->fourier) {
        const VolDesc &d = ctx->vols_h[0];
        const double V = (double)d.nx * d.ny * d.nz;
        cudaError_t e = cudaSuccess;
        const spg::CufftApi &cf = spg::cufft_api();
        const bool anc = ctx->gamma_f > 0.f;
        if (ctx->xown) {
            cufftComplex *Fc = reinterpret_cast<cufftComplex *>(ctx->Fh);
            e = launch_xpass_r2c_extrap(d.nx, ctx->st_d, ctx->vols_d, ctx->beta_d, ctx->X, d.pitch, d.ny, d.nz,
                                        ctx->Fh, ctx->xtw, ctx->stream);
            if (e != cudaSuccess) return e;
            if (cf.exec_c2c(ctx->pyc, Fc, Fc, CUFFT_FORWARD) != CUFFT_SUCCESS) return cudaErrorUnknown;
            if (ctx->zmapsx_ok[anc ? 1 : 0])
                e = launch_zfft_residual_tma(ctx->Fh, (float)(1.0 / V), ctx->zplan, ctx->ztw, ctx->zmapsx[anc ? 1 : 0],
                                             &ctx->st_d->err, ctx->stream);
            else
                e = launch_zfft_residual(ctx->Fh, anc ? ctx->Nstx : ctx->Nx, anc ? ctx->Cstx : ctx->Cx,
                                         (float)(1.0 / V), ctx->zplan, ctx->ztw, ctx->stream);
            if (e != cudaSuccess) return e;
            if (cf.exec_c2c(ctx->pyc, Fc, Fc, CUFFT_INVERSE) != CUFFT_SUCCESS) return cudaErrorUnknown;
            e = launch_xpass_c2r(d.nx, ctx->Fh, d.ny, d.nz, static_cast<float *>(ctx->B), d.pitch, ctx->xtw,
                                 ctx->stream);
            if (e != cudaSuccess) return e;
            ctx->launches += 3;
        } else {
            if (cf.exec_r2c(ctx->pr2c, ctx->Ybuf, reinterpret_cast<cufftComplex *>(ctx->Fh)) != CUFFT_SUCCESS)
                return cudaErrorUnknown;
            const float *Nw = anc ? ctx->Nst : ctx->Nh;
            const float2 *Cw = anc ? ctx->Cst : ctx->Ch;
            if (!ctx->zown)
                e = launch_spec_scale(ctx->Fh, Nw, Cw, ctx->nhalf, (float)(1.0 / V), ctx->stream);
            else if (ctx->zmaps_ok[anc ? 1 : 0])
                e = launch_zfft_residual_tma(ctx->Fh, (float)(1.0 / V), ctx->zplan, ctx->ztw, ctx->zmaps[anc ? 1 : 0],
                                             &ctx->st_d->err, ctx->stream);
            else
                e = launch_zfft_residual(ctx->Fh, Nw, Cw, (float)(1.0 / V), ctx->zplan, ctx->ztw, ctx->stream);
            if (e != cudaSuccess) return e;
            if (cf.exec_c2r(ctx->pc2r, reinterpret_cast<cufftComplex *>(ctx->Fh), static_cast<float *>(ctx->B)) !=
                CUFFT_SUCCESS)
                return cudaErrorUnknown;
            ctx->launches += 1;
        }
    }
    if (ctx->kread) {
        GenericParams g;
        g.vols = ctx->vols_d;
        g.plane_vol = ctx->plane_vol_d;
        g.nplanes = ctx->nplanes;
        g.nvol = ctx->nvol;
        g.st = ctx->st_d;
        g.plane_part = ctx->plane_part_d;
        for (int q = 0; q < 4; q++) g.xbuf[q] = ctx->X[q];
        g.xd = ctx->xd() ? 1 : 0;
        g.b = static_cast<const float *>(ctx->B);
        g.w = static_cast<const float *>(ctx->W);
        g.om1 = ctx->OM1;
        g.omtv = ctx->OMTV;
        g.beta = ctx->beta_d;
        g.hist = ctx->hist_d;
        g.hist_cap = ctx->hist_cap;
        g.hist_every = ctx->hist_every;
        return launch_generic_step(g, ctx->stream);
    }
    return step_launch(ctx->var, ctx->grid, p, ctx->stream);
}

spg_status launch_steps(spg_ctx *ctx, int k)
{
    const StepParams p = step_params(ctx);
    // kernels of this library per iteration
    const long long per_iter = ctx->fourier ? (ctx->xown ? 4 : 2) : 1;
    if (ctx->fourier && !ctx->xown && k > 0 && !ctx->y_fresh) {
        // y_k of the first step; every fused step then writes the next one
        CK(launch_form_y(ctx->st_d, ctx->vols_d, ctx->beta_d, ctx->X, ctx->Ybuf, ctx->total, ctx->stream), "form y");
        ctx->launches += 1;
        ctx->y_fresh = true;
    }
    if (k >= kGraphLen && !ctx->gexec) {
        const long long counted = ctx->launches;  // capturing launches nothing
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        for (int i = 0; i < kGraphLen; i++) {
            cudaError_t e = issue_iteration(ctx, p);
            if (e != cudaSuccess) {
                cudaStreamEndCapture(ctx->stream, &g);
                if (g) cudaGraphDestroy(g);
                ctx->launches = counted;
                return cuda_fail(ctx, e, "capture fused step");
            }
        }
        ctx->launches = counted;
        CK(cudaStreamEndCapture(ctx->stream, &g), "end capture");
        cudaError_t e = cudaGraphInstantiate(&ctx->gexec, g, 0);
        cudaGraphDestroy(g);
        CK(e, "instantiate graph");
    }
    while (k >= kGraphLen && ctx->gexec) {
        CK(cudaGraphLaunch(ctx->gexec, ctx->stream), "graph launch");
        ctx->launches += kGraphLen * per_iter;
        k -= kGraphLen;
    }
    for (int i = 0; i < k; i++) {
        const long long counted = ctx->launches;
        CK(issue_iteration(ctx, p), "fused step launch");
        ctx->launches = counted + per_iter;
    }
    return SPG_OK;
}

}  // namespace

namespace {
struct StateHeader {
    uint64_t magic;
    int32_t version, nvol, k_round, reweighted;
    int64_t k_total;
    int32_t dtype, momentum, storage, pad;
};
static_assert(sizeof(StateHeader) == 48, "state blob header layout");
}  // namespace

namespace {

struct Scratch {
    std::vector<void *> ptrs;
    ~Scratch()
    {
        for (void *p : ptrs) cudaFree(p);
    }
    template <class T>
    cudaError_t get(T **p, size_t bytes)
    {
        cudaError_t e = dalloc(p, bytes);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

// The context's workspace, at least `bytes` long. Calls on a context are
// ordered on its stream, so a call may reuse what an earlier one left there;
// growing it frees the old buffer first (cudaFree waits for the device).
cudaError_t workspace(spg_ctx *ctx, size_t bytes, char **p)
{
    if (ctx->ws_bytes < bytes) {
        if (ctx->ws) {
            cudaError_t e = cudaFree(ctx->ws);
            ctx->ws = nullptr;
            ctx->ws_bytes = 0;
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = dalloc(&ctx->ws, bytes);
        if (e != cudaSuccess) {
            ctx->ws = nullptr;
            return e;
        }
        ctx->ws_bytes = bytes;
    }
    *p = static_cast<char *>(ctx->ws);
    return cudaSuccess;
}

// Consecutive 256-byte aligned pieces of a workspace; with base null it only
// counts the bytes (the first pass of a two-pass sizing).
struct Carve {
    char *base = nullptr;
    size_t off = 0;
    template <class T>
    T *take(size_t bytes)
    {
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += (bytes + 255) / 256 * 256;
        return p;
    }
};

std::vector<float> beta_table_host(const spg_ctx *ctx, int K)
{
    std::vector<float> b(std::max(K, 1));
    double t = 1.0;
    for (int k = 0; k < K; k++) {
        const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        b[k] = ctx->opt.momentum == SPG_ISTA ? 0.f : (float)((t - 1.0) / tn);
        t = tn;
    }
    return b;
}


// Forward steps of the unrolled map through the fused kernel, on caller
// buffers: previous-iterate storage, a private device state and a private
// copy of the volume descriptor (the context's own state, history and
// iterate buffers are untouched). Steps are planned first (add), their
// tensor maps encoded and uploaded once (upload), then launched in order
// (launch); step k uses the extrapolation weight beta_k.
struct Sweep {
    struct Entry {
        float *xk, *xkm1, *xout;
        int k;
    };
    spg_ctx *ctx;
    StepVariant v;
    DevState *st = nullptr;
    VolDesc *vol = nullptr;
    TmapSet *tm = nullptr;
    std::vector<Entry> plan;
    std::vector<int> kvals;  // extrapolation indices copied to the device (kept alive)
    int launched = 0, kmom_dev = 0;

    explicit Sweep(spg_ctx *c) : ctx(c), v(c->var) { v.xd = false; }
    void add(float *xk, float *xkm1, float *xout, int k) { plan.push_back({xk, xkm1, xout, k}); }
    // device state, descriptor and tensor maps of n planned steps, from a workspace
    static void carve(Carve &cv, size_t n, DevState **st, VolDesc **vol, TmapSet **tm)
    {
        *st = cv.take<DevState>(sizeof(DevState));
        *vol = cv.take<VolDesc>(sizeof(VolDesc));
        *tm = cv.take<TmapSet>(std::max<size_t>(1, n) * sizeof(TmapSet));
    }
    // cv: where the step state lives (carved after what cv already holds)
    cudaError_t upload(Carve &cv)
    {
        int occ = 0;
        cudaError_t e = step_configure(v, &occ);
        carve(cv, plan.size(), &st, &vol, &tm);
        if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(DevState), ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(vol, ctx->vols_d, sizeof(VolDesc), cudaMemcpyDeviceToDevice, ctx->stream);
        if (e != cudaSuccess) return e;
        std::vector<TmapSet> h(plan.size());
        for (size_t j = 0; j < plan.size(); j++) {
            const int cur = (int)(j % 3);
            float *xq[4] = {nullptr, nullptr, nullptr, nullptr};
            xq[cur] = plan[j].xk;
            xq[(cur + 2) % 3] = plan[j].xkm1;
            if ((e = encode_set(ctx, ctx->vols_h[0], v, xq, &h[j])) != cudaSuccess) return e;
        }
        kvals.resize(plan.size());
        if (!h.empty())
            e = cudaMemcpyAsync(tm, h.data(), h.size() * sizeof(TmapSet), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // h goes out of scope
        kmom_dev = -1;  // the copied descriptor's index is the context's: set before the first step
        return e;
    }
    cudaError_t launch()
    {
        const Entry &E = plan[launched];
        cudaError_t e = cudaSuccess;
        if (kmom_dev != E.k) {
            kvals[launched] = E.k;
            e = cudaMemcpyAsync(reinterpret_cast<char *>(vol) + offsetof(VolDesc, kmom), &kvals[launched],
                                sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
            if (e != cudaSuccess) return e;
        }
        const int cur = launched % 3;  // the private state's buffer index advances by one per step
        StepParams p;
        p.vols = vol;
        p.items = ctx->items_d;
        p.sched = ctx->sched_d;
        p.tmaps = tm + launched;
        p.xbuf[cur] = E.xk;
        p.xbuf[(cur + 2) % 3] = E.xkm1;
        p.xbuf[(cur + 1) % 3] = E.xout;
        p.xbuf[3] = nullptr;
        p.beta = ctx->beta_d;
        p.beta_len = ctx->max_iters;
        p.st = st;
        p.partials = ctx->partials_d;
        p.hist = ctx->hist_d;
        p.nitems = ctx->nitems;
        p.nvol = 1;
        p.hist_cap = ctx->hist_cap;
        p.hist_every = 0;  // no objective, no history
        p.restart = 0;
        p.fourier = 0;
        p.ybuf = nullptr;
        p.timeout_ns = kTimeoutNs;
        e = step_launch(v, ctx->grid, p, ctx->stream);
        ctx->launches += 1;
        launched++;
        kmom_dev = E.k + 1;
        return e;
    }
    // SPG_ETIMEOUT if a step gave up waiting for its copies (synchronises).
    spg_status status()
    {
        int err = 0;
        if (cudaMemcpyAsync(&err, reinterpret_cast<char *>(st) + offsetof(DevState, err), sizeof(int),
                            cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            return SPG_ECUDA;
        return err ? (spg_status)err : SPG_OK;
    }
};
}  // namespace

extern "C" {

spg_status spg_create_batch(int nvol, const spg_volume_params *params, const spg_options *opt, void *stream,
                            spg_ctx **out)
{
    SPG_TRACE();
    if (!out || !params || nvol < 1) return fail(nullptr, SPG_EINVAL, "spg_create: bad arguments");
    *out = nullptr;
    for (int j = 0; j < nvol; j++)
        if (!params_ok(params[j])) return fail(nullptr, SPG_EINVAL, "spg_create: invalid volume parameters");
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, SPG_ECUDA, std::string("spg_create: no usable CUDA device: ") + cudaGetErrorString(e));
    }
    int major = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    if (major < 10) return fail(nullptr, SPG_ECUDA, "spg_create: needs a Blackwell (sm_10x) GPU");
    if (!encode_fn()) return fail(nullptr, SPG_ECUDA, "spg_create: cuTensorMapEncodeTiled unavailable");

    spg_ctx *ctx = new spg_ctx();
    ctx->nvol = nvol;
    ctx->vp.assign(params, params + nvol);
    if (opt) ctx->opt = *opt;
    if (ctx->opt.data_dtype != SPG_F32 && ctx->opt.data_dtype != SPG_BF16) {
        delete ctx;
        return fail(nullptr, SPG_EINVAL, "spg_create: bad data dtype");
    }
    if (ctx->opt.readings < 0 || ctx->opt.readings > (SPG_READ_FORWARD | SPG_READ_PERIODIC | SPG_READ_POST_DIV)) {
        delete ctx;
        return fail(nullptr, SPG_EINVAL, "spg_create: bad readings flags");
    }
    ctx->reversed = ctx->opt.readings == SPG_READ_FORWARD;
    ctx->kread = ctx->reversed ? 0 : ctx->opt.readings;
    if (ctx->kread && (ctx->opt.data_dtype != SPG_F32 || ctx->opt.restart)) {
        delete ctx;
        return fail(nullptr, SPG_EINVAL, "spg_create: alternative readings need float32 data and no restart");
    }
    ctx->hist_every = ctx->opt.hist_every > 0 ? ctx->opt.hist_every : 1;
    ctx->hist_cap = ctx->opt.hist_capacity > 0 ? ctx->opt.hist_capacity : 4096;
    ctx->max_iters = ctx->opt.max_iters_per_round > 0 ? ctx->opt.max_iters_per_round : 100000;
    ctx->num_sms = nsm;
    ctx->data_set.assign(nvol, 0);
    if (stream) {
        ctx->stream = static_cast<cudaStream_t>(stream);
    } else {
        e = cudaStreamCreate(&ctx->stream);
        if (e != cudaSuccess) {
            delete ctx;
            return fail(nullptr, SPG_ECUDA, "spg_create: stream creation failed");
        }
        ctx->own_stream = true;
    }

    // layout
    long long off = 0;
    int plane = 0;
    for (int j = 0; j < nvol; j++) {
        const auto &p = params[j];
        VolDesc d{};
        d.nx = p.nx;
        d.ny = p.ny;
        d.nz = p.nz;
        d.pitch = (int)round_up(p.nx, 8);
        d.off = off;
        d.lambda_l1 = p.lambda_l1;
        d.lambda_tv = p.lambda_tv;
        d.mu = p.mu;
        d.eps = p.eps;
        d.eps_tv = p.eps_tv;
        d.tau = 0.f;
        d.plane_begin = plane;
        d.readings = ctx->kread;
        ctx->vols_h.push_back(d);
        for (int z = 0; z < p.nz; z++) ctx->plane_vol_h.push_back(j);
        off += round_up((long long)d.pitch * d.ny * d.nz, 64);
        plane += p.nz;
    }
    ctx->total = off;
    ctx->nplanes = plane;

    auto bail = [&](cudaError_t err, const char *what) {
        std::string m = std::string("spg_create: ") + what + ": " + cudaGetErrorString(err);
        spg_status s = err == cudaErrorMemoryAllocation ? SPG_ENOMEM : SPG_ECUDA;
        cudaGetLastError();
        free_all(ctx);
        delete ctx;
        return fail(nullptr, s, m);
    };
    const size_t vb = (size_t)ctx->total * 4, db = (size_t)ctx->total * ctx->data_es();
    if ((e = dalloc(&ctx->vols_d, nvol * sizeof(VolDesc))) != cudaSuccess) return bail(e, "alloc");
    if ((e = dalloc(&ctx->tmaps_d, nvol * sizeof(TmapSet))) != cudaSuccess) return bail(e, "alloc");
    if ((e = dalloc(&ctx->plane_vol_d, plane * sizeof(int))) != cudaSuccess) return bail(e, "alloc");
    if (ctx->opt.iterate_storage != SPG_STORE_DELTA && ctx->opt.iterate_storage != SPG_STORE_PREV) {
        free_all(ctx);
        delete ctx;
        return fail(nullptr, SPG_EINVAL, "spg_create: bad iterate storage");
    }
    for (int q = 0; q < ctx->nalloc(); q++)
        if ((e = dalloc(&ctx->X[q], vb)) != cudaSuccess) return bail(e, "alloc iterates");
    if ((e = dalloc(&ctx->B, db)) != cudaSuccess) return bail(e, "alloc b");
    if ((e = dalloc(&ctx->W, db)) != cudaSuccess) return bail(e, "alloc w");
    if ((e = dalloc(&ctx->OM1, vb)) != cudaSuccess) return bail(e, "alloc om1");
    if ((e = dalloc(&ctx->OMTV, vb)) != cudaSuccess) return bail(e, "alloc omtv");
    if ((e = dalloc(&ctx->beta_d, ctx->max_iters * sizeof(float))) != cudaSuccess) return bail(e, "alloc beta");
    if ((e = dalloc(&ctx->st_d, sizeof(DevState))) != cudaSuccess) return bail(e, "alloc state");
    if ((e = dalloc(&ctx->hist_d, (size_t)ctx->hist_cap * nvol * 5 * sizeof(double))) != cudaSuccess)
        return bail(e, "alloc history");
    if ((e = dalloc(&ctx->plane_part_d, (size_t)plane * AUX_SEG * 4 * sizeof(double))) != cudaSuccess)
        return bail(e, "alloc partials");
    if ((e = dalloc(&ctx->vol_out_d, (size_t)nvol * 8 * sizeof(double))) != cudaSuccess) return bail(e, "alloc");
    if ((e = dalloc(&ctx->maxw_d, (size_t)nvol * sizeof(double))) != cudaSuccess) return bail(e, "alloc");
    if ((e = dalloc(&ctx->rstats_d, (size_t)nvol * 6 * sizeof(double))) != cudaSuccess) return bail(e, "alloc");

    {
        const std::pair<void *, size_t> zero[] = {
            {ctx->X[0], vb}, {ctx->X[1], vb}, {ctx->X[2], vb}, {ctx->X[3], vb}, {ctx->B, db}, {ctx->W, db},
            {ctx->OM1, vb}, {ctx->OMTV, vb}, {ctx->st_d, sizeof(DevState)},
            {ctx->hist_d, (size_t)ctx->hist_cap * nvol * 5 * sizeof(double)},
            {ctx->rstats_d, (size_t)nvol * 6 * sizeof(double)}};
        for (const auto &z : zero)
            if (z.first && (e = cudaMemsetAsync(z.first, 0, z.second, ctx->stream)) != cudaSuccess)
                return bail(e, "clear buffers");
    }
    // extrapolation table, FP64 recurrence, stored as float32
    const std::vector<float> beta = beta_table_host(ctx, ctx->max_iters);
    if ((e = cudaMemcpyAsync(ctx->beta_d, beta.data(), beta.size() * sizeof(float), cudaMemcpyHostToDevice,
                             ctx->stream)) != cudaSuccess)
        return bail(e, "upload beta");
    if ((e = cudaMemcpyAsync(ctx->plane_vol_d, ctx->plane_vol_h.data(), plane * sizeof(int), cudaMemcpyHostToDevice,
                             ctx->stream)) != cudaSuccess)
        return bail(e, "upload plane map");
    if ((e = cudaMemcpyAsync(ctx->vols_d, ctx->vols_h.data(), nvol * sizeof(VolDesc), cudaMemcpyHostToDevice,
                             ctx->stream)) != cudaSuccess)
        return bail(e, "upload descriptors");
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return bail(e, "synchronise");

    const StepVariant v =
        ctx->opt.tile ? variant_from_tile(ctx->opt.tile, ctx->bf16(), ctx->xd()) : default_variant(ctx);
    spg_status s = build_plan(ctx, v, ctx->opt.zchunk);
    if (s != SPG_OK) {
        std::string m = "spg_create: " + ctx->err;
        free_all(ctx);
        delete ctx;
        return fail(nullptr, s, m);
    }
    *out = ctx;
    return SPG_OK;
}

spg_status spg_create(const spg_volume_params *params, const spg_options *opt, void *stream, spg_ctx **out)
{
    SPG_TRACE();
    return spg_create_batch(1, params, opt, stream, out);
}

spg_status spg_set_data(spg_ctx *ctx, int vol, const void *b, const void *w, spg_dtype src)
{
    SPG_TRACE();
    if (!ctx) return fail(nullptr, SPG_EINVAL, "null context");
    if (vol < 0 || vol >= ctx->nvol || !b || !w) return fail(ctx, SPG_EINVAL, "spg_set_data: bad arguments");
    if (src != SPG_F32 && src != SPG_BF16) return fail(ctx, SPG_EINVAL, "spg_set_data: bad dtype");
    if (ctx->fourier) {
        ctx->fourier = false;  // back to the real-space data term
        if (ctx->gexec) {
            cudaGraphExecDestroy(ctx->gexec);
            ctx->gexec = nullptr;
        }
    }
    const VolDesc &d = ctx->vols_h[vol];
    const long long n = (long long)d.pitch * d.ny * d.nz;
    const bool store_bf16 = ctx->bf16();
    spg_status s;
    if ((src == SPG_BF16) == store_bf16) {
        if ((s = copy_volume_in(ctx, ctx->B, ctx->data_es(), d, b)) != SPG_OK) return s;
        if ((s = copy_volume_in(ctx, ctx->W, ctx->data_es(), d, w)) != SPG_OK) return s;
    } else {
        // stage in the weight buffers (they are re-set by the next spg_reweight)
        const size_t ses = src == SPG_BF16 ? 2 : 4;
        if ((s = copy_volume_in(ctx, ctx->OM1, ses, d, b)) != SPG_OK) return s;
        if ((s = copy_volume_in(ctx, ctx->OMTV, ses, d, w)) != SPG_OK) return s;
        if (store_bf16) {
            CK(launch_convert_to_bf16(ctx->OM1 + d.off, static_cast<uint16_t *>(ctx->B) + d.off, n, ctx->stream),
               "convert b");
            CK(launch_convert_to_bf16(ctx->OMTV + d.off, static_cast<uint16_t *>(ctx->W) + d.off, n, ctx->stream),
               "convert w");
        } else {
            CK(launch_convert_to_f32(reinterpret_cast<const uint16_t *>(ctx->OM1) + d.off,
                                     static_cast<float *>(ctx->B) + d.off, n, ctx->stream),
               "convert b");
            CK(launch_convert_to_f32(reinterpret_cast<const uint16_t *>(ctx->OMTV) + d.off,
                                     static_cast<float *>(ctx->W) + d.off, n, ctx->stream),
               "convert w");
        }
        ctx->reweighted = false;
    }
    ctx->launches += 1;
    CK(launch_validate(aux_params(ctx), vol, d.nz, ctx->B, ctx->W, store_bf16, ctx->maxw_d, ctx->stream),
       "validate");
    double o[8];
    CK(cudaMemcpyAsync(o, ctx->vol_out_d + (size_t)vol * 8, sizeof(o), cudaMemcpyDeviceToHost, ctx->stream),
       "read validation");
    CK(cudaStreamSynchronize(ctx->stream), "synchronise");
    if (o[3] > 0) return fail(ctx, SPG_ENONFINITE, "spg_set_data: b has non-finite values");
    if (o[2] > 0) return fail(ctx, SPG_EINVAL, "spg_set_data: w must be finite and > 0");
    ctx->data_set[vol] = 1;
    return SPG_OK;
}

spg_status spg_set_data_fourier(spg_ctx *ctx, int vol, const void *y_half, const float *N_half)
{
    SPG_TRACE();
    if (!ctx) return fail(nullptr, SPG_EINVAL, "null context");
    if (vol != 0 || ctx->nvol != 1 || !y_half || !N_half)
        return fail(ctx, SPG_EINVAL, "spg_set_data_fourier: single-volume contexts, vol = 0, non-null arrays");
    if (ctx->opt.readings) return fail(ctx, SPG_EINVAL, "spg_set_data_fourier: not available with alternative readings");
    if (ctx->bf16() || !ctx->xd())
        return fail(ctx, SPG_EINVAL, "spg_set_data_fourier: needs SPG_F32 storage and SPG_STORE_DELTA");
    const spg::CufftApi &cf = spg::cufft_api();
    if (!cf.ok) return fail(ctx, SPG_ECUDA, "spg_set_data_fourier: cuFFT library could not be loaded");
    const VolDesc &d = ctx->vols_h[0];
    const int nxh = d.nx / 2 + 1;
    ctx->nhalf = (long long)d.nz * d.ny * nxh;
    if (!ctx->Ybuf) {
        CK(dalloc(&ctx->Ybuf, (size_t)ctx->total * sizeof(float)), "alloc");
        CK(dalloc(&ctx->Fh, (size_t)ctx->nhalf * sizeof(float2)), "alloc");
        CK(dalloc(&ctx->Yh, (size_t)ctx->nhalf * sizeof(float2)), "alloc");
        CK(dalloc(&ctx->Nh, (size_t)ctx->nhalf * sizeof(float)), "alloc");
        CK(dalloc(&ctx->Ch, (size_t)ctx->nhalf * sizeof(float2)), "alloc");
        CK(dalloc(&ctx->Nmax, sizeof(float)), "alloc");
        CK(dalloc(&ctx->fpart, 1025 * sizeof(double)), "alloc");
        CK(cudaMemsetAsync(ctx->Ybuf, 0, (size_t)ctx->total * sizeof(float), ctx->stream), "memset");
    }
    if (!ctx->plans) {
        // power-of-two nz: 3-D transforms = a batch of per-plane 2-D transforms
        // (x, y) and the own transform along z, which also forms the residual
        // spectrum; other lengths: 3-D library transforms around a spectrum pass
        std::vector<float2> tw;
        ctx->zown = zfft_plan(d.nz, (long long)d.ny * nxh, &ctx->zplan, &tw);
        if (ctx->zown) {
            CK(dalloc(&ctx->ztw, tw.size() * sizeof(float2)), "alloc");
            CK(cudaMemcpyAsync(ctx->ztw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice,
                               ctx->stream),
               "twiddles");
            CK(cudaStreamSynchronize(ctx->stream), "synchronise");
        }
        const int rank = ctx->zown ? 2 : 3;
        int n[3] = {d.nz, d.ny, d.nx};
        int real_embed[3] = {d.nz, d.ny, d.pitch};
        int cplx_embed[3] = {d.nz, d.ny, nxh};
        const long long rdist64 = (long long)(ctx->zown ? 1 : d.nz) * d.ny * d.pitch;
        const long long cdist64 = (long long)(ctx->zown ? 1 : d.nz) * d.ny * nxh;
        if (rdist64 > INT_MAX || cdist64 > INT_MAX)
            return fail(ctx, SPG_EINVAL,
                        "spg_set_data_fourier: a transform of more than 2^31 elements needs a power-of-two nz");
        const int rdist = (int)rdist64, cdist = (int)cdist64;
        const int batch = ctx->zown ? d.nz : 1;
        const int o = 3 - rank;  // the 2-D plans take the last two extents
        if (cf.plan_many(&ctx->pr2c, rank, n + o, real_embed + o, 1, rdist, cplx_embed + o, 1, cdist, CUFFT_R2C,
                         batch) != CUFFT_SUCCESS)
            return fail(ctx, SPG_ECUDA, "spg_set_data_fourier: cufft plan");
        if (cf.plan_many(&ctx->pc2r, rank, n + o, cplx_embed + o, 1, cdist, real_embed + o, 1, rdist, CUFFT_C2R,
                         batch) != CUFFT_SUCCESS) {
            cf.destroy(ctx->pr2c);
            return fail(ctx, SPG_ECUDA, "spg_set_data_fourier: cufft plan");
        }
        cf.set_stream(ctx->pr2c, ctx->stream);
        cf.set_stream(ctx->pc2r, ctx->stream);
        ctx->plans = true;
        ctx->zmaps_ok[0] = ctx->zown && zfft_tma_ok(ctx->zplan) &&
                           encode_zmaps(ctx->zplan, ctx->Fh, ctx->Nh, ctx->Ch, &ctx->zmaps[0]);
        // power-of-two nx 128 .. 1024: the own row pass and the library's
        // transform along y over contiguous lines (SPG_ROW_PASS=0 in the
        // environment keeps the library's per-plane 2-D transforms)
        const char *rp = std::getenv("SPG_ROW_PASS");
        const long long ylines = (long long)d.nz * nxh;
        if (ctx->zown && xpass_supported(d.nx, d.nz) && !(rp && std::strcmp(rp, "0") == 0) &&
            ylines * d.ny <= INT_MAX) {
            int ny1[1] = {d.ny};
            if (cf.plan_many(&ctx->pyc, 1, ny1, ny1, 1, d.ny, ny1, 1, d.ny, CUFFT_C2C, (int)ylines) == CUFFT_SUCCESS) {
                ctx->xown = true;  // the plan exists from here on (destroyed with the context)
                cf.set_stream(ctx->pyc, ctx->stream);
                std::vector<float2> xt;
                xpass_twiddles(d.nx, &xt);
                CK(dalloc(&ctx->xtw, xt.size() * sizeof(float2)), "alloc");
                CK(cudaMemcpyAsync(ctx->xtw, xt.data(), xt.size() * sizeof(float2), cudaMemcpyHostToDevice,
                                   ctx->stream),
                   "twiddles");
                CK(dalloc(&ctx->Nx, (size_t)ctx->nhalf * sizeof(float)), "alloc");
                CK(dalloc(&ctx->Cx, (size_t)ctx->nhalf * sizeof(float2)), "alloc");
                CK(cudaStreamSynchronize(ctx->stream), "synchronise");
                ctx->zmapsx_ok[0] = zfft_tma_ok(ctx->zplan) &&
                                    encode_zmaps(ctx->zplan, ctx->Fh, ctx->Nx, ctx->Cx, &ctx->zmapsx[0]);
            }
        }
    }
    CK(cudaMemcpyAsync(ctx->Yh, y_half, (size_t)ctx->nhalf * sizeof(float2), cudaMemcpyDefault, ctx->stream),
       "copy y");
    CK(cudaMemcpyAsync(ctx->Nh, N_half, (size_t)ctx->nhalf * sizeof(float), cudaMemcpyDefault, ctx->stream),
       "copy N");
    // data spectrum sqrt(N) y / sqrt(V), subtracted from N F / V each iteration; b starts at 0
    const double V = (double)d.nx * d.ny * d.nz;
    CK(launch_spec_prep(ctx->Ch, ctx->Yh, ctx->Nh, ctx->nhalf, (float)(1.0 / std::sqrt(V)), ctx->stream), "prep");
    if (ctx->xown) {
        CK(launch_kx_major(ctx->Nh, ctx->Nx, d.ny, nxh, d.nz, ctx->stream), "N kx-major");
        CK(launch_kx_major(ctx->Ch, ctx->Cx, d.ny, nxh, d.nz, ctx->stream), "C kx-major");
        ctx->launches += 2;
    }
    CK(cudaMemsetAsync(ctx->B, 0, (size_t)ctx->total * sizeof(float), ctx->stream), "memset");
    CK(launch_spec_max(ctx->Nh, ctx->nhalf, ctx->Nmax, ctx->stream), "max N");
    ctx->launches += 2;  // prep and max
    float nmax = 0.f;
    CK(cudaMemcpyAsync(&nmax, ctx->Nmax, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream), "read max N");
    CK(cudaStreamSynchronize(ctx->stream), "synchronise");
    if (!(nmax >= 0.f) || !std::isfinite(nmax)) return fail(ctx, SPG_EINVAL, "spg_set_data_fourier: bad N");
    const double m = nmax;
    CK(cudaMemcpyAsync(ctx->maxw_d, &m, sizeof(double), cudaMemcpyHostToDevice, ctx->stream), "write max N");
    CK(cudaStreamSynchronize(ctx->stream), "synchronise");
    if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);  // the iteration body changes
        ctx->gexec = nullptr;
    }
    ctx->fourier = true;
    ctx->gamma_f = 0.f;  // new data: no anchor term until spg_set_anchor
    ctx->y_fresh = false;
    ctx->data_set[0] = 1;
    ctx->reweighted = false;
    return SPG_OK;
}

spg_status spg_set_anchor(spg_ctx *ctx, int vol, float gamma, const float *x_anchor)
{
    SPG_TRACE();
    if (!ctx) return fail(nullptr, SPG_EINVAL, "null context");
    if (vol < 0 || vol >= ctx->nvol || !x_anchor || !(gamma >= 0.f) || !std::isfinite(gamma))
        return fail(ctx, SPG_EINVAL, "spg_set_anchor: bad arguments");
    if (!ctx->data_set[vol]) return fail(ctx, SPG_ENOTREADY, "spg_set_anchor: call spg_set_data first");
    const VolDesc &d = ctx->vols_h[vol];
    if (ctx->fourier) {
        // gamma |x - a|^2 enters the spectrum pass (N + 2 gamma, C + 2 gamma A a / V) and L (+ 2 gamma)
        if (!ctx->Anc) {
            CK(dalloc(&ctx->Anc, (size_t)ctx->total * sizeof(float)), "alloc");
            CK(dalloc(&ctx->Nst, (size_t)ctx->nhalf * sizeof(float)), "alloc");
            CK(dalloc(&ctx->Cst, (size_t)ctx->nhalf * sizeof(float2)), "alloc");
            CK(cudaMemsetAsync(ctx->Anc, 0, (size_t)ctx->total * sizeof(float), ctx->stream), "memset");
            ctx->zmaps_ok[1] = ctx->zmaps_ok[0] && encode_zmaps(ctx->zplan, ctx->Fh, ctx->Nst, ctx->Cst, &ctx->zmaps[1]);
            if (ctx->xown) {
                CK(dalloc(&ctx->Nstx, (size_t)ctx->nhalf * sizeof(float)), "alloc");
                CK(dalloc(&ctx->Cstx, (size_t)ctx->nhalf * sizeof(float2)), "alloc");
                ctx->zmapsx_ok[1] =
                    ctx->zmapsx_ok[0] && encode_zmaps(ctx->zplan, ctx->Fh, ctx->Nstx, ctx->Cstx, &ctx->zmapsx[1]);
            }
        }
        spg_status s = copy_volume_in(ctx, ctx->Anc, 4, d, x_anchor);
        if (s != SPG_OK) return s;
        const double V = (double)d.nx * d.ny * d.nz;
        if (spg::cufft_api().exec_r2c(ctx->pr2c, ctx->Anc, reinterpret_cast<cufftComplex *>(ctx->Fh)) != CUFFT_SUCCESS)
            return fail(ctx, SPG_ECUDA, "spg_set_anchor: transform");
        if (ctx->zown) {
            CK(launch_zfft(ctx->Fh, ctx->zplan, ctx->ztw, ctx->stream), "transform along z");
            ctx->launches += 1;
        }
        CK(launch_spec_anchor(ctx->Nh, ctx->Ch, ctx->Fh, ctx->nhalf, 2.f * gamma, (float)(1.0 / V), ctx->Nst, ctx->Cst,
                              ctx->stream),
           "anchor spectrum");
        ctx->launches += 1;
        if (ctx->xown) {
            const int nxh = d.nx / 2 + 1;
            CK(launch_kx_major(ctx->Nst, ctx->Nstx, d.ny, nxh, d.nz, ctx->stream), "N kx-major");
            CK(launch_kx_major(ctx->Cst, ctx->Cstx, d.ny, nxh, d.nz, ctx->stream), "C kx-major");
            ctx->launches += 2;
        }
        float nmax = 0.f;
        CK(launch_spec_max(ctx->Nh, ctx->nhalf, ctx->Nmax, ctx->stream), "max N");
        ctx->launches += 1;
        CK(cudaMemcpyAsync(&nmax, ctx->Nmax, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream), "read max N");
        CK(cudaStreamSynchronize(ctx->stream), "synchronise");
        const double m = (double)nmax + 2.0 * gamma;
        CK(cudaMemcpyAsync(ctx->maxw_d, &m, sizeof(double), cudaMemcpyHostToDevice, ctx->stream), "write max N");
        CK(cudaStreamSynchronize(ctx->stream), "synchronise");
        ctx->gamma_f = gamma;
        if (ctx->gexec) {
            cudaGraphExecDestroy(ctx->gexec);  // the spectrum pass reads other buffers now
            ctx->gexec = nullptr;
        }
        ctx->y_fresh = false;
        ctx->reweighted = false;
        return SPG_OK;
    }
    // stage the anchor in the l1-weight buffer (re-set by the next spg_reweight)
    spg_status s = copy_volume_in(ctx, ctx->OM1, 4, d, x_anchor);
    if (s != SPG_OK) return s;
    CK(launch_anchor(aux_params(ctx), vol, d.nz, ctx->B, ctx->W, ctx->bf16(), ctx->OM1, gamma, ctx->maxw_d,
                     ctx->stream),
       "anchor");
    ctx->launches += 1;
    ctx->reweighted = false;
    return device_status(ctx);
}

spg_status spg_param_scales(spg_ctx *ctx, int vol, double out[4])
{
    SPG_TRACE();
    if (!ctx) return fail(nullptr, SPG_EINVAL, "null context");
    if (vol < 0 || vol >= ctx->nvol || !out) return fail(ctx, SPG_EINVAL, "spg_param_scales: bad arguments");
    if (!ctx->data_set[vol]) return fail(ctx, SPG_ENOTREADY, "spg_param_scales: call spg_set_data first");
    const VolDesc &d = ctx->vols_h[vol];
    if (ctx->fourier) {
        // from the spectrum: RMS(A^H D y) (Parseval), mean, max and min of N
        Scratch sc;
        double *part = nullptr;
        CK(sc.get(&part, (1024 * 4 + 4) * sizeof(double)), "alloc");
        CK(launch_spec_scales(ctx->Ch, ctx->Nh, d.nz, d.ny, d.nx, part, part + 4096, ctx->stream), "scales");
        ctx->launches += 2;
        double o[4];
        CK(cudaMemcpyAsync(o, part + 4096, sizeof(o), cudaMemcpyDeviceToHost, ctx->stream), "read scales");
        CK(cudaStreamSynchronize(ctx->stream), "synchronise");
        const double V = (double)d.nx * d.ny * d.nz;
        out[0] = std::sqrt(o[0]);
        out[1] = o[1] / V;
        out[2] = o[2];
        out[3] = o[3];
        return SPG_OK;
    }
    CK(launch_scales(aux_params(ctx), vol, d.nz, ctx->B, ctx->W, ctx->bf16(), ctx->stream), "scales");
    ctx->launches += 1;
    double o[8];
    CK(cudaMemcpyAsync(o, ctx->vol_out_d + (size_t)vol * 8, sizeof(o), cudaMemcpyDeviceToHost, ctx->stream),
       "read scales");
    spg_status s = device_status(ctx);
    if (s != SPG_OK) return s;
    for (int q = 0; q < 4; q++) out[q] = o[q];
    return SPG_OK;
}

spg_status spg_set_x(spg_ctx *ctx, int vol, const float *x)
{
    SPG_TRACE();
    if (!ctx) return fail(nullptr, SPG_EINVAL, "null context");
    if (vol < 0 || vol >= ctx->nvol || !x) return fail(ctx, SPG_EINVAL, "spg_set_x: bad arguments");
    ctx->y_fresh = false;
    const VolDesc &d = ctx->vols_h[vol];
    const int c = ctx->cur();
    spg_status s;
    if ((s = copy_volume_in(ctx, ctx->X[c], 4, d, x)) != SPG_OK) return s;
    {
        // the extrapolation restarts from this iterate
        const int zero = 0;
        CK(cudaMemcpyAsync(&ctx->vols_d[vol].kmom, &zero, sizeof(int), cudaMemcpyHostToDevice, ctx->stream),
           "reset extrapolation");
        CK(cudaStreamSynchronize(ctx->stream), "synchronise");
    }
    if (ctx->xd()) {
        CK(cudaMemsetAsync(ctx->X[ctx->aux_of(c)] + d.off, 0, (size_t)d.pitch * d.ny * d.nz * 4, ctx->stream),
           "reset increment");
    } else if ((s = copy_volume_in(ctx, ctx->X[ctx->aux_of(c)], 4, d, x)) != SPG_OK) {
        return s;
    }
    return SPG_OK;
}

spg_status spg_get_x(spg_ctx *ctx, int vol, float *x)
{
    SPG_TRACE();
    if (!ctx) return fail(nullptr, SPG_EINVAL, "null context");
    if (vol < 0 || vol >= ctx->nvol || !x) return fail(ctx, SPG_EINVAL, "spg_get_x: bad arguments");
    return copy_volume_out(ctx, x, ctx->X[ctx->cur()], 4, ctx->vols_h[vol]);
}

spg_status spg_reweight(spg_ctx *ctx)
{
    SPG_TRACE();
    if (!ctx) return fail(nullptr, SPG_EINVAL, "null context");
    for (int j = 0; j < ctx->nvol; j++)
        if (!ctx->data_set[j]) return fail(ctx, SPG_ENOTREADY, "spg_reweight: data not set for every volume");
    const float *xb[1] = {ctx->X[ctx->cur()]};
    CK(launch_reweight(aux_params(ctx), xb, ctx->OM1, ctx->OMTV, ctx->maxw_d, ctx->rstats_d, ctx->vols_d, ctx->stream),
       "reweight");
    ctx->launches += 1;
    ctx->k_round = 0;
    ctx->reweighted = true;
    ctx->y_fresh = false;  // the extrapolation restarts
    return SPG_OK;
}

spg_status spg_iterate(spg_ctx *ctx, int k)
{
    SPG_TRACE();
    if (!ctx) return fail(nullptr, SPG_EINVAL, "null context");
    if (k < 0) return fail(ctx, SPG_EINVAL, "spg_iterate: negative count");
    if (!ctx->reweighted) return fail(ctx, SPG_ENOTREADY, "spg_iterate: call spg_reweight first");
    if ((long long)ctx->k_round + k > ctx->max_iters)
        return fail(ctx, SPG_EINVAL, "spg_iterate: round longer than max_iters_per_round");
    spg_status s = launch_steps(ctx, k);
    if (s != SPG_OK) return s;
    ctx->k_round += k;
    ctx->k_total += k;
    return SPG_OK;
}

spg_status spg_objective(spg_ctx *ctx, int vol, double out[4])
{
    SPG_TRACE();
    if (!ctx) return fail(nullptr, SPG_EINVAL, "null context");
    if (vol < 0 || vol >= ctx->nvol || !out) return fail(ctx, SPG_EINVAL, "spg_objective: bad arguments");
    if (!ctx->reweighted) return fail(ctx, SPG_ENOTREADY, "spg_objective: weights not set (call spg_reweight)");
    const float *xb[1] = {ctx->X[ctx->cur()]};
    CK(launch_objective(aux_params(ctx), xb, ctx->fourier ? nullptr : ctx->B, ctx->fourier ? nullptr : ctx->W,
                        ctx->bf16(), ctx->OM1, ctx->OMTV, ctx->stream),
       "objective");
    ctx->launches += 1;
    double o[8];
    CK(cudaMemcpyAsync(o, ctx->vol_out_d + (size_t)vol * 8, sizeof(o), cudaMemcpyDeviceToHost, ctx->stream),
       "read objective");
    if (ctx->fourier) {
        // data term 1/2 |y - D A x|^2 from the spectrum of x
        const VolDesc &d = ctx->vols_h[0];
        const double V = (double)d.nx * d.ny * d.nz;
        ctx->y_fresh = false;  // the transform below works in the y buffer
        CK(cudaMemcpyAsync(ctx->Ybuf, ctx->X[ctx->cur()], (size_t)ctx->total * sizeof(float), cudaMemcpyDeviceToDevice,
                           ctx->stream),
           "copy x");
        if (spg::cufft_api().exec_r2c(ctx->pr2c, ctx->Ybuf, reinterpret_cast<cufftComplex *>(ctx->Fh)) !=
            CUFFT_SUCCESS)
            return fail(ctx, SPG_ECUDA, "spg_objective: transform");
        if (ctx->zown) {
            CK(launch_zfft(ctx->Fh, ctx->zplan, ctx->ztw, ctx->stream), "transform along z");
            ctx->launches += 1;
        }
        CK(launch_spec_data_value(ctx->Fh, ctx->Yh, ctx->Nh, d.nz, d.ny, d.nx, (float)(1.0 / std::sqrt(V)),
                                  ctx->fpart, ctx->fpart + 1024, ctx->stream),
           "data value");
        ctx->launches += 2;
        double dv = 0;
        CK(cudaMemcpyAsync(&dv, ctx->fpart + 1024, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "read");
        CK(cudaStreamSynchronize(ctx->stream), "synchronise");
        o[0] = dv;
        if (ctx->gamma_f > 0.f) {  // + gamma |x - a|^2
            CK(launch_sq_diff(ctx->X[ctx->cur()], ctx->Anc, d.nx, d.pitch, (long long)d.nz * d.ny * d.pitch, ctx->fpart,
                              ctx->fpart + 1024, ctx->stream),
               "anchor value");
            ctx->launches += 2;
            double sq = 0;
            CK(cudaMemcpyAsync(&sq, ctx->fpart + 1024, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "read");
            CK(cudaStreamSynchronize(ctx->stream), "synchronise");
            o[0] += (double)ctx->gamma_f * sq;
        }
        o[3] = o[0] + o[1] + o[2];
    }
    spg_status s = device_status(ctx);
    if (s != SPG_OK) return s;
    for (int q = 0; q < 4; q++) out[q] = o[q];
    if (!std::isfinite(o[3])) return fail(ctx, SPG_ENONFINITE, "non-finite objective");
    return SPG_OK;
}

spg_status spg_history(spg_ctx *ctx, int vol, double *host, int max_entries, int *n)
{
    SPG_TRACE();
    if (!ctx) return fail(nullptr, SPG_EINVAL, "null context");
    if (vol < 0 || vol >= ctx->nvol || !n || max_entries < 0 || (max_entries > 0 && !host))
        return fail(ctx, SPG_EINVAL, "spg_history: bad arguments");
    DevState st;
    CK(cudaMemcpyAsync(&st, ctx->st_d, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream), "read state");
    std::vector<double> ring((size_t)ctx->hist_cap * ctx->nvol * 5);
    CK(cudaMemcpyAsync(ring.data(), ctx->hist_d, ring.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
       "read history");
    spg_status s = device_status(ctx);
    if (s != SPG_OK) return s;
    const long long total = st.hist_count;
    const long long avail = std::min<long long>(total, ctx->hist_cap);
    const long long take = std::min<long long>(avail, max_entries);
    for (long long i = 0; i < take; i++) {
        const long long e = total - take + i;
        const double *src = ring.data() + ((size_t)(e % ctx->hist_cap) * ctx->nvol + vol) * 5;
        std::memcpy(host + i * 5, src, 5 * sizeof(double));
    }
    *n = (int)take;
    return SPG_OK;
}

spg_status spg_round_stats(spg_ctx *ctx, int vol, double out[6])
{
    SPG_TRACE();
    if (!ctx) return fail(nullptr, SPG_EINVAL, "null context");
    if (vol < 0 || vol >= ctx->nvol || !out) return fail(ctx, SPG_EINVAL, "spg_round_stats: bad arguments");
    CK(cudaMemcpyAsync(out, ctx->rstats_d + (size_t)vol * 6, 6 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
       "read round stats");
    return device_status(ctx);
}

// ---------------- z-slab decomposition of one volume ----------------

spg_status spg_set_halo(spg_ctx *ctx, int vol, int lo, int hi)
{
    SPG_TRACE();
    if (!ctx) return fail(nullptr, SPG_EINVAL, "null context");
    if (vol < 0 || vol >= ctx->nvol || (lo != 0 && lo != 1) || (hi != 0 && hi != 1))
        return fail(ctx, SPG_EINVAL, "spg_set_halo: bad arguments");
    if (ctx->kread || ctx->opt.restart || ctx->fourier)
        return fail(ctx, SPG_EINVAL,
                    "spg_set_halo: needs the adopted readings, no gradient restart and the real-space data term");
    VolDesc &d = ctx->vols_h[vol];
    if (d.nz - lo - hi < 1) return fail(ctx, SPG_EINVAL, "spg_set_halo: no interior plane left");
    d.halo_lo = lo;
    d.halo_hi = hi;
    return build_plan(ctx, ctx->var, ctx->opt.zchunk);  // items over the interior; descriptors uploaded
}

spg_status spg_step_bound(spg_ctx *ctx, int vol, double out[2])
{
    SPG_TRACE();
    if (!ctx) return fail(nullptr, SPG_EINVAL, "null context");
    if (vol < 0 || vol >= ctx->nvol || !out) return fail(ctx, SPG_EINVAL, "spg_step_bound: bad arguments");
    if (!ctx->reweighted) return fail(ctx, SPG_ENOTREADY, "spg_step_bound: call spg_reweight first");
    double mw = 0.0, st[6];
    CK(cudaMemcpyAsync(&mw, ctx->maxw_d + vol, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "read max w");
    CK(cudaMemcpyAsync(st, ctx->rstats_d + (size_t)vol * 6, 6 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
       "read round stats");
    spg_status s = device_status(ctx);
    if (s != SPG_OK) return s;
    out[0] = mw;
    out[1] = st[0];
    return SPG_OK;
}

spg_status spg_set_lambdas(spg_ctx *ctx, int vol, float lambda_l1, float lambda_tv)
{
    SPG_TRACE();
    if (!ctx) return fail(nullptr, SPG_EINVAL, "null context");
    if (vol < 0 || vol >= ctx->nvol || !std::isfinite(lambda_l1) || !std::isfinite(lambda_tv) ||
        !(lambda_l1 >= 0.f) || !(lambda_tv >= 0.f))
        return fail(ctx, SPG_EINVAL, "spg_set_lambdas: bad arguments");
    // only these two fields of the device descriptor: tau and the
    // extrapolation index there belong to the device
    const float l[2] = {lambda_l1, lambda_tv};
    static_assert(offsetof(VolDesc, lambda_tv) == offsetof(VolDesc, lambda_l1) + sizeof(float),
                  "lambda_l1 and lambda_tv are adjacent");
    CK(cudaMemcpyAsync(reinterpret_cast<char *>(ctx->vols_d + vol) + offsetof(VolDesc, lambda_l1), l, sizeof(l),
                       cudaMemcpyHostToDevice, ctx->stream),
       "write lambdas");
    CK(cudaStreamSynchronize(ctx->stream), "synchronise");
    ctx->vols_h[vol].lambda_l1 = lambda_l1;
    ctx->vols_h[vol].lambda_tv = lambda_tv;
    ctx->vp[vol].lambda_l1 = lambda_l1;
    ctx->vp[vol].lambda_tv = lambda_tv;
    ctx->reweighted = false;  // tau depends on lambda_tv
    return SPG_OK;
}

spg_status spg_set_step_bound(spg_ctx *ctx, int vol, double max_w, double max_omtv)
{
    SPG_TRACE();
    if (!ctx) return fail(nullptr, SPG_EINVAL, "null context");
    if (vol < 0 || vol >= ctx->nvol || !std::isfinite(max_w) || !std::isfinite(max_omtv) || !(max_w > 0.0) ||
        !(max_omtv >= 0.0))
        return fail(ctx, SPG_EINVAL, "spg_set_step_bound: bad arguments");
    if (!ctx->reweighted || ctx->k_round != 0)
        return fail(ctx, SPG_ENOTREADY, "spg_set_step_bound: call it after spg_reweight, before the round's first step");
    const VolDesc &d = ctx->vols_h[vol];
    // the re-weighting kernel's expression, evaluated in the same order
    const double L = max_w + 12.0 * (double)d.lambda_tv * max_omtv / (double)d.mu;
    const double tau = 1.0 / L;
    const float tf = (float)tau;
    const double lt[2] = {L, tau};
    CK(cudaMemcpyAsync(reinterpret_cast<char *>(ctx->vols_d + vol) + offsetof(VolDesc, tau), &tf, sizeof(float),
                       cudaMemcpyHostToDevice, ctx->stream),
       "write step");
    CK(cudaMemcpyAsync(ctx->rstats_d + (size_t)vol * 6 + 4, lt, 2 * sizeof(double), cudaMemcpyHostToDevice,
                       ctx->stream),
       "write round stats");
    CK(cudaStreamSynchronize(ctx->stream), "synchronise");
    ctx->vols_h[vol].tau = tf;
    return SPG_OK;
}

// planes [z0, z0 + n) of the current iterate x_k and of its pair (d_k or
// x_{k-1}) between the context and a caller's contiguous [n][ny][nx] arrays
static spg_status copy_planes(spg_ctx *ctx, int vol, int z0, int n, float *x, float *pair, bool in, const char *who)
{
    if (!ctx) return fail(nullptr, SPG_EINVAL, "null context");
    if (vol < 0 || vol >= ctx->nvol || n < 1 || z0 < 0 || (!x && !pair))
        return fail(ctx, SPG_EINVAL, std::string(who) + ": bad arguments");
    const VolDesc &d = ctx->vols_h[vol];
    if ((long long)z0 + n > d.nz) return fail(ctx, SPG_EINVAL, std::string(who) + ": planes outside the volume");
    if (ctx->reversed || ctx->kread) return fail(ctx, SPG_EINVAL, std::string(who) + ": needs the adopted readings");
    const int c = ctx->cur();
    float *bufs[2] = {ctx->X[c], ctx->X[ctx->aux_of(c)]};
    float *user[2] = {x, pair};
    for (int q = 0; q < 2; q++) {
        if (!user[q]) continue;
        float *dev = bufs[q] + d.off + (size_t)z0 * d.ny * d.pitch;
        const size_t dp = (size_t)d.pitch * sizeof(float), up = (size_t)d.nx * sizeof(float);
        if (in)
            CK(cudaMemcpy2DAsync(dev, dp, user[q], up, up, (size_t)d.ny * n, cudaMemcpyDefault, ctx->stream),
               "copy planes in");
        else
            CK(cudaMemcpy2DAsync(user[q], up, dev, dp, up, (size_t)d.ny * n, cudaMemcpyDefault, ctx->stream),
               "copy planes out");
    }
    if (in) ctx->y_fresh = false;
    CK(cudaStreamSynchronize(ctx->stream), "synchronise");
    return SPG_OK;
}

spg_status spg_get_planes(spg_ctx *ctx, int vol, int z0, int n, float *x, float *pair)
{
    SPG_TRACE();
    return copy_planes(ctx, vol, z0, n, x, pair, false, "spg_get_planes");
}

spg_status spg_set_planes(spg_ctx *ctx, int vol, int z0, int n, const float *x, const float *pair)
{
    SPG_TRACE();
    return copy_planes(ctx, vol, z0, n, const_cast<float *>(x), const_cast<float *>(pair), true, "spg_set_planes");
}

spg_status spg_certificate(spg_ctx *ctx, int vol, double *out)
{
    SPG_TRACE();
    if (!ctx) return fail(nullptr, SPG_EINVAL, "null context");
    if (vol < 0 || vol >= ctx->nvol || !out) return fail(ctx, SPG_EINVAL, "spg_certificate: bad arguments");
    if (ctx->kread) return fail(ctx, SPG_EINVAL, "spg_certificate: not available with these readings");
    if (!ctx->reweighted || ctx->k_round < 1)
        return fail(ctx, SPG_ENOTREADY, "spg_certificate: needs one iteration in the current round");
    if (ctx->fourier) return fail(ctx, SPG_EINVAL, "spg_certificate: not available with the Fourier-domain data term");
    const int c = ctx->cur();
    // x_{k+1} = X[c]; x_k and its pair are one rotation back
    const int k = (c + ctx->nbuf() - 1) % ctx->nbuf();
    const float *xb[4] = {ctx->X[c], ctx->X[k], ctx->xd() ? nullptr : ctx->X[ctx->aux_of(k)],
                          ctx->xd() ? ctx->X[ctx->aux_of(k)] : nullptr};
    if (!ctx->certQ) CK(dalloc(&ctx->certQ, (size_t)ctx->total * 3 * sizeof(float)), "alloc certificate field");
    CK(launch_certificate4(aux_params(ctx), xb, ctx->W, ctx->bf16(), ctx->OMTV, ctx->certQ, ctx->total, ctx->stream),
       "certificate");
    ctx->launches += 2;
    double o[8];
    CK(cudaMemcpyAsync(o, ctx->vol_out_d + (size_t)vol * 8, sizeof(o), cudaMemcpyDeviceToHost, ctx->stream),
       "read certificate");
    spg_status s = device_status(ctx);
    if (s != SPG_OK) return s;
    *out = o[4];
    return SPG_OK;
}

spg_status spg_counters(spg_ctx *ctx, long long *k_total, int *k_round)
{
    SPG_TRACE();
    if (!ctx) return fail(nullptr, SPG_EINVAL, "null context");
    if (k_total) *k_total = ctx->k_total;
    if (k_round) *k_round = ctx->k_round;
    return SPG_OK;
}

// ---------------- checkpoint / resume ----------------

spg_status spg_get_state(spg_ctx *ctx, void *blob, size_t *size)
{
    SPG_TRACE();
    if (!ctx || !size) return fail(ctx, SPG_EINVAL, "spg_get_state: bad arguments");
    size_t need = sizeof(StateHeader);
    for (const auto &d : ctx->vols_h)
        need += 4 * (size_t)d.nx * d.ny * d.nz * 4 + 2 * sizeof(float) + sizeof(int32_t) + sizeof(int32_t) +
                6 * sizeof(double);
    if (!blob) {
        *size = need;
        return SPG_OK;
    }
    if (*size < need) return fail(ctx, SPG_EINVAL, "spg_get_state: buffer too small");
    char *p = static_cast<char *>(blob);
    StateHeader h{kStateMagic, 3, ctx->nvol, ctx->k_round, ctx->reweighted ? 1 : 0, ctx->k_total,
                  (int32_t)ctx->opt.data_dtype, (int32_t)ctx->opt.momentum, (int32_t)ctx->opt.iterate_storage, 0};
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    std::vector<VolDesc> dev(ctx->nvol);
    CK(cudaMemcpyAsync(dev.data(), ctx->vols_d, ctx->nvol * sizeof(VolDesc), cudaMemcpyDeviceToHost, ctx->stream),
       "read descriptors");
    const int c = ctx->cur();
    for (int j = 0; j < ctx->nvol; j++) {
        const VolDesc &d = ctx->vols_h[j];
        const size_t vb = (size_t)d.nx * d.ny * d.nz * 4;
        spg_status s;
        if ((s = copy_volume_out(ctx, p, ctx->X[c], 4, d)) != SPG_OK) return s;
        p += vb;
        if ((s = copy_volume_out(ctx, p, ctx->X[ctx->aux_of(c)], 4, d)) != SPG_OK) return s;
        p += vb;
        if ((s = copy_volume_out(ctx, p, ctx->OM1, 4, d)) != SPG_OK) return s;
        p += vb;
        if ((s = copy_volume_out(ctx, p, ctx->OMTV, 4, d)) != SPG_OK) return s;
        p += vb;
        CK(cudaStreamSynchronize(ctx->stream), "synchronise");
        std::memcpy(p, &dev[j].tau, sizeof(float));
        p += sizeof(float);
        std::memcpy(p, &dev[j].beta_last, sizeof(float));
        p += sizeof(float);
        const int32_t km[2] = {dev[j].kmom, 0};
        std::memcpy(p, km, sizeof(km));
        p += sizeof(km);
        CK(cudaMemcpyAsync(p, ctx->rstats_d + (size_t)j * 6, 6 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
           "read stats");
        p += 6 * sizeof(double);
    }
    return device_status(ctx);
}

spg_status spg_set_state(spg_ctx *ctx, const void *blob, size_t size)
{
    SPG_TRACE();
    if (!ctx || !blob) return fail(ctx, SPG_EINVAL, "spg_set_state: bad arguments");
    size_t need = 0;
    spg_get_state(ctx, nullptr, &need);
    if (size < need) return fail(ctx, SPG_EINVAL, "spg_set_state: blob too small");
    ctx->y_fresh = false;
    const char *p = static_cast<const char *>(blob);
    StateHeader h;
    std::memcpy(&h, p, sizeof(h));
    p += sizeof(h);
    if (h.magic != kStateMagic || h.version != 3 || h.nvol != ctx->nvol || h.dtype != (int)ctx->opt.data_dtype ||
        h.momentum != (int)ctx->opt.momentum || h.storage != (int)ctx->opt.iterate_storage)
        return fail(ctx, SPG_EINVAL, "spg_set_state: blob does not match this context");
    CK(cudaStreamSynchronize(ctx->stream), "synchronise");
    // x_k goes to X[0] and its pair (d_k or x_{k-1}) to its pair buffer; the
    // device state names X[0] as current
    std::vector<VolDesc> dev(ctx->nvol);
    CK(cudaMemcpy(dev.data(), ctx->vols_d, ctx->nvol * sizeof(VolDesc), cudaMemcpyDeviceToHost), "read descriptors");
    for (int j = 0; j < ctx->nvol; j++) {
        const VolDesc &d = ctx->vols_h[j];
        const size_t vb = (size_t)d.nx * d.ny * d.nz * 4;
        spg_status s;
        if ((s = copy_volume_in(ctx, ctx->X[0], 4, d, p)) != SPG_OK) return s;
        p += vb;
        if ((s = copy_volume_in(ctx, ctx->X[ctx->aux_of(0)], 4, d, p)) != SPG_OK) return s;
        p += vb;
        if ((s = copy_volume_in(ctx, ctx->OM1, 4, d, p)) != SPG_OK) return s;
        p += vb;
        if ((s = copy_volume_in(ctx, ctx->OMTV, 4, d, p)) != SPG_OK) return s;
        p += vb;
        std::memcpy(&dev[j].tau, p, sizeof(float));
        ctx->vols_h[j].tau = dev[j].tau;
        p += sizeof(float);
        std::memcpy(&dev[j].beta_last, p, sizeof(float));
        p += sizeof(float);
        int32_t km[2];
        std::memcpy(km, p, sizeof(km));
        dev[j].kmom = km[0];
        p += sizeof(km);
        CK(cudaMemcpyAsync(ctx->rstats_d + (size_t)j * 6, p, 6 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream),
           "write stats");
        CK(cudaStreamSynchronize(ctx->stream), "synchronise");
        p += 6 * sizeof(double);
    }
    CK(cudaMemcpy(ctx->vols_d, dev.data(), ctx->nvol * sizeof(VolDesc), cudaMemcpyHostToDevice), "write descriptors");
    DevState st;
    CK(cudaMemcpy(&st, ctx->st_d, sizeof(st), cudaMemcpyDeviceToHost), "read state");
    st.cur = 0;
    st.k_round = h.k_round;
    st.k_total = h.k_total;
    st.ticket = 0;
    st.ticket_aux = 0;
    st.err = 0;
    CK(cudaMemcpy(ctx->st_d, &st, sizeof(st), cudaMemcpyHostToDevice), "write state");
    ctx->k_round = h.k_round;
    ctx->k_total = h.k_total;
    ctx->cur0 = (int)(((-h.k_total) % ctx->nbuf() + ctx->nbuf()) % ctx->nbuf());
    ctx->reweighted = h.reweighted != 0;
    return SPG_OK;
}

// ---------------- unrolled forward and adjoint (single volume) ----------------

spg_status spg_unrolled(spg_ctx *ctx, int K, float *xK)
{
    SPG_TRACE();
    if (!ctx || !xK || K < 0) return fail(ctx, SPG_EINVAL, "spg_unrolled: bad arguments");
    if (ctx->nvol != 1) return fail(ctx, SPG_EINVAL, "spg_unrolled: single-volume contexts only");
    if (ctx->fourier) return fail(ctx, SPG_EINVAL, "spg_unrolled: not available with the Fourier-domain data term");
    if (ctx->kread) return fail(ctx, SPG_EINVAL, "spg_unrolled: not available with these readings");
    if (!ctx->reweighted) return fail(ctx, SPG_ENOTREADY, "spg_unrolled: call spg_reweight first");
    if (K > ctx->max_iters) return fail(ctx, SPG_EINVAL, "spg_unrolled: K above max_iters_per_round");
    const VolDesc &d = ctx->vols_h[0];
    const size_t vb = (size_t)ctx->total * 4;
    // three rotating iterate buffers, then the steps' state
    Carve cv;
    {
        Carve size;
        for (int q = 0; q < 3; q++) size.take<float>(vb);
        DevState *s0;
        VolDesc *v0;
        TmapSet *t0;
        Sweep::carve(size, (size_t)K, &s0, &v0, &t0);
        CK(workspace(ctx, size.off, &cv.base), "alloc workspace");
    }
    float *buf[3];
    for (int q = 0; q < 3; q++) buf[q] = cv.take<float>(vb);
    CK(cudaMemcpyAsync(buf[0], ctx->X[ctx->cur()], vb, cudaMemcpyDeviceToDevice, ctx->stream), "copy x0");
    CK(cudaMemcpyAsync(buf[2], buf[0], vb, cudaMemcpyDeviceToDevice, ctx->stream), "copy x0");
    Sweep sw(ctx);
    int c = 0;
    for (int k = 0; k < K; k++) {
        sw.add(buf[c], buf[(c + 2) % 3], buf[(c + 1) % 3], k);
        c = (c + 1) % 3;
    }
    CK(sw.upload(cv), "plan the unrolled steps");
    for (int k = 0; k < K; k++) CK(sw.launch(), "fused step");
    spg_status s = sw.status();
    if (s != SPG_OK) return fail(ctx, s, "spg_unrolled: a fused step failed");
    s = copy_volume_out(ctx, xK, buf[c], 4, d);
    if (s != SPG_OK) return s;
    return device_status(ctx);
}

spg_status spg_backward(spg_ctx *ctx, int K, const float *gx, float *gb, float *gw, double g_scalars[2],
                        int ckpt_every)
{
    SPG_TRACE();
    if (!ctx || !gx || !gb || !gw || !g_scalars || K < 1) return fail(ctx, SPG_EINVAL, "spg_backward: bad arguments");
    if (ctx->nvol != 1) return fail(ctx, SPG_EINVAL, "spg_backward: single-volume contexts only");
    if (ctx->fourier) return fail(ctx, SPG_EINVAL, "spg_backward: not available with the Fourier-domain data term");
    if (ctx->kread) return fail(ctx, SPG_EINVAL, "spg_backward: not available with these readings");
    if (!ctx->reweighted) return fail(ctx, SPG_ENOTREADY, "spg_backward: call spg_reweight first");
    if (K > ctx->max_iters) return fail(ctx, SPG_EINVAL, "spg_backward: K above max_iters_per_round");
    const int C = ckpt_every > 0 ? ckpt_every : 10;
    const VolDesc &d = ctx->vols_h[0];
    const size_t vb = (size_t)ctx->total * 4;
    const int nck = (K + C - 1) / C;  // checkpoints at k = 0, C, 2C, ... (< K)
    // one forward sweep plus, per segment, the recomputation of all but its last step
    const size_t nsteps = (size_t)K + (size_t)(K - nck);
    // workspace: checkpoints, segment, adjoint volumes, scalar partials, the steps' state
    float *ck = nullptr, *seg = nullptr, *ga[3], *m = nullptr, *accb = nullptr, *accw = nullptr;
    double *pp = nullptr;
    const int nblk = adjoint_blocks(d.nx, d.ny, d.nz);  // CTAs of each adjoint pass, one scalar partial each
    Carve cv;
    for (int pass = 0; pass < 2; pass++) {
        Carve t;
        t.base = cv.base;
        ck = t.take<float>(vb * 2 * nck);
        seg = t.take<float>(vb * (C + 2));
        for (int q = 0; q < 3; q++) ga[q] = t.take<float>(vb);
        m = t.take<float>(vb);
        accb = t.take<float>(vb);
        accw = t.take<float>(vb);
        pp = t.take<double>((size_t)K * nblk * 4 * sizeof(double));
        if (pass == 0) {
            DevState *s0;
            VolDesc *v0;
            TmapSet *t0;
            Sweep::carve(t, nsteps, &s0, &v0, &t0);
            CK(workspace(ctx, t.off, &cv.base), "alloc workspace");
        } else {
            cv = t;  // the steps' state follows
        }
    }
    const auto beta = beta_table_host(ctx, K);
    auto vol_at = [&](float *base, int i) { return base + (size_t)i * ctx->total; };

    // Plan every forward step through the fused kernel: the sweep from x_0
    // (three rotating buffers, checkpoints of (x_k, x_{k-1}) copied out every
    // C steps) and, per segment in reverse order, the recomputation of the
    // segment's iterates from its checkpoint into seg[1..].
    Sweep sw(ctx);
    float *b3[3];
    for (int q = 0; q < 3; q++) b3[q] = vol_at(seg, q);
    {
        int c = 0;
        for (int k = 0; k < K; k++) {
            sw.add(b3[c], b3[(c + 2) % 3], b3[(c + 1) % 3], k);
            c = (c + 1) % 3;
        }
        for (int sgm = nck - 1; sgm >= 0; sgm--) {
            const int k0 = sgm * C, k1 = std::min(K, k0 + C);
            for (int k = k0; k < k1 - 1; k++) {
                const int i = k - k0 + 1;
                sw.add(vol_at(seg, i), vol_at(seg, i - 1), vol_at(seg, i + 1), k);
            }
        }
    }
    if (sw.plan.size() != nsteps) return fail(ctx, SPG_EINVAL, "spg_backward: step plan size mismatch");
    CK(sw.upload(cv), "plan the forward steps");
    // forward sweep, keeping (x_k, x_{k-1}) at every checkpoint
    {
        CK(cudaMemcpyAsync(b3[0], ctx->X[ctx->cur()], vb, cudaMemcpyDeviceToDevice, ctx->stream), "copy x0");
        CK(cudaMemcpyAsync(b3[2], b3[0], vb, cudaMemcpyDeviceToDevice, ctx->stream), "copy x0");
        int c = 0;
        for (int k = 0; k < K; k++) {
            if (k % C == 0) {
                CK(cudaMemcpyAsync(vol_at(ck, 2 * (k / C)), b3[c], vb, cudaMemcpyDeviceToDevice, ctx->stream), "ckpt");
                CK(cudaMemcpyAsync(vol_at(ck, 2 * (k / C) + 1), b3[(c + 2) % 3], vb, cudaMemcpyDeviceToDevice,
                                   ctx->stream),
                   "ckpt");
            }
            CK(sw.launch(), "fused step");
            c = (c + 1) % 3;
        }
    }
    // adjoint sweep
    CK(cudaMemsetAsync(accb, 0, vb, ctx->stream), "memset");
    CK(cudaMemsetAsync(accw, 0, vb, ctx->stream), "memset");
    CK(cudaMemsetAsync(ga[0], 0, vb, ctx->stream), "memset");
    CK(cudaMemsetAsync(ga[1], 0, vb, ctx->stream), "memset");
    CK(cudaMemsetAsync(ga[2], 0, vb, ctx->stream), "memset");
    spg_status s = copy_volume_in(ctx, ga[0], 4, d, gx);  // ga[0] = dL/dx_K
    if (s != SPG_OK) return s;
    int inext = 0, icur = 1, iprev = 2;
    for (int sgm = nck - 1; sgm >= 0; sgm--) {
        const int k0 = sgm * C, k1 = std::min(K, k0 + C);
        // seg[0] = x_{k0-1}, seg[1] = x_{k0}, seg[i+1] = x_{k0+i}
        CK(cudaMemcpyAsync(vol_at(seg, 0), vol_at(ck, 2 * sgm + 1), vb, cudaMemcpyDeviceToDevice, ctx->stream), "rst");
        CK(cudaMemcpyAsync(vol_at(seg, 1), vol_at(ck, 2 * sgm), vb, cudaMemcpyDeviceToDevice, ctx->stream), "rst");
        for (int k = k0; k < k1 - 1; k++) CK(sw.launch(), "recompute");
        for (int k = k1 - 1; k >= k0; k--) {
            const int i = k - k0 + 1;
            AdjParams a;
            a.vols = ctx->vols_d;
            a.nplanes = d.nz;
            a.xk = vol_at(seg, i);
            a.xkm1 = vol_at(seg, i - 1);
            a.beta = beta[k];
            a.b = ctx->B;
            a.w = ctx->W;
            a.bf16 = ctx->bf16();
            a.om1 = ctx->OM1;
            a.omtv = ctx->OMTV;
            a.gnext = ga[inext];
            a.m = m;
            a.gcur = ga[icur];
            // x_{-1} = x_0: the k = 0 step's extrapolation cotangent folds into dL/dx_0
            a.gprev = k >= 1 ? ga[iprev] : ga[icur];
            a.gb = accb;
            a.gw = accw;
            a.plane_part = pp + (size_t)k * nblk * 4;
            a.nblocks = nblk;
            a.prev_fresh = k >= 1 ? 1 : 0;  // dL/dx_{k-1} gets its first contribution here
            CK(launch_adjoint_mask(a, ctx->stream), "adjoint mask");
            CK(launch_adjoint_apply(a, ctx->stream), "adjoint apply");
            ctx->launches += 2;
            // rotate: dL/dx_k is complete; the old dL/dx_{k+1} buffer becomes dL/dx_{k-2},
            // which the next step writes (no clearing needed)
            const int t = inext;
            inext = icur;
            icur = iprev;
            iprev = t;
        }
    }
    if ((s = copy_volume_out(ctx, gb, accb, 4, d)) != SPG_OK) return s;
    if ((s = copy_volume_out(ctx, gw, accw, 4, d)) != SPG_OK) return s;
    const size_t segs = (size_t)nblk;
    std::vector<double> hp((size_t)K * segs * 4);
    CK(cudaMemcpyAsync(hp.data(), pp, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "read");
    CK(cudaStreamSynchronize(ctx->stream), "synchronise");
    double s1 = 0, s2 = 0;
    for (int k = K - 1; k >= 0; k--)
        for (size_t q = 0; q < segs; q++) {
            s1 += hp[((size_t)k * segs + q) * 4 + 0];
            s2 += hp[((size_t)k * segs + q) * 4 + 1];
        }
    g_scalars[0] = s1;
    g_scalars[1] = s2;
    return device_status(ctx);
}

spg_status spg_probe_timeout(spg_ctx *ctx, long long timeout_ns)
{
    SPG_TRACE();
    if (!ctx || timeout_ns <= 0 || timeout_ns > kTimeoutNs) return fail(ctx, SPG_EINVAL, "spg_probe_timeout: bad arguments");
    CK(launch_timeout_probe(ctx->st_d, timeout_ns, ctx->stream), "timeout probe");
    ctx->launches += 1;
    return device_status(ctx);
}

namespace {

std::string tune_key(const spg_ctx *ctx)
{
    cudaDeviceProp prop;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    std::string k = std::string(prop.name) + "|" + std::to_string(prop.multiProcessorCount) + "|" +
                    (ctx->bf16() ? "bf16" : "f32") + "|" + (ctx->xd() ? "delta" : "prev") + "|";
    for (const auto &d : ctx->vols_h) k += std::to_string(d.nx) + "x" + std::to_string(d.ny) + "x" + std::to_string(d.nz) + ";";
    for (auto &c : k)
        if (c == ' ') c = '_';
    return k;
}

bool cache_lookup(const std::string &key, int *tile, int *zchunk)
{
    const char *path = std::getenv("SPG_AUTOTUNE_CACHE");
    if (!path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char kbuf[4096];
    int t = 0, z = 0;
    bool found = false;
    while (std::fscanf(f, "%4095s %d %d", kbuf, &t, &z) == 3)
        if (key == kbuf) {
            *tile = t;
            *zchunk = z;
            found = true;
        }
    std::fclose(f);
    return found;
}

void cache_store(const std::string &key, int tile, int zchunk)
{
    const char *path = std::getenv("SPG_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d\n", key.c_str(), tile, zchunk);
    std::fclose(f);
}

}  // namespace

spg_status spg_autotune(spg_ctx *ctx, int trial_iters, int info[6])
{
    SPG_TRACE();
    if (!ctx || trial_iters < 1) return fail(ctx, SPG_EINVAL, "spg_autotune: bad arguments");
    if (ctx->kread) return fail(ctx, SPG_EINVAL, "spg_autotune: not available with these readings");
    if (!ctx->reweighted) return fail(ctx, SPG_ENOTREADY, "spg_autotune: call spg_reweight first");
    ctx->y_fresh = false;
    const std::string key = tune_key(ctx);
    int tile = 0, zc = 0;
    spg_status s;
    if (cache_lookup(key, &tile, &zc)) {
        s = build_plan(ctx, variant_from_tile(tile, ctx->bf16(), ctx->xd()), zc);
        if (s != SPG_OK) return s;
        return spg_plan_info(ctx, info);
    }
    // save what the trial iterations change: the iterate pair, device state, history ring
    const size_t vb = (size_t)ctx->total * 4;
    const int c0 = ctx->cur();
    Scratch sc;
    float *sx = nullptr, *sa = nullptr;
    CK(sc.get(&sx, vb), "alloc");
    CK(sc.get(&sa, vb), "alloc");
    CK(cudaMemcpyAsync(sx, ctx->X[c0], vb, cudaMemcpyDeviceToDevice, ctx->stream), "save");
    CK(cudaMemcpyAsync(sa, ctx->X[ctx->aux_of(c0)], vb, cudaMemcpyDeviceToDevice, ctx->stream), "save");
    DevState st0;
    CK(cudaMemcpyAsync(&st0, ctx->st_d, sizeof(st0), cudaMemcpyDeviceToHost, ctx->stream), "save state");
    std::vector<double> hist0((size_t)ctx->hist_cap * ctx->nvol * 5);
    CK(cudaMemcpyAsync(hist0.data(), ctx->hist_d, hist0.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
       "save history");
    std::vector<VolDesc> vd0(ctx->nvol);  // device-owned tau and extrapolation index
    CK(cudaMemcpyAsync(vd0.data(), ctx->vols_d, ctx->nvol * sizeof(VolDesc), cudaMemcpyDeviceToHost, ctx->stream),
       "save descriptors");
    CK(cudaStreamSynchronize(ctx->stream), "synchronise");
    const long long kt0 = ctx->k_total;
    const int kr0 = ctx->k_round;
    auto restore = [&]() -> spg_status {
        std::vector<VolDesc> cur(ctx->nvol);
        CK(cudaMemcpyAsync(cur.data(), ctx->vols_d, ctx->nvol * sizeof(VolDesc), cudaMemcpyDeviceToHost,
                           ctx->stream),
           "read descriptors");
        CK(cudaStreamSynchronize(ctx->stream), "synchronise");
        for (int j = 0; j < ctx->nvol; j++) {
            cur[j].tau = vd0[j].tau;
            cur[j].kmom = vd0[j].kmom;
            cur[j].beta_last = vd0[j].beta_last;
        }
        CK(cudaMemcpyAsync(ctx->vols_d, cur.data(), ctx->nvol * sizeof(VolDesc), cudaMemcpyHostToDevice,
                           ctx->stream),
           "restore descriptors");
        CK(cudaMemcpyAsync(ctx->X[c0], sx, vb, cudaMemcpyDeviceToDevice, ctx->stream), "restore");
        CK(cudaMemcpyAsync(ctx->X[ctx->aux_of(c0)], sa, vb, cudaMemcpyDeviceToDevice, ctx->stream), "restore");
        CK(cudaMemcpyAsync(ctx->st_d, &st0, sizeof(st0), cudaMemcpyHostToDevice, ctx->stream), "restore state");
        CK(cudaMemcpyAsync(ctx->hist_d, hist0.data(), hist0.size() * sizeof(double), cudaMemcpyHostToDevice,
                           ctx->stream),
           "restore history");
        CK(cudaStreamSynchronize(ctx->stream), "synchronise");
        ctx->k_total = kt0;
        ctx->k_round = kr0;
        return SPG_OK;
    };
    const int tiles[] = {SPG_TILE_128x7, SPG_TILE_128x7_S4, SPG_TILE_128x8, SPG_TILE_128x15,
                         SPG_TILE_128x4, SPG_TILE_64x7,     SPG_TILE_64x8,  SPG_TILE_64x4};
    const int zchunks[] = {0, 64, 32};
    const int trial = std::min(trial_iters, ctx->max_iters - ctx->k_round - 4);
    if (trial < 1) return fail(ctx, SPG_EINVAL, "spg_autotune: no room left in the round for trials");
    float best_ms = 1e30f;
    int best_tile = tile_code(ctx->var), best_z = ctx->opt.zchunk;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    for (int t : tiles)
        for (int z : zchunks) {
            if ((s = build_plan(ctx, variant_from_tile(t, ctx->bf16(), ctx->xd()), z)) != SPG_OK) continue;
            if ((s = launch_steps(ctx, 2)) != SPG_OK) break;  // warm-up (graph capture happens here too)
            cudaEventRecord(e0, ctx->stream);
            if ((s = launch_steps(ctx, trial)) != SPG_OK) break;
            cudaEventRecord(e1, ctx->stream);
            CK(cudaEventSynchronize(e1), "time trial");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                best_tile = t;
                best_z = z;
            }
            if ((s = restore()) != SPG_OK) break;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    spg_status rs = restore();
    if (rs != SPG_OK) return rs;
    if ((s = build_plan(ctx, variant_from_tile(best_tile, ctx->bf16(), ctx->xd()), best_z)) != SPG_OK) return s;
    cache_store(key, best_tile, best_z);
    spg_status ds = device_status(ctx);
    if (ds != SPG_OK) return ds;
    return spg_plan_info(ctx, info);
}

long long spg_launch_count(const spg_ctx *ctx) { return ctx ? ctx->launches : 0; }

spg_status spg_plan_info(const spg_ctx *ctx, int info[6])
{
    SPG_TRACE();
    if (!ctx || !info) return SPG_EINVAL;
    info[0] = 32 * ctx->var.vx;
    info[1] = ctx->var.ty;
    info[2] = ctx->zchunk;
    info[3] = ctx->nitems;
    info[4] = ctx->grid;
    info[5] = ctx->ctas_per_sm;
    return SPG_OK;
}

const char *spg_last_error(const spg_ctx *ctx) { return ctx ? ctx->err.c_str() : g_last_error.c_str(); }

void spg_destroy(spg_ctx *ctx)
{
    SPG_TRACE();
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    delete ctx;
}

}  // extern "C"
