// The C-ABI of libpkmom (include/pkmom.h): argument checking, the per-call
// assignment plan (sort-key segment length, deposit tile, scratch layout),
// cached cuFFT plans and per-grid tables, context-owned buffers for
// pkmom_estimate / pkmom_estimate_host, stage timing with CUDA events.
#include <cufft.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include "pkmom_internal.cuh"

using namespace pkmom;

struct PlanEntry {
    int ng, prec;
    cufftHandle h;
    size_t work;  // bytes of the workspace cuFFT allocated for the plan
    int batch;    // grids per execution: 4 (the whole set) for small grids, else 1
};

// Grids up to this size are transformed four at a time by one plan: at 128^3 a plan
// over the four grids took half the time per grid of one grid per plan (measured; from
// 256^3 on the time per grid was the same either way).
constexpr int kFftBatchMaxNg = 128;

struct TimedEvent {
    int stage;
    cudaEvent_t a, b;
};

struct pkmom_ctx {
    int device = 0;
    int num_sms = 0;
    std::string last_error;
    int *d_err = nullptr;  // device-side data error word
    LaunchStats st;
    std::vector<PlanEntry> plans;
    // a deque: the addresses of cached tables stay valid while more are added (a batch
    // holds pointers to several of them at once)
    std::deque<SpectraTables> tables;
    // buffers owned for pkmom_estimate / pkmom_estimate_host
    void *grids = nullptr;
    size_t grids_bytes = 0;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    double *moments = nullptr;
    double *out_dev = nullptr;
    size_t out_bytes = 0;
    void *staging = nullptr;
    size_t staging_bytes = 0;
    // pkmom_estimate_host_async: two staging slots filled on a copy stream, the events
    // that order them against the estimates, and a ring of completion events by ticket
    static constexpr int kRing = 8;
    void *aslot[2] = {nullptr, nullptr};
    size_t aslot_bytes[2] = {0, 0};
    cudaStream_t copy_stream = nullptr;
    cudaStream_t aux_stream = nullptr;  // reads of the error word
    cudaEvent_t slot_copied[2] = {nullptr, nullptr};
    cudaEvent_t slot_free[2] = {nullptr, nullptr};
    cudaEvent_t done[kRing] = {};
    int64_t next_ticket = 0;
    // work arrays of pkmom_spectra_mu
    void *mu_partials = nullptr;
    size_t mu_partials_bytes = 0;
    void *mu_sums = nullptr;
    size_t mu_sums_bytes = 0;
    // tuning overrides (-1: automatic)
    int tune_tile = -1;
    int tune_list_cap = -1;
    // timing
    bool timing = false;
    std::vector<TimedEvent> pending;
    std::vector<cudaEvent_t> pool;
    double ms[PKMOM_NSTAGES] = {0};
    int64_t calls[PKMOM_NSTAGES] = {0};
};

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

pkmom_status fail(pkmom_ctx *ctx, pkmom_status s, const std::string &msg)
{
    if (ctx) ctx->last_error = msg;
    return s;
}

pkmom_status cuda_fail(pkmom_ctx *ctx, cudaError_t e, const char *where)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(ctx, PKMOM_ENOMEM, std::string(where) + ": " + cudaGetErrorString(e));
    return fail(ctx, PKMOM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define PK_CUDA(call, where)                                  \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
    } while (0)

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

double umin_of(const pkmom_params &p) { return p.kmin_kf > 0 ? p.kmin_kf : 1.0; }
double umax_of(const pkmom_params &p) { return p.kmax_kf > 0 ? p.kmax_kf : 0.5 * p.ng; }

pkmom_status check_params(pkmom_ctx *ctx, const pkmom_params *p)
{
    if (!p) return fail(ctx, PKMOM_EINVAL, "params is NULL");
    if (!(p->box_L > 0) || !std::isfinite(p->box_L)) return fail(ctx, PKMOM_EINVAL, "box_L must be > 0");
    if (p->ng < 16 || p->ng > 1024 || p->ng % 8) return fail(ctx, PKMOM_EINVAL, "ng must be a multiple of 8 in [16, 1024]");
    if (p->order < 1 || p->order > 5) return fail(ctx, PKMOM_EINVAL, "order must be 1..5");
    if (p->precision != PKMOM_F32 && p->precision != PKMOM_F64) return fail(ctx, PKMOM_EINVAL, "bad precision");
    if (p->nbins < 1 || p->nbins > 1024) return fail(ctx, PKMOM_EINVAL, "nbins must be 1..1024");
    const double lo = umin_of(*p), hi = umax_of(*p);
    if (!(hi <= 0.5 * p->ng) || !(lo < hi)) return fail(ctx, PKMOM_EINVAL, "need 0 < kmin_kf < kmax_kf <= ng/2");
    if (p->theta_sn_mode != 0 && p->theta_sn_mode != 1) return fail(ctx, PKMOM_EINVAL, "theta_sn_mode must be 0 or 1");
    if (!std::isfinite(p->theta_scale)) return fail(ctx, PKMOM_EINVAL, "theta_scale must be finite");
    if (p->bl_radius != 0 && (p->bl_radius < 2 || p->bl_radius > 4 || p->order != 4))
        return fail(ctx, PKMOM_EINVAL, "bl_radius must be 0, or 2..4 with order 4");
    return PKMOM_OK;
}

pkmom_status check_catalog(pkmom_ctx *ctx, const pkmom_catalog *c, const pkmom_params *p)
{
    if (!c) return fail(ctx, PKMOM_EINVAL, "catalog is NULL");
    if (c->n < 1 || c->n >= (int64_t(1) << 31)) return fail(ctx, PKMOM_EINVAL, "n must be in [1, 2^31)");
    if (!c->x || !c->y || !c->z || !c->vx || !c->vy || !c->vz) return fail(ctx, PKMOM_EINVAL, "null catalog array");
    if (c->stride < 1) return fail(ctx, PKMOM_EINVAL, "stride must be >= 1");
    if (c->dtype != p->precision) return fail(ctx, PKMOM_EINVAL, "catalog dtype must equal params precision");
    return PKMOM_OK;
}

// How one assignment is laid out: sort-key segment length, deposit tile and scratch.
AssignPlan plan_assign(const pkmom_params &p, int64_t n, int num_sms, int tile_override = -1, int list_override = -1)
{
    AssignPlan pl;
    pl.ng = p.ng;
    pl.order = p.order;
    pl.bl_radius = p.bl_radius;
    pl.prec = p.precision;
    const double cells = double(p.ng) * p.ng * p.ng;
    // deposit tile: the largest listed shape that divides ng, for this precision
    const int pref32[] = {0, 3};
    const int pref64[] = {4, 6};
    const int *pref = p.precision == PKMOM_F32 ? pref32 : pref64;
    pl.tile = pref[1];
    for (int k = 0; k < 2; ++k) {
        int d[3];
        deposit_tile_shape(pref[k], p.precision, d);
        if (d[0] && p.ng % d[0] == 0 && p.ng % d[1] == 0 && p.ng % d[2] == 0) {
            pl.tile = pref[k];
            break;
        }
    }
    // cubic order at half a particle per cell or more: home tiles (each particle deposited
    // once, by the tile owning its cell)
    const double ppc = double(n) / cells;
    if (p.precision == PKMOM_F32 && p.order == 4 && p.bl_radius == 0 && p.ng % 16 == 0 && ppc >= 0.5)
        pl.tile = kHomeTile;
    if (tile_override >= 0) {
        int d[3];
        deposit_tile_shape(tile_override, p.precision, d);
        if (d[0] && p.ng % d[0] == 0 && p.ng % d[1] == 0 && p.ng % d[2] == 0) pl.tile = tile_override;
    }
    // the direct BL deposit is built for the gather tiles 16^3 / 8^3 (FP32) and 8x8x16 / 8^3 (FP64)
    if (p.bl_radius != 0) {
        const bool big = p.ng % 16 == 0;
        pl.tile = p.precision == PKMOM_F32 ? (big ? 0 : 3) : (big ? 4 : 6);
    }
    int td[3];
    deposit_tile_shape(pl.tile, p.precision, td);
    // one sort key per cell keeps each row's particles in z order, which the deposit's
    // lane mapping relies on (coarser z segments measured slower even for sparse
    // catalogues); segments only where 32-bit offsets would not suffice
    int sshift = 0;
    while ((1 << (sshift + 1)) <= td[2] && (p.ng % (1 << (sshift + 1))) == 0 && cells / (1 << sshift) > double(1u << 30))
        ++sshift;
    pl.sshift = sshift;
    if (pl.tile == kHomeTile && sshift != 0) pl.tile = 0;  // home tiles need one sort key per cell
    // sparse catalogues: list each tile's particles in shared memory (room for about
    // twice the expected count of its reach; larger tiles fall back to searching)
    const double reach = double(td[0] + 3) * (td[1] + 3) * (td[2] + 3);
    if (p.precision == PKMOM_F32 && ppc < 0.5) {
        const double want = 2.0 * ppc * reach + 64.0;
        pl.list_cap = static_cast<int>(std::min(8192.0, std::ceil(want / 256.0) * 256.0));
    }
    if (p.precision == PKMOM_F32 && list_override >= 0) pl.list_cap = std::min(list_override, 8192) / 32 * 32;
    pl.nkeys = int64_t(p.ng) * p.ng * (p.ng >> sshift);
    pl.hist_blocks = num_sms * 8;
    pl.scan_blocks = (pl.nkeys + 8191) / 8192;
    const size_t rec = p.precision == PKMOM_F32 ? 32 : 64;
    size_t off = 0;
    pl.off_counts = off;
    off = align_up(off + key_table_bytes(pl.nkeys));
    pl.off_records = off;
    off = align_up(off + size_t(n) * rec);
    pl.off_partials = off;
    off = align_up(off + size_t(pl.hist_blocks) * kMomentWords * 8);
    pl.off_blocksums = off;
    off = align_up(off + size_t(pl.scan_blocks + 1) * 4);
    pl.off_qmax = off;
    off = align_up(off + 4 * sizeof(unsigned));
    if (pl.tile == kHomeTile && p.order == 4) {
        pl.off_halo = off;
        off = align_up(off + home_halo_bytes(p.ng));
    }
    pl.total = off;
    return pl;
}

int device_sms(int device)
{
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0) v = 152;
    return v;
}

cudaEvent_t take_event(pkmom_ctx *ctx)
{
    if (!ctx->pool.empty()) {
        cudaEvent_t e = ctx->pool.back();
        ctx->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// NVTX range names of the stages (host ranges around each stage's launches, for
// profilers: e.g. ncu --nvtx --nvtx-include "pkmom deposit/")
const char *const kStageNames[PKMOM_NSTAGES] = {"pkmom histogram", "pkmom scan", "pkmom scatter", "pkmom deposit",
                                                "pkmom fft", "pkmom binning", "pkmom finalize"};

struct StageTimer {
    pkmom_ctx *ctx;
    int stage;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    bool open = true;
    StageTimer(pkmom_ctx *c, int stg, cudaStream_t st) : ctx(c), stage(stg), s(st)
    {
        nvtxRangePushA(kStageNames[stg]);
        if (ctx->timing) {
            a = take_event(ctx);
            cudaEventRecord(a, s);
        }
    }
    void stop()
    {
        if (ctx->timing && a) {
            cudaEvent_t b = take_event(ctx);
            cudaEventRecord(b, s);
            ctx->pending.push_back({stage, a, b});
            a = nullptr;
        }
        if (open) {
            nvtxRangePop();
            open = false;
        }
    }
    ~StageTimer() { stop(); }
};

pkmom_status get_plan(pkmom_ctx *ctx, int ng, int prec, cufftHandle *out)
{
    for (auto &e : ctx->plans)
        if (e.ng == ng && e.prec == prec) {
            *out = e.h;
            return PKMOM_OK;
        }
    cufftHandle h;
    long long n[3] = {ng, ng, ng};
    long long inembed[3] = {ng, ng, ng + 2};
    long long onembed[3] = {ng, ng, ng / 2 + 1};
    const long long idist = 1LL * ng * ng * (ng + 2);
    const long long odist = 1LL * ng * ng * (ng / 2 + 1);
    size_t work = 0;
    // larger grids: one grid per plan, executed four times (a batch of four 1024^3 grids
    // made cuFFT allocate a 17 GB workspace and run twice as long, measured)
    const int batch = ng <= kFftBatchMaxNg ? 4 : 1;
    cufftResult r = cufftCreate(&h);
    if (r == CUFFT_SUCCESS) {
        r = cufftMakePlanMany64(h, 3, n, inembed, 1, idist, onembed, 1, odist,
                                prec == PKMOM_F32 ? CUFFT_R2C : CUFFT_D2Z, batch, &work);
        if (r != CUFFT_SUCCESS) cufftDestroy(h);
    }
    if (r != CUFFT_SUCCESS) {
        char buf[96];
        std::snprintf(buf, sizeof buf, "cufftPlanMany(ng=%d) failed with code %d", ng, int(r));
        return fail(ctx, r == CUFFT_ALLOC_FAILED ? PKMOM_ENOMEM : PKMOM_ECUFFT, buf);
    }
    ctx->plans.push_back({ng, prec, h, work, batch});
    *out = h;
    return PKMOM_OK;
}

pkmom_status get_tables(pkmom_ctx *ctx, const pkmom_params &p, cudaStream_t s, const SpectraTables **out)
{
    const double lo = umin_of(p), hi = umax_of(p);
    for (auto &t : ctx->tables)
        if (t.ng == p.ng && t.order == p.order && t.direct == (p.bl_radius != 0) && t.nbins == p.nbins &&
            t.umin == lo && t.umax == hi &&
            t.prec == p.precision) {
            *out = &t;
            return PKMOM_OK;
        }
    SpectraTables t;
    cudaError_t e = build_spectra_tables(t, p.ng, p.order, p.bl_radius != 0, p.nbins, lo, hi, p.precision,
                                         ctx->num_sms, s, ctx->st);
    if (e != cudaSuccess) {
        free_spectra_tables(t);
        return cuda_fail(ctx, e, "building spectra tables");
    }
    ctx->tables.push_back(t);
    *out = &ctx->tables.back();
    return PKMOM_OK;
}

pkmom_status ensure(pkmom_ctx *ctx, void **buf, size_t *have, size_t want, const char *what)
{
    if (*have >= want && *buf) return PKMOM_OK;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    cudaError_t e = cudaMalloc(buf, want);
    if (e != cudaSuccess) {
        *buf = nullptr;
        return cuda_fail(ctx, e, what);
    }
    *have = want;
    return PKMOM_OK;
}

// Arguments of a host-catalogue estimate (pkmom_estimate_host and its async form).
pkmom_status check_host_request(pkmom_ctx *ctx, const pkmom_catalog *cat, const pkmom_params *p, const double *out)
{
    pkmom_status s;
    if ((s = check_params(ctx, p)) != PKMOM_OK) return s;
    if ((s = check_catalog(ctx, cat, p)) != PKMOM_OK) return s;
    if (!out) return fail(ctx, PKMOM_EINVAL, "null output");
    const size_t elem = p->precision == PKMOM_F64 ? 8 : 4;
    const char *bx = static_cast<const char *>(cat->x);
    const char *bv = static_cast<const char *>(cat->vx);
    const bool pos_il = cat->stride == 3 && static_cast<const char *>(cat->y) == bx + elem &&
                        static_cast<const char *>(cat->z) == bx + 2 * elem;
    const bool vel_il = cat->stride == 3 && static_cast<const char *>(cat->vy) == bv + elem &&
                        static_cast<const char *>(cat->vz) == bv + 2 * elem;
    if (cat->stride != 1 && !(pos_il && vel_il))
        return fail(ctx, PKMOM_EUNSUPPORTED, "host catalogues must be separate arrays or interleaved (n,3) arrays");
    return PKMOM_OK;
}

// Device staging of a host catalogue: seven blocks of n elements (x, y, z, vx, vy, vz, m).
size_t staging_bytes(int64_t n, size_t elem) { return 7 * align_up(size_t(n) * elem); }

// Copies a host catalogue into the staging area stg on stream st (one cudaMemcpyAsync per
// array; interleaved (n,3) arrays as one block each) and describes the device copy.
pkmom_status stage_catalog(pkmom_ctx *ctx, const pkmom_catalog &cat, size_t elem, char *stg, cudaStream_t st,
                           pkmom_catalog *dcat)
{
    const int64_t n = cat.n;
    const size_t block = align_up(size_t(n) * elem);
    *dcat = cat;
    if (cat.stride == 3) {
        PK_CUDA(cudaMemcpyAsync(stg, cat.x, 3 * size_t(n) * elem, cudaMemcpyHostToDevice, st), "copy positions");
        PK_CUDA(cudaMemcpyAsync(stg + 3 * block, cat.vx, 3 * size_t(n) * elem, cudaMemcpyHostToDevice, st),
                "copy velocities");
        dcat->x = stg, dcat->y = stg + elem, dcat->z = stg + 2 * elem;
        dcat->vx = stg + 3 * block, dcat->vy = stg + 3 * block + elem, dcat->vz = stg + 3 * block + 2 * elem;
    } else {
        const void *src[6] = {cat.x, cat.y, cat.z, cat.vx, cat.vy, cat.vz};
        const void **dst[6] = {&dcat->x, &dcat->y, &dcat->z, &dcat->vx, &dcat->vy, &dcat->vz};
        for (int a = 0; a < 6; ++a) {
            PK_CUDA(cudaMemcpyAsync(stg + a * block, src[a], size_t(n) * elem, cudaMemcpyHostToDevice, st),
                    "copy catalogue");
            *dst[a] = stg + a * block;
        }
    }
    if (cat.mass) {
        PK_CUDA(cudaMemcpyAsync(stg + 6 * block, cat.mass, size_t(n) * elem, cudaMemcpyHostToDevice, st),
                "copy masses");
        dcat->mass = stg + 6 * block;
    }
    return PKMOM_OK;
}

// Returns (and clears) a device-side data error latched by the context's kernels, and in
// checked builds a failed index test of any kernel on this device.
pkmom_status check_error_word(pkmom_ctx *ctx)
{
    // read on a stream of the context's own, so that the read waits for nothing but itself
    // (a copy on the legacy default stream would wait for every blocking stream's work)
    if (!ctx->aux_stream) PK_CUDA(cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking), "aux stream");
    int flag = 0;
    PK_CUDA(cudaMemcpyAsync(&flag, ctx->d_err, sizeof flag, cudaMemcpyDeviceToHost, ctx->aux_stream),
            "read error word");
    PK_CUDA(cudaStreamSynchronize(ctx->aux_stream), "read error word");
    if (flag) {
        PK_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->aux_stream), "clear error word");
        PK_CUDA(cudaStreamSynchronize(ctx->aux_stream), "clear error word");
        return fail(ctx, PKMOM_EDATA, "catalogue held non-finite or out-of-range positions (|x ng/L| >= 2^30)");
    }
    if (PKMOM_CHECKED) {
        const unsigned w = take_check_word_assign() | take_check_word_spectra();
        if (w) {
            char buf[96];
            std::snprintf(buf, sizeof buf, "index out of range in the checked build (test codes 0x%x)", w);
            return fail(ctx, PKMOM_EDATA, buf);
        }
    }
    return PKMOM_OK;
}

}  // namespace

extern "C" {

void pkmom_params_default(pkmom_params *p, double box_L, int ng, int nbins)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->box_L = box_L;
    p->ng = ng;
    p->order = 4;
    p->precision = PKMOM_F32;
    p->nbins = nbins;
    p->kmin_kf = 1.0;
    p->kmax_kf = 0.5 * ng;
    p->theta_scale = 1.0;
    p->subtract_shot_noise = 1;
    p->bulk = 1;
    p->theta_sn_mode = 0;
}

const char *pkmom_strerror(pkmom_status s)
{
    switch (s) {
    case PKMOM_OK: return "ok";
    case PKMOM_EINVAL: return "invalid argument";
    case PKMOM_ENOMEM: return "device out of memory";
    case PKMOM_ECUDA: return "CUDA error";
    case PKMOM_ECUFFT: return "cuFFT error";
    case PKMOM_ETIMEOUT: return "device wait timed out";
    case PKMOM_EUNSUPPORTED: return "unsupported";
    case PKMOM_ESCRATCH: return "scratch buffer too small";
    case PKMOM_EDATA: return "non-finite or out-of-range particle positions";
    }
    return "unknown status";
}

const char *pkmom_last_error(const pkmom_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

pkmom_status pkmom_create(pkmom_ctx **out, int device)
{
    if (!out) return PKMOM_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return PKMOM_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return PKMOM_ECUDA;
    auto *ctx = new pkmom_ctx;
    ctx->device = device;
    ctx->num_sms = device_sms(device);
    cudaError_t e = cudaMalloc(&ctx->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        delete ctx;
        return e == cudaErrorMemoryAllocation ? PKMOM_ENOMEM : PKMOM_ECUDA;
    }
    *out = ctx;
    return PKMOM_OK;
}

pkmom_status pkmom_destroy(pkmom_ctx *ctx)
{
    if (!ctx) return PKMOM_EINVAL;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto &p : ctx->plans) cufftDestroy(p.h);
    for (auto &t : ctx->tables) free_spectra_tables(t);
    for (auto &t : ctx->pending) cudaEventDestroy(t.a), cudaEventDestroy(t.b);
    for (auto e : ctx->pool) cudaEventDestroy(e);
    cudaFree(ctx->grids);
    cudaFree(ctx->scratch);
    cudaFree(ctx->moments);
    cudaFree(ctx->out_dev);
    cudaFree(ctx->staging);
    for (int k = 0; k < 2; ++k) {
        cudaFree(ctx->aslot[k]);
        if (ctx->slot_copied[k]) cudaEventDestroy(ctx->slot_copied[k]);
        if (ctx->slot_free[k]) cudaEventDestroy(ctx->slot_free[k]);
    }
    for (auto e : ctx->done)
        if (e) cudaEventDestroy(e);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
    cudaFree(ctx->mu_partials);
    cudaFree(ctx->mu_sums);
    cudaFree(ctx->d_err);
    delete ctx;
    return PKMOM_OK;
}

size_t pkmom_grid_bytes(int ng, int precision)
{
    if (ng <= 0) return 0;
    return size_t(4) * ng * ng * (ng + 2) * (precision == PKMOM_F64 ? 8 : 4);
}

size_t pkmom_assign_scratch_bytes(const pkmom_params *p, int64_t n)
{
    if (!p || check_params(nullptr, p) != PKMOM_OK || n < 1) return 0;
    int dev = 0;
    cudaGetDevice(&dev);
    return plan_assign(*p, n, device_sms(dev)).total;
}

size_t pkmom_footprint_bytes(const pkmom_params *p, int64_t n)
{
    if (!p || check_params(nullptr, p) != PKMOM_OK || n < 1) return 0;
    const size_t elem = p->precision == PKMOM_F64 ? 8 : 4;
    const size_t grids = pkmom_grid_bytes(p->ng, p->precision);
    const size_t staging = size_t(n) * 7 * elem;
    // cuFFT's in-place workspace: at most one grid's worth per grid in the plan's batch
    const size_t fft_work = p->ng <= kFftBatchMaxNg ? grids : grids / 4;
    return grids + fft_work + pkmom_assign_scratch_bytes(p, n) + staging + (size_t(64) << 10);
}

pkmom_status pkmom_assign(pkmom_ctx *ctx, const pkmom_catalog *cat, const pkmom_params *p, void *grids,
                          void *moments_dev, void *scratch, size_t scratch_bytes, void *stream)
{
    if (!ctx) return PKMOM_EINVAL;
    pkmom_status s;
    if ((s = check_params(ctx, p)) != PKMOM_OK) return s;
    if ((s = check_catalog(ctx, cat, p)) != PKMOM_OK) return s;
    if (!grids || !moments_dev || !scratch) return fail(ctx, PKMOM_EINVAL, "null grids, moments or scratch");
    if (reinterpret_cast<uintptr_t>(grids) % 16 || reinterpret_cast<uintptr_t>(scratch) % 16)
        return fail(ctx, PKMOM_EINVAL, "grids and scratch must be 16-byte aligned");
    PK_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    const AssignPlan pl = plan_assign(*p, cat->n, ctx->num_sms, ctx->tune_tile, ctx->tune_list_cap);
    if (scratch_bytes < pl.total) return fail(ctx, PKMOM_ESCRATCH, "scratch smaller than pkmom_assign_scratch_bytes");
    cudaStream_t st = as_stream(stream);
    {
        StageTimer t(ctx, PKMOM_STAGE_HIST, st);
        PK_CUDA(launch_hist_moments(*cat, pl, p->box_L, scratch, ctx->d_err, st, ctx->st), "histogram");
    }
    {
        StageTimer t(ctx, PKMOM_STAGE_SCAN, st);
        PK_CUDA(launch_scan(pl, scratch, st, ctx->st), "scan");
    }
    {
        StageTimer t(ctx, PKMOM_STAGE_SCATTER, st);
        PK_CUDA(launch_scatter(*cat, pl, p->box_L, scratch, st, ctx->st), "scatter and moments");
        PK_CUDA(launch_moments_final(pl, cat->n, scratch, static_cast<double *>(moments_dev), st, ctx->st),
                "moments");
    }
    {
        StageTimer t(ctx, PKMOM_STAGE_DEPOSIT, st);
        PK_CUDA(launch_deposit(pl, scratch, grids, st, ctx->st), "deposit");
    }
    return PKMOM_OK;
}

pkmom_status pkmom_fft(pkmom_ctx *ctx, const pkmom_params *p, void *grids, void *stream)
{
    if (!ctx) return PKMOM_EINVAL;
    pkmom_status s;
    if ((s = check_params(ctx, p)) != PKMOM_OK) return s;
    if (!grids) return fail(ctx, PKMOM_EINVAL, "null grids");
    PK_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    cufftHandle h;
    if ((s = get_plan(ctx, p->ng, p->precision, &h)) != PKMOM_OK) return s;
    cudaStream_t st = as_stream(stream);
    if (cufftSetStream(h, st) != CUFFT_SUCCESS) return fail(ctx, PKMOM_ECUFFT, "cufftSetStream failed");
    StageTimer t(ctx, PKMOM_STAGE_FFT, st);
    const size_t gelems = size_t(p->ng) * p->ng * (p->ng + 2);
    const int execs = p->ng <= kFftBatchMaxNg ? 1 : 4;  // the plan's batch covers 4 / execs grids
    for (int f = 0; f < execs; ++f) {
        cufftResult r;
        if (p->precision == PKMOM_F32) {
            auto *g = static_cast<cufftReal *>(grids) + f * gelems;
            r = cufftExecR2C(h, g, reinterpret_cast<cufftComplex *>(g));
        } else {
            auto *g = static_cast<cufftDoubleReal *>(grids) + f * gelems;
            r = cufftExecD2Z(h, g, reinterpret_cast<cufftDoubleComplex *>(g));
        }
        if (r != CUFFT_SUCCESS) return fail(ctx, PKMOM_ECUFFT, "cufftExec failed with code " + std::to_string(int(r)));
    }
    return PKMOM_OK;
}

pkmom_status pkmom_spectra(pkmom_ctx *ctx, const pkmom_params *p, const void *grids, const void *moments_dev,
                           double *out_dev, void *stream)
{
    if (!ctx) return PKMOM_EINVAL;
    pkmom_status s;
    if ((s = check_params(ctx, p)) != PKMOM_OK) return s;
    if (!grids || !moments_dev || !out_dev) return fail(ctx, PKMOM_EINVAL, "null grids, moments or output");
    PK_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t st = as_stream(stream);
    const SpectraTables *t = nullptr;
    if ((s = get_tables(ctx, *p, st, &t)) != PKMOM_OK) return s;
    {
        StageTimer tm(ctx, PKMOM_STAGE_BIN, st);
        PK_CUDA(launch_bin_shells(*t, grids, static_cast<const double *>(moments_dev), st, ctx->st), "binning");
    }
    {
        StageTimer tm(ctx, PKMOM_STAGE_FINAL, st);
        PK_CUDA(launch_finalize(*t, *p, static_cast<const double *>(moments_dev), out_dev, st, ctx->st, true),
                "finalize");
    }
    return PKMOM_OK;
}

pkmom_status pkmom_spectra_mu(pkmom_ctx *ctx, const pkmom_params *p, const void *grids, const void *moments_dev,
                              const double *direction, int nmu, double *out_dev, void *stream)
{
    if (!ctx) return PKMOM_EINVAL;
    pkmom_status s;
    if ((s = check_params(ctx, p)) != PKMOM_OK) return s;
    if (!grids || !moments_dev || !out_dev) return fail(ctx, PKMOM_EINVAL, "null grids, moments or output");
    if (nmu < 1 || nmu > 64) return fail(ctx, PKMOM_EINVAL, "nmu must be 1..64");
    double dir[3];
    if (direction) {
        const double nrm = std::sqrt(direction[0] * direction[0] + direction[1] * direction[1] +
                                     direction[2] * direction[2]);
        if (!(nrm > 0) || !std::isfinite(nrm)) return fail(ctx, PKMOM_EINVAL, "direction must be finite and non-zero");
        for (int a = 0; a < 3; ++a) dir[a] = direction[a] / nrm;
    }
    PK_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t st = as_stream(stream);
    const SpectraTables *t = nullptr;
    if ((s = get_tables(ctx, *p, st, &t)) != PKMOM_OK) return s;
    if ((s = ensure(ctx, &ctx->mu_partials, &ctx->mu_partials_bytes, spectra_mu_partial_bytes(p->ng, p->nbins, nmu),
                    "mu partials")) != PKMOM_OK)
        return s;
    if ((s = ensure(ctx, &ctx->mu_sums, &ctx->mu_sums_bytes, spectra_mu_sum_bytes(p->nbins, nmu), "mu sums")) !=
        PKMOM_OK)
        return s;
    StageTimer tm(ctx, PKMOM_STAGE_BIN, st);
    PK_CUDA(launch_spectra_mu(*t, *p, grids, static_cast<const double *>(moments_dev), direction ? dir : nullptr, nmu,
                              static_cast<double *>(ctx->mu_partials), static_cast<double *>(ctx->mu_sums), out_dev,
                              st, ctx->st),
            "mu binning");
    return PKMOM_OK;
}

pkmom_status pkmom_estimate(pkmom_ctx *ctx, const pkmom_catalog *cat, const pkmom_params *p, double *out_dev,
                            void *stream)
{
    if (!ctx) return PKMOM_EINVAL;
    pkmom_status s;
    if ((s = check_params(ctx, p)) != PKMOM_OK) return s;
    if ((s = check_catalog(ctx, cat, p)) != PKMOM_OK) return s;
    if (!out_dev) return fail(ctx, PKMOM_EINVAL, "null output");
    PK_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    const AssignPlan pl = plan_assign(*p, cat->n, ctx->num_sms, ctx->tune_tile, ctx->tune_list_cap);
    if ((s = ensure(ctx, &ctx->grids, &ctx->grids_bytes, pkmom_grid_bytes(p->ng, p->precision), "grids")) != PKMOM_OK)
        return s;
    if ((s = ensure(ctx, &ctx->scratch, &ctx->scratch_bytes, pl.total, "scratch")) != PKMOM_OK) return s;
    if (!ctx->moments) PK_CUDA(cudaMalloc(reinterpret_cast<void **>(&ctx->moments), kMomentWords * 8), "moments");
    if ((s = pkmom_assign(ctx, cat, p, ctx->grids, ctx->moments, ctx->scratch, ctx->scratch_bytes, stream)) != PKMOM_OK)
        return s;
    if ((s = pkmom_fft(ctx, p, ctx->grids, stream)) != PKMOM_OK) return s;
    return pkmom_spectra(ctx, p, ctx->grids, ctx->moments, out_dev, stream);
}

pkmom_status pkmom_estimate_host(pkmom_ctx *ctx, const pkmom_catalog *cat, const pkmom_params *p, double *out_host,
                                 void *stream)
{
    if (!ctx) return PKMOM_EINVAL;
    pkmom_status s;
    if ((s = check_host_request(ctx, cat, p, out_host)) != PKMOM_OK) return s;
    PK_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    const size_t elem = p->precision == PKMOM_F64 ? 8 : 4;
    if ((s = ensure(ctx, &ctx->staging, &ctx->staging_bytes, staging_bytes(cat->n, elem), "staging")) != PKMOM_OK)
        return s;
    const size_t out_bytes = size_t(PKMOM_NROWS) * p->nbins * sizeof(double);
    if ((s = ensure(ctx, reinterpret_cast<void **>(&ctx->out_dev), &ctx->out_bytes, out_bytes, "output")) != PKMOM_OK)
        return s;
    cudaStream_t st = as_stream(stream);
    pkmom_catalog dcat;
    if ((s = stage_catalog(ctx, *cat, elem, static_cast<char *>(ctx->staging), st, &dcat)) != PKMOM_OK) return s;
    if ((s = pkmom_estimate(ctx, &dcat, p, ctx->out_dev, stream)) != PKMOM_OK) return s;
    PK_CUDA(cudaMemcpyAsync(out_host, ctx->out_dev, out_bytes, cudaMemcpyDeviceToHost, st), "copy result");
    return pkmom_sync(ctx, stream);
}

pkmom_status pkmom_estimate_host_async(pkmom_ctx *ctx, const pkmom_catalog *cat, const pkmom_params *p,
                                       double *out_host, void *stream, int64_t *ticket)
{
    if (!ctx) return PKMOM_EINVAL;
    pkmom_status s;
    if ((s = check_host_request(ctx, cat, p, out_host)) != PKMOM_OK) return s;
    if (!ticket) return fail(ctx, PKMOM_EINVAL, "null ticket");
    PK_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    const size_t elem = p->precision == PKMOM_F64 ? 8 : 4;
    cudaStream_t st = as_stream(stream);
    if (!ctx->copy_stream) {
        PK_CUDA(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking), "copy stream");
        for (int k = 0; k < 2; ++k) {
            PK_CUDA(cudaEventCreateWithFlags(&ctx->slot_copied[k], cudaEventDisableTiming), "slot event");
            PK_CUDA(cudaEventCreateWithFlags(&ctx->slot_free[k], cudaEventDisableTiming), "slot event");
            PK_CUDA(cudaEventRecord(ctx->slot_free[k], ctx->copy_stream), "slot event");
        }
        for (auto &e : ctx->done) PK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "ticket event");
    }
    const int64_t t = ctx->next_ticket;
    const int k = static_cast<int>(t & 1);
    const size_t want = staging_bytes(cat->n, elem);
    if (ctx->aslot_bytes[k] < want) {
        // a larger slot: nothing may still read or fill the old one
        PK_CUDA(cudaStreamSynchronize(ctx->copy_stream), "copy stream synchronize");
        PK_CUDA(cudaEventSynchronize(ctx->slot_free[k]), "slot event synchronize");
        if ((s = ensure(ctx, &ctx->aslot[k], &ctx->aslot_bytes[k], want, "staging slot")) != PKMOM_OK) return s;
    }
    const size_t out_bytes = size_t(PKMOM_NROWS) * p->nbins * sizeof(double);
    if (ctx->out_bytes < out_bytes) {
        PK_CUDA(cudaStreamSynchronize(st), "stream synchronize");
        if ((s = ensure(ctx, reinterpret_cast<void **>(&ctx->out_dev), &ctx->out_bytes, out_bytes, "output")) !=
            PKMOM_OK)
            return s;
    }
    // fill slot k on the copy stream once the estimate that last read it has moved on
    PK_CUDA(cudaStreamWaitEvent(ctx->copy_stream, ctx->slot_free[k], 0), "copy stream wait");
    pkmom_catalog dcat;
    if ((s = stage_catalog(ctx, *cat, elem, static_cast<char *>(ctx->aslot[k]), ctx->copy_stream, &dcat)) != PKMOM_OK)
        return s;
    PK_CUDA(cudaEventRecord(ctx->slot_copied[k], ctx->copy_stream), "slot event");
    // the estimate on the caller's stream: assign reads the slot, then frees it
    PK_CUDA(cudaStreamWaitEvent(st, ctx->slot_copied[k], 0), "stream wait");
    const AssignPlan pl = plan_assign(*p, cat->n, ctx->num_sms, ctx->tune_tile, ctx->tune_list_cap);
    if ((s = ensure(ctx, &ctx->grids, &ctx->grids_bytes, pkmom_grid_bytes(p->ng, p->precision), "grids")) != PKMOM_OK)
        return s;
    if ((s = ensure(ctx, &ctx->scratch, &ctx->scratch_bytes, pl.total, "scratch")) != PKMOM_OK) return s;
    if (!ctx->moments) PK_CUDA(cudaMalloc(reinterpret_cast<void **>(&ctx->moments), kMomentWords * 8), "moments");
    if ((s = pkmom_assign(ctx, &dcat, p, ctx->grids, ctx->moments, ctx->scratch, ctx->scratch_bytes, stream)) !=
        PKMOM_OK)
        return s;
    PK_CUDA(cudaEventRecord(ctx->slot_free[k], st), "slot event");
    if ((s = pkmom_fft(ctx, p, ctx->grids, stream)) != PKMOM_OK) return s;
    if ((s = pkmom_spectra(ctx, p, ctx->grids, ctx->moments, ctx->out_dev, stream)) != PKMOM_OK) return s;
    PK_CUDA(cudaMemcpyAsync(out_host, ctx->out_dev, out_bytes, cudaMemcpyDeviceToHost, st), "copy result");
    PK_CUDA(cudaEventRecord(ctx->done[t % pkmom_ctx::kRing], st), "ticket event");
    ctx->next_ticket = t + 1;
    *ticket = t;
    return PKMOM_OK;
}

pkmom_status pkmom_wait(pkmom_ctx *ctx, int64_t ticket)
{
    if (!ctx) return PKMOM_EINVAL;
    if (ticket < 0 || ticket >= ctx->next_ticket) return fail(ctx, PKMOM_EINVAL, "unknown ticket");
    PK_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    // the ring slot holds this ticket or a later one of the same stream: waiting on it
    // waits at least until this ticket's result is on the host
    PK_CUDA(cudaEventSynchronize(ctx->done[ticket % pkmom_ctx::kRing]), "ticket synchronize");
    return check_error_word(ctx);
}

namespace {
struct BatchLayout {
    size_t counter = 0, total = 0;
    std::vector<size_t> partials, sums;  // offsets per item (FP32 items), else unused
};
BatchLayout batch_layout(int n, const pkmom_batch_item *items)
{
    BatchLayout L;
    size_t off = align_up(sizeof(unsigned long long));
    L.partials.assign(n, 0);
    L.sums.assign(n, 0);
    for (int k = 0; k < n; ++k) {
        const pkmom_params &p = items[k].p;
        if (p.precision != PKMOM_F32) continue;
        L.partials[k] = off;
        off = align_up(off + size_t(p.ng) * p.nbins * kBinVals * sizeof(double));
        L.sums[k] = off;
        off = align_up(off + size_t(kBinVals) * p.nbins * sizeof(double));
    }
    L.total = off;
    return L;
}
}  // namespace

size_t pkmom_batch_work_bytes(int n, const pkmom_batch_item *items)
{
    if (n < 1 || n > PKMOM_BATCH_MAX || !items) return 0;
    for (int k = 0; k < n; ++k)
        if (check_params(nullptr, &items[k].p) != PKMOM_OK) return 0;
    return batch_layout(n, items).total;
}

pkmom_status pkmom_estimate_batch(pkmom_ctx *ctx, int n, const pkmom_batch_item *items, void *work,
                                  size_t work_bytes, void *stream)
{
    if (!ctx) return PKMOM_EINVAL;
    if (n < 1 || n > PKMOM_BATCH_MAX || !items) return fail(ctx, PKMOM_EINVAL, "need 1..PKMOM_BATCH_MAX items");
    if (!work || reinterpret_cast<uintptr_t>(work) % 16) return fail(ctx, PKMOM_EINVAL, "work must be 16-byte aligned");
    pkmom_status s;
    std::vector<AssignPlan> plans(n);
    std::vector<const SpectraTables *> tabs(n, nullptr);
    PK_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t st = as_stream(stream);
    for (int k = 0; k < n; ++k) {
        const pkmom_batch_item &it = items[k];
        if ((s = check_params(ctx, &it.p)) != PKMOM_OK) return s;
        if ((s = check_catalog(ctx, &it.cat, &it.p)) != PKMOM_OK) return s;
        if (!it.grids || !it.moments_dev || !it.scratch || !it.out_dev)
            return fail(ctx, PKMOM_EINVAL, "null grids, moments, scratch or output in a batch item");
        if (reinterpret_cast<uintptr_t>(it.grids) % 16 || reinterpret_cast<uintptr_t>(it.scratch) % 16)
            return fail(ctx, PKMOM_EINVAL, "grids and scratch must be 16-byte aligned");
        if (it.deposit_tile >= deposit_tile_count() || it.list_cap > 8192)
            return fail(ctx, PKMOM_EINVAL, "bad tuning values in a batch item");
        plans[k] = plan_assign(it.p, it.cat.n, ctx->num_sms, it.deposit_tile < 0 ? -1 : it.deposit_tile,
                               it.list_cap < 0 ? -1 : it.list_cap);
        if (it.scratch_bytes < plans[k].total)
            return fail(ctx, PKMOM_ESCRATCH, "scratch of a batch item smaller than its assignment needs");
        cufftHandle h;
        if ((s = get_plan(ctx, it.p.ng, it.p.precision, &h)) != PKMOM_OK) return s;
        if ((s = get_tables(ctx, it.p, st, &tabs[k])) != PKMOM_OK) return s;
    }
    const BatchLayout L = batch_layout(n, items);
    if (work_bytes < L.total) return fail(ctx, PKMOM_ESCRATCH, "work buffer smaller than pkmom_batch_work_bytes");
    char *wk = static_cast<char *>(work);
    auto *counter = reinterpret_cast<unsigned long long *>(wk + L.counter);
    {
        StageTimer t(ctx, PKMOM_STAGE_HIST, st);
        for (int k = 0; k < n; ++k)
            PK_CUDA(launch_hist_moments(items[k].cat, plans[k], items[k].p.box_L, items[k].scratch, ctx->d_err, st,
                                        ctx->st),
                    "histogram");
    }
    {
        StageTimer t(ctx, PKMOM_STAGE_SCAN, st);
        for (int k = 0; k < n; ++k) PK_CUDA(launch_scan(plans[k], items[k].scratch, st, ctx->st), "scan");
    }
    {
        StageTimer t(ctx, PKMOM_STAGE_SCATTER, st);
        for (int k = 0; k < n; ++k) {
            PK_CUDA(launch_scatter(items[k].cat, plans[k], items[k].p.box_L, items[k].scratch, st, ctx->st),
                    "scatter and moments");
            PK_CUDA(launch_moments_final(plans[k], items[k].cat.n, items[k].scratch,
                                         static_cast<double *>(items[k].moments_dev), st, ctx->st),
                    "moments");
        }
    }
    {
        StageTimer t(ctx, PKMOM_STAGE_DEPOSIT, st);
        FxBatch fb{};
        for (int k = 0; k < n; ++k) {
            if (batchable_deposit(plans[k])) fb.job[fb.n++] = deposit_job(plans[k], items[k].scratch, items[k].grids);
            else PK_CUDA(launch_deposit(plans[k], items[k].scratch, items[k].grids, st, ctx->st), "deposit");
        }
        if (fb.n) PK_CUDA(launch_deposit_batch(fb, counter, ctx->num_sms, st, ctx->st), "batched deposit");
    }
    for (int k = 0; k < n; ++k)
        if ((s = pkmom_fft(ctx, &items[k].p, items[k].grids, stream)) != PKMOM_OK) return s;
    {
        StageTimer t(ctx, PKMOM_STAGE_BIN, st);
        BinBatch bb{};
        bb.counter = reinterpret_cast<unsigned *>(counter);  // the deposit's counter, free again
        std::vector<const SpectraTables *> btabs;
        std::vector<const pkmom_params *> bpar;
        std::vector<double *> bsums, bout;
        for (int k = 0; k < n; ++k) {
            const pkmom_batch_item &it = items[k];
            if (it.p.precision != PKMOM_F32) {
                PK_CUDA(launch_bin_shells(*tabs[k], it.grids, static_cast<const double *>(it.moments_dev), st,
                                          ctx->st),
                        "binning");
                PK_CUDA(launch_finalize(*tabs[k], it.p, static_cast<const double *>(it.moments_dev), it.out_dev, st,
                                        ctx->st, true),
                        "finalize");
                continue;
            }
            BinJob &j = bb.job[bb.n++];
            j.grids = it.grids;
            j.mom = static_cast<const double *>(it.moments_dev);
            j.thresh = tabs[k]->thresh;
            j.gf = static_cast<const float *>(tabs[k]->g_full);
            j.gh = static_cast<const float *>(tabs[k]->g_half);
            j.partials = reinterpret_cast<double *>(wk + L.partials[k]);
            j.ng = it.p.ng;
            j.nbins = it.p.nbins;
            btabs.push_back(tabs[k]);
            bpar.push_back(&it.p);
            bsums.push_back(reinterpret_cast<double *>(wk + L.sums[k]));
            bout.push_back(it.out_dev);
        }
        if (bb.n)
            PK_CUDA(launch_bin_batch(bb, btabs.data(), bpar.data(), bsums.data(), bout.data(), ctx->num_sms, st,
                                     ctx->st),
                    "batched binning");
    }
    return PKMOM_OK;
}

pkmom_status pkmom_sync(pkmom_ctx *ctx, void *stream)
{
    if (!ctx) return PKMOM_EINVAL;
    PK_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    PK_CUDA(cudaStreamSynchronize(as_stream(stream)), "stream synchronize");
    return check_error_word(ctx);
}

pkmom_status pkmom_timing_enable(pkmom_ctx *ctx, int on)
{
    if (!ctx) return PKMOM_EINVAL;
    ctx->timing = on != 0;
    return PKMOM_OK;
}

pkmom_status pkmom_timing_read(pkmom_ctx *ctx, double ms[PKMOM_NSTAGES], int64_t calls[PKMOM_NSTAGES])
{
    if (!ctx || !ms || !calls) return PKMOM_EINVAL;
    for (auto &t : ctx->pending) {
        PK_CUDA(cudaEventSynchronize(t.b), "event synchronize");
        float v = 0.f;
        PK_CUDA(cudaEventElapsedTime(&v, t.a, t.b), "event elapsed");
        ctx->ms[t.stage] += v;
        ctx->calls[t.stage] += 1;
        ctx->pool.push_back(t.a);
        ctx->pool.push_back(t.b);
    }
    ctx->pending.clear();
    for (int k = 0; k < PKMOM_NSTAGES; ++k) {
        ms[k] = ctx->ms[k];
        calls[k] = ctx->calls[k];
        ctx->ms[k] = 0;
        ctx->calls[k] = 0;
    }
    return PKMOM_OK;
}

int64_t pkmom_kernel_launches(const pkmom_ctx *ctx) { return ctx ? ctx->st.launches : 0; }

int pkmom_checked(void) { return PKMOM_CHECKED; }

pkmom_status pkmom_checked_selftest(pkmom_ctx *ctx, void *stream)
{
    if (!ctx) return PKMOM_EINVAL;
#if PKMOM_CHECKED
    PK_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    PK_CUDA(launch_check_selftest(as_stream(stream)), "self-test");
    ctx->st.launches++;
    return PKMOM_OK;
#else
    (void)stream;
    return fail(ctx, PKMOM_EUNSUPPORTED, "not a checked build");
#endif
}

size_t pkmom_context_bytes(const pkmom_ctx *ctx)
{
    if (!ctx) return 0;
    size_t b = sizeof(int) + ctx->grids_bytes + ctx->scratch_bytes + ctx->out_bytes + ctx->staging_bytes +
               ctx->aslot_bytes[0] + ctx->aslot_bytes[1] + ctx->mu_partials_bytes + ctx->mu_sums_bytes + (ctx->moments ? kMomentWords * 8 : 0);
    for (const auto &p : ctx->plans) b += p.work;
    for (const auto &t : ctx->tables) b += t.bytes;
    return b;
}

pkmom_status pkmom_set_tuning(pkmom_ctx *ctx, int deposit_tile, int list_cap)
{
    if (!ctx) return PKMOM_EINVAL;
    if (deposit_tile >= deposit_tile_count() || list_cap > 8192) return fail(ctx, PKMOM_EINVAL, "bad tuning values");
    ctx->tune_tile = deposit_tile < 0 ? -1 : deposit_tile;
    ctx->tune_list_cap = list_cap < 0 ? -1 : list_cap;
    return PKMOM_OK;
}

size_t pkmom_assign_scratch_bytes_tuned(const pkmom_ctx *ctx, const pkmom_params *p, int64_t n)
{
    if (!ctx || !p || check_params(nullptr, p) != PKMOM_OK || n < 1) return 0;
    return plan_assign(*p, n, ctx->num_sms, ctx->tune_tile, ctx->tune_list_cap).total;
}

}  // extern "C"
